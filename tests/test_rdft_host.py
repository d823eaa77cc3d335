"""The register DFTs of the general-grid kernel (5-smooth lengths up to 32,
mixed radix in registers with compiler-evaluated twiddles) checked on the
host: tests/rdft_host.cu is built as host code with nvcc and compares rdft<N>
with the direct DFT in double, and the compile-time cos/sin with the C
library. No GPU is needed."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_register_dfts_match_direct_dft(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "rdft_host"
    src = os.path.join(ROOT, "tests", "rdft_host.cu")
    inc = os.path.join(ROOT, "paper_1302_0120_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", inc, "-I", os.path.join(ROOT, "include"), src, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict(line.split() for line in out if line.strip())
    assert len(vals) == 14
    for n, e in vals.items():
        if n == "cs":
            assert float(e) <= 1e-14, e  # double rounding of the angle and of the C library only
        else:
            assert float(e) <= 2e-7, (n, e)  # FP32 rounding of about log2(n) stages
