"""bench.py keeps its output contract on a GPU: one JSON line with the
metric, the timing and the evidence fields (roofline with its HBM, FP32 and
L2 roofs, the oracle baseline, the end-to-end figure, the clocks and the
launch count), from a short run with the extra fields switched off."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_prints_one_contract_line():
    cmd = [sys.executable, "bench.py", "--steps", "3", "--warmup", "3", "--batch", "1", "--serve-seconds", "0",
           "--adam-steps", "0", "--tc-steps", "0", "--paper-steps", "0", "--mixed-steps", "0", "--small-steps", "0",
           "--cpu-budget-s", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["metric"].startswith("ms per 1024") and d["unit"] == "ms/mask" and d["higher_is_better"] is False
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["dtype"] == "f32" and d["data"] == "synthetic" and "workload" in d["config"]
    assert d["vs_baseline"] is None and d["scaling"] == "weak"
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"],
                                                                                              rel=1e-3)
    assert rf["l2"]["peak"] > 0 and 0 < rf["l2"]["frac"] < 2 and 0 < rf["alu_frac"] < 2
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1 and cb["unit"] == "ms/mask"
    e2e = d["e2e"]
    assert e2e["value"] >= d["value"] * 0.9 and e2e["h2d_bytes_per_step"] == 2 * 1024 * 1024 * 4
    assert e2e["d2h_bytes_per_step"] >= 1024 * 1024 * 4
    assert d["gpu_launches"] == 3
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
