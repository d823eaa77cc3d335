"""Compile the CUDA library (libgs_gb300.so) in-tree for sm_103a.

The translation units are compiled in parallel with nvcc and linked into one
shared library with the CUDA runtime linked statically. Nothing here runs on
the GPU; the same command works on a machine without one.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB_NAME = "libgs_gb300.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)

# (source, object name, extra flags): the iteration kernel is compiled once per
# log2(nx) so that the 64 size instantiations build in parallel.
SOURCES = [("gs_api.cu", "gs_api", []), ("gs_launch.cu", "gs_launch", []), ("gs_noalloc.cu", "gs_noalloc", []), ("gs_loss_inst.cu", "gs_loss_inst", []), ("gs_tc_inst.cu", "gs_tc_inst", []), ("gs_tc5_inst.cu", "gs_tc5_inst", []),
    ("gs_general_inst.cu", "gs_general_inst", []),
    ("gs_serve.cu", "gs_serve", []),
    ("gs_mixed_inst.cu", "gs_mixed_inst", []), ("gs_adam.cu", "gs_adam", []), ("gs_peak.cu", "gs_peak", []), ("gs_notify.cu", "gs_notify", []),
    ("gs_small_inst.cu", "gs_small_inst", [])] + [
    ("gs_inst.cu", f"gs_inst_lx{lx}", [f"-DGS_LX={lx}"]) for lx in range(5, 13)
] + [("gs_rg_inst.cu", f"gs_rg_inst_{nx}", [f"-DGS_RG_NX={nx}"]) for nx in (600, 768, 800, 1024)]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [
    "-O3",
    "-lineinfo",
    "-std=c++17",
    "-Xcompiler",
    "-fPIC",
    "-Xcompiler",
    "-fno-strict-aliasing",
    "--expt-relaxed-constexpr",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgs_gb300.so")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Build the library if needed; return its path."""
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + GENCODE + ["-I", INCLUDE, "-I", CSRC] + list(extra_flags or [])
    objs = []

    def compile_one(item):
        src, name, defs = item
        obj = os.path.join(OUT_DIR, name + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + flags + defs
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + ".tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + GENCODE + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true", help="print register/smem usage")
    a = ap.parse_args()
    extra = ["-Xptxas", "-v"] if a.ptxas_info else None
    print(build(force=a.force or a.ptxas_info, verbose=a.verbose or a.ptxas_info, extra_flags=extra))
