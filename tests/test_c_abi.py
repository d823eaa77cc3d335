"""The boundary is plain C: include/gs.h compiles as C11 with every warning
an error, and a C program links against the library and calls the entry
points that need no GPU (error strings, workspace sizes, argument checks)."""

import os
import shutil
import subprocess

import pytest

from paper_1302_0120_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stddef.h>
#include "gs.h"

int main(void) {
  gs_ctx* c = (gs_ctx*)0;
  size_t a = gs_workspace_bytes(1024, 1024, GS_FINAL_RESIDUAL);
  size_t b = gs_workspace_bytes_batched(1024, 1024, 8, GS_FINAL_RESIDUAL);
  size_t bad = gs_workspace_bytes(1000, 7, 0u);
  /* argument checks that answer before any CUDA call */
  int e1 = gs_create(&c, 1021, 1024, 0u, NULL); /* 1021 is prime: not a valid side */
  int e2 = gs_run(NULL, NULL, NULL, 1, NULL, NULL, NULL);
  int e3 = gs_destroy(NULL);
  printf("%s|%s|%zu|%zu|%zu|%d|%d|%d|%d\n", gs_strerror(GS_ETIMEOUT), gs_strerror(GS_ENUMERIC), a, b, bad, e1,
         e2, e3, c == NULL);
  return 0;
}
"""


def test_header_compiles_as_c_and_links(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    so = build_lib.build()
    libdir = os.path.dirname(so)
    src = tmp_path / "probe.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "probe"
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Wpedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-L", libdir, "-lgs_gb300", f"-Wl,-rpath,{libdir}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    msg_t, msg_n, a, b, bad, e1, e2, e3, still_null = r.stdout.strip().split("|")
    assert msg_t == "device-side wait timed out"
    assert msg_n == "target intensity is non-finite, negative or zero"
    assert int(a) > 12 * 1024 * 1024 and int(b) > 8 * int(a) // 2 and int(bad) == 0
    assert int(e1) == -1 and int(e2) == -1 and int(e3) == 0 and still_null == "1"
