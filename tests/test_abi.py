"""The C-ABI library loads and exports every symbol include/*.h declares, and
its host-side validation answers without touching the GPU."""

import ctypes
import glob
import os
import re

import pytest

from paper_1302_0120_gb300 import _binding as B
from paper_1302_0120_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return B.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(gs_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gs_create", "gs_run", "gs_run_host", "gs_status", "gs_destroy", "gs_strerror",
                 "gs_workspace_bytes"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(B.SIGNATURES)


def test_strerror(lib):
    assert B.gs_strerror(B.GS_OK) == "success"
    for code in (B.GS_EINVAL, B.GS_ENOMEM, B.GS_ECUDA, B.GS_ETIMEOUT, B.GS_ENUMERIC, B.GS_ECORRUPT, 12345):
        assert len(B.gs_strerror(code)) > 0


def test_workspace_bytes(lib):
    for n in (32, 64, 512, 1024, 4096):
        w = B.gs_workspace_bytes(n, n)
        # field (8 B/px) + amplitude (4) + host staging (2 x 4), plus FP64 partials
        assert w >= 20 * n * n
        assert w < 20 * n * n + (4 << 20)
    assert B.gs_workspace_bytes(1024, 512) > 0
    # sides that are not powers of two: 5-smooth, at most 1536
    for ok in ((800, 600), (600, 800), (1536, 1536), (96, 4096), (1000, 45 * 32)):
        assert B.gs_workspace_bytes(*ok) >= 20 * ok[0] * ok[1]
    for bad in ((4, 64), (64, 6), (33, 64), (8192, 64), (0, 0), (-64, 64), (98, 128), (77, 64), (1600, 600),
                (1620, 64), (7, 64)):
        assert B.gs_workspace_bytes(*bad) == 0
    # small sides (below 32) run on the general kernel
    for ok in ((8, 8), (16, 64), (30, 64), (12, 10)):
        assert B.gs_workspace_bytes(*ok) > 0


def test_create_validates_before_cuda(lib):
    h = ctypes.c_void_p(123)
    for nx, ny in ((33, 64), (64, 8192), (4, 4), (0, 64), (98, 64), (1600, 600)):
        rc = lib.gs_create(ctypes.byref(h), nx, ny, 1, None)
        assert rc == B.GS_EINVAL
        assert h.value is None
    assert lib.gs_create(None, 64, 64, 1, None) == B.GS_EINVAL
    assert lib.gs_create(ctypes.byref(h), 64, 64, 0x80, None) == B.GS_EINVAL
    # the tensor-core form exists for square 256, 512 and 1024 only
    for nx, ny in ((64, 64), (128, 128), (2048, 2048), (512, 256), (1024, 512), (800, 800), (768, 768)):
        assert lib.gs_create(ctypes.byref(h), nx, ny, B.GS_FINAL_RESIDUAL | B.GS_TENSOR_CORE, None) == B.GS_EINVAL
        assert h.value is None


def test_null_context_calls(lib):
    assert lib.gs_run(None, None, None, 1, None, None, None) == B.GS_EINVAL
    assert lib.gs_run_host(None, None, None, 1, None, None, None) == B.GS_EINVAL
    assert lib.gs_status(None) == B.GS_EINVAL
    assert lib.gs_set_grid(None, 4) == B.GS_EINVAL
    out = ctypes.c_int(0)
    assert lib.gs_get_grid(None, ctypes.byref(out)) == B.GS_EINVAL
    assert lib.gs_destroy(None) == B.GS_OK
    assert lib.gs_set_slm_amplitude(None, None) == B.GS_EINVAL
    assert lib.gs_test_barrier_timeout(None, 1) == B.GS_EINVAL
    assert lib.gs_physical_error(None, None, None, None) == B.GS_EINVAL
    assert lib.gs_loss_grad(None, None, None, None, None) == B.GS_EINVAL
    assert lib.gs_run_mixed(None, None, None, None, 1, None, None, None) == B.GS_EINVAL
    assert lib.gs_set_mask_group(None, 2) == B.GS_EINVAL
    assert lib.gs_set_trace(None, 1) == B.GS_EINVAL
    assert lib.gs_check_workspace(None) == B.GS_EINVAL
    n = ctypes.c_int(0)
    assert lib.gs_get_trace(None, None, 0, ctypes.byref(n), ctypes.byref(n)) == B.GS_EINVAL
    assert B.gs_adam_step(0, 0, 0, 0, 16, 0, 0.05, 0.9, 0.999, 1e-8) == B.GS_EINVAL
    assert B.gs_loss_prepare(0, 0) == B.GS_EINVAL
    assert B.gs_loss_grad_prepared(0, 0, 0, 0) == B.GS_EINVAL
    assert B.gs_loss_adam_prepared(0, 0, 0, 0, 0, 0.05, 0.9, 0.999, 1e-8, 0) == B.GS_EINVAL
    assert B.gs_loss_adam_run(0, 0, 0, 0, 0, 0.05, 0.9, 0.999, 1e-8, 10, 0) == B.GS_EINVAL


def test_create_mixed_validates_before_cuda(lib):
    h = ctypes.c_void_p(123)
    for mb in ((0, 0, 0), (65, 0, 0), (40, 20, 5), (-1, 2, 2), (0, 0, 65)):
        arr = (ctypes.c_int * 3)(*mb)
        assert lib.gs_create_mixed(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), 1, None) == B.GS_EINVAL
        assert h.value is None
    arr = (ctypes.c_int * 3)(2, 2, 2)
    assert lib.gs_create_mixed(None, ctypes.cast(arr, ctypes.c_void_p), 1, None) == B.GS_EINVAL
    assert lib.gs_create_mixed(ctypes.byref(h), None, 1, None) == B.GS_EINVAL
    assert lib.gs_create_mixed(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), 0x80, None) == B.GS_EINVAL


def test_noalloc_validates_before_cuda(lib):
    """Host-side rejection only (NULL arrays everywhere): sizes over the static
    scratch (nx * ny > 512 * 512), sizes that are not powers of two in
    [32, 4096], unknown flags, NULL arrays and negative iteration counts."""
    for nx, ny in ((1024, 512), (1024, 1024), (4096, 128), (4096, 4096), (16, 64), (33, 64), (64, 8192)):
        assert lib.gs_run_noalloc(nx, ny, 1, None, None, None, 1, None, None, None, None) == B.GS_EINVAL
    assert lib.gs_run_noalloc(64, 64, 0x80, None, None, None, 1, None, None, None, None) == B.GS_EINVAL
    assert lib.gs_run_noalloc(256, 256, B.GS_TENSOR_CORE, None, None, None, 1, None, None, None, None) == B.GS_EINVAL
    assert lib.gs_run_noalloc(64, 64, 1, None, None, None, 1, None, None, None, None) == B.GS_EINVAL
    assert lib.gs_run_noalloc(64, 64, 1, None, None, None, -1, None, None, None, None) == B.GS_EINVAL


def test_serve_validates_before_cuda(lib):
    """The persistent server's arguments are checked before any CUDA call."""
    h = ctypes.c_void_p()
    assert lib.gs_serve_create(None, 512, 4, 0, None) == B.GS_EINVAL
    for n, slots, grid in ((300, 4, 0), (128, 4, 0), (2048, 4, 0), (512, 0, 0), (512, 17, 0), (512, 4, -1)):
        assert lib.gs_serve_create(ctypes.byref(h), n, slots, grid, None) == B.GS_EINVAL, (n, slots, grid)
        assert h.value is None
    seq = ctypes.c_uint(0)
    d, st = ctypes.c_uint(0), ctypes.c_int(0)
    assert lib.gs_serve_submit(None, 0, 512, None, None, 30, None, None, None, ctypes.byref(seq)) == B.GS_EINVAL
    assert lib.gs_serve_poll(None, 0, ctypes.byref(d), ctypes.byref(st)) == B.GS_EINVAL
    assert lib.gs_serve_stop(None) == B.GS_EINVAL
    assert lib.gs_serve_grid(None) == 0
    assert lib.gs_serve_test_tick_limit(None, 5) == B.GS_EINVAL
    lib.gs_serve_destroy(None)  # a no-op


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        B.lib()


def test_optimize_phase_validates_before_cuda():
    from paper_1302_0120_gb300.differentiable import optimize_phase

    for kw in ({"steps": -1}, {"steps": 5, "record_every": 0}):
        with pytest.raises(ValueError):
            optimize_phase(None, None, **kw)
