"""ctypes binding of the C ABI declared in include/gs.h.

Argument marshalling only: every function here forwards to the CUDA library
of the same name. The library must have been built (build_lib.build()); if it
is missing the import of the symbols fails loudly. There is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

from .build_lib import LIB_PATH

GS_OK = 0
GS_EINVAL = -1
GS_ENOMEM = -2
GS_ECUDA = -3
GS_ETIMEOUT = -4
GS_ENUMERIC = -5
GS_ECORRUPT = -6

GS_FINAL_RESIDUAL = 1
GS_INIT_FROM_TARGET = 2
GS_TENSOR_CORE = 4
GS_BF16 = 8
GS_TC_MMA_SYNC = 16

_c_int = ctypes.c_int
_c_uint = ctypes.c_uint
_vp = ctypes.c_void_p

# name -> (restype, argtypes), mirroring include/gs.h
SIGNATURES = {
    "gs_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_uint, _vp]),
    "gs_run": (_c_int, [_vp, _vp, _vp, _c_int, _vp, _vp, _vp]),
    "gs_run_host": (_c_int, [_vp, _vp, _vp, _c_int, _vp, _vp, _vp]),
    "gs_status": (_c_int, [_vp]),
    "gs_set_grid": (_c_int, [_vp, _c_int]),
    "gs_get_grid": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "gs_destroy": (_c_int, [_vp]),
    "gs_strerror": (ctypes.c_char_p, [_c_int]),
    "gs_workspace_bytes": (ctypes.c_size_t, [_c_int, _c_int, _c_uint]),
    "gs_run_noalloc": (_c_int, [_c_int, _c_int, _c_uint, _vp, _vp, _vp, _c_int, _vp, _vp, _vp, _vp]),
    "gs_create_batched": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_int, _c_uint, _vp]),
    "gs_run_batched": (_c_int, [_vp, _c_int, _vp, _vp, _c_int, _vp, _vp, _vp]),
    "gs_workspace_bytes_batched": (ctypes.c_size_t, [_c_int, _c_int, _c_int, _c_uint]),
    "gs_loss_grad": (_c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gs_loss_prepare": (_c_int, [_vp, _vp]),
    "gs_loss_grad_prepared": (_c_int, [_vp, _vp, _vp, _vp]),
    "gs_loss_adam_prepared": (_c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, _vp]),
    "gs_loss_adam_run": (_c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, _c_int, _vp]),
    "gs_set_slm_amplitude": (_c_int, [_vp, _vp]),
    "gs_test_barrier_timeout": (_c_int, [_vp, _c_int]),
    "gs_physical_error": (_c_int, [_vp, _vp, _vp, _vp]),
    "gs_create_mixed": (_c_int, [ctypes.POINTER(_vp), _vp, _c_uint, _vp]),
    "gs_run_mixed": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _vp, _vp, _vp]),
    "gs_set_mask_group": (_c_int, [_vp, _c_int]),
    "gs_set_trace": (_c_int, [_vp, _c_int]),
    "gs_check_workspace": (_c_int, [_vp]),
    "gs_test_corrupt_workspace": (_c_int, [_vp]),
    "gs_get_trace": (_c_int, [_vp, _vp, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "gs_fp32_peak": (_c_int, [ctypes.POINTER(ctypes.c_double), _vp]),
    "gs_stream_notify": (_c_int, [_vp, _c_int]),
    "gs_serve_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_int, _vp]),
    "gs_serve_submit": (_c_int, [_vp, _c_int, _c_int, _vp, _vp, _c_int, _vp, _vp, _vp, ctypes.POINTER(_c_uint)]),
    "gs_serve_poll": (_c_int, [_vp, _c_int, ctypes.POINTER(_c_uint), ctypes.POINTER(_c_int)]),
    "gs_serve_stop": (_c_int, [_vp]),
    "gs_serve_grid": (_c_int, [_vp]),
    "gs_serve_test_tick_limit": (_c_int, [_vp, _c_int]),
    "gs_serve_destroy": (None, [_vp]),
    "gs_adam_step": (_c_int, [_vp, _vp, _vp, _vp, ctypes.c_longlong, _vp, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, _vp]),
}

_lib = None


class GSError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {gs_strerror(code)} ({code})" if what else f"{gs_strerror(code)} ({code})")


def lib() -> ctypes.CDLL:
    """The loaded CUDA library. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_1302_0120_gb300.build_lib.build() "
                "(requires nvcc); there is no CPU fallback"
            )
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def gs_strerror(code: int) -> str:
    return lib().gs_strerror(int(code)).decode()


def gs_workspace_bytes(nx: int, ny: int, flags: int = GS_FINAL_RESIDUAL) -> int:
    return int(lib().gs_workspace_bytes(int(nx), int(ny), int(flags)))


def gs_workspace_bytes_batched(nx: int, ny: int, max_batch: int, flags: int = GS_FINAL_RESIDUAL) -> int:
    return int(lib().gs_workspace_bytes_batched(int(nx), int(ny), int(max_batch), int(flags)))


def gs_create_batched(nx: int, ny: int, max_batch: int, flags: int = GS_FINAL_RESIDUAL,
                      stream: int | None = None) -> int:
    """Create a context for up to max_batch masks per run; returns its handle. Raises GSError."""
    h = _vp()
    rc = lib().gs_create_batched(ctypes.byref(h), int(nx), int(ny), int(max_batch), int(flags), _vp(stream or 0))
    if rc != GS_OK:
        raise GSError(rc, "gs_create_batched")
    return h.value


def gs_run_batched(ctx: int, batch: int, target_intensity: int, phase_in: int, iters: int, phase_out: int,
                   residual_out: int = 0, object_gap_out: int = 0) -> int:
    """Enqueue a run of `batch` strided masks on device pointers; returns the status code."""
    return lib().gs_run_batched(_vp(ctx), int(batch), _vp(target_intensity), _vp(phase_in), int(iters),
                                _vp(phase_out), _vp(residual_out or 0), _vp(object_gap_out or 0))


def _arr3(ctype, vals):
    return (ctype * 3)(*vals)


def gs_create_mixed(max_batch, flags: int = GS_FINAL_RESIDUAL, stream: int | None = None) -> int:
    """Create a context for masks of size 256, 512 and 1024 (max_batch per
    size, a sequence of 3 ints) run together; returns its handle. Raises GSError."""
    h = _vp()
    mb = _arr3(_c_int, [int(x) for x in max_batch])
    rc = lib().gs_create_mixed(ctypes.byref(h), ctypes.cast(mb, _vp), int(flags), _vp(stream or 0))
    if rc != GS_OK:
        raise GSError(rc, "gs_create_mixed")
    return h.value


def gs_run_mixed(ctx: int, batch, target_intensity, phase_in, iters: int, phase_out, residual_out=None,
                 object_gap_out=None) -> int:
    """Enqueue one launch over three size classes. ``batch`` is 3 ints; the
    array arguments are sequences of 3 device pointers (0 for unused entries)
    or None where the header allows NULL; returns the status code."""
    keep = []

    def ptrs(v):
        if v is None:
            return None
        a = _arr3(_vp, [int(x or 0) or None for x in v])
        keep.append(a)
        return ctypes.cast(a, _vp)

    b = _arr3(_c_int, [int(x) for x in batch])
    return lib().gs_run_mixed(_vp(ctx), ctypes.cast(b, _vp), ptrs(target_intensity), ptrs(phase_in), int(iters),
                              ptrs(phase_out), ptrs(residual_out), ptrs(object_gap_out))


def gs_adam_step(phase: int, grad: int, m: int, v: int, n: int, state: int, lr: float, beta1: float, beta2: float,
                 eps: float, stream: int | None = None) -> int:
    """Enqueue one Adam update on device pointers; returns the status code."""
    return lib().gs_adam_step(_vp(phase), _vp(grad), _vp(m), _vp(v), int(n), _vp(state), float(lr), float(beta1),
                              float(beta2), float(eps), _vp(stream or 0))


def gs_check_workspace(ctx: int) -> int:
    """Compare the workspace's canary words (synchronises); returns the status code."""
    return lib().gs_check_workspace(_vp(ctx))


def gs_test_corrupt_workspace(ctx: int) -> int:
    """Test hook: overwrite one canary byte from the host; returns the status code."""
    return lib().gs_test_corrupt_workspace(_vp(ctx))


def gs_set_trace(ctx: int, enable: bool) -> int:
    """Record pass timestamps of later runs; returns the status code."""
    return lib().gs_set_trace(_vp(ctx), 1 if enable else 0)


def gs_get_trace(ctx: int):
    """The last traced launch as a numpy uint64 array [passes + 1, grid, 2]
    (row 0: launch start; row 1 + q: pass q done, released). Raises GSError."""
    import numpy as np

    cap = 2 * (2 * 128 + 5) * 256
    buf = np.zeros(cap, dtype=np.uint64)
    passes, grid = _c_int(0), _c_int(0)
    rc = lib().gs_get_trace(_vp(ctx), _vp(buf.ctypes.data), cap, ctypes.byref(passes), ctypes.byref(grid))
    if rc != GS_OK:
        raise GSError(rc, "gs_get_trace")
    return buf[: 2 * (passes.value + 1) * grid.value].reshape(passes.value + 1, grid.value, 2)


def pass_times(trace):
    """Per pass (microseconds): the slowest block's work (from its release by
    the previous barrier, or the launch start, to its arrival) and the
    barrier latency (last arrival to the median release)."""
    import numpy as np

    t = trace.astype(np.float64)
    prev = t[:-1, :, 1]
    done = t[1:, :, 0]
    rel = t[1:, :, 1]
    work = (done - prev).max(axis=1) / 1e3
    barrier = (np.median(rel, axis=1) - done.max(axis=1)) / 1e3
    return work, barrier


def gs_set_mask_group(ctx: int, masks: int) -> int:
    """Masks of a batched run iterated together (0: automatic); returns the status code."""
    return lib().gs_set_mask_group(_vp(ctx), int(masks))


def gs_create(nx: int, ny: int, flags: int = GS_FINAL_RESIDUAL, stream: int | None = None) -> int:
    """Create a context; returns its handle (an int). Raises GSError."""
    h = _vp()
    rc = lib().gs_create(ctypes.byref(h), int(nx), int(ny), int(flags), _vp(stream or 0))
    if rc != GS_OK:
        raise GSError(rc, "gs_create")
    return h.value


def gs_run(ctx: int, target_intensity: int, phase_in: int, iters: int, phase_out: int,
           residual_out: int = 0, object_gap_out: int = 0) -> int:
    """Enqueue a run on device pointers; returns the status code."""
    return lib().gs_run(_vp(ctx), _vp(target_intensity), _vp(phase_in), int(iters), _vp(phase_out),
                        _vp(residual_out or 0), _vp(object_gap_out or 0))


def gs_run_host(ctx: int, target_intensity: int, phase_in: int, iters: int, phase_out: int,
                residual_out: int = 0, object_gap_out: int = 0) -> int:
    """Run on host pointers (synchronous); returns the status code."""
    return lib().gs_run_host(_vp(ctx), _vp(target_intensity), _vp(phase_in), int(iters), _vp(phase_out),
                             _vp(residual_out or 0), _vp(object_gap_out or 0))


def gs_loss_grad(ctx: int, target_intensity: int, phase: int, loss_out: int, grad_out: int = 0) -> int:
    """Enqueue the intensity loss (and its gradient when grad_out != 0); returns the status code."""
    return lib().gs_loss_grad(_vp(ctx), _vp(target_intensity), _vp(phase), _vp(loss_out), _vp(grad_out or 0))


def gs_loss_prepare(ctx: int, target_intensity: int) -> int:
    """Enqueue the staging of a target for gs_loss_grad_prepared; returns the status code."""
    return lib().gs_loss_prepare(_vp(ctx), _vp(target_intensity))


def gs_loss_grad_prepared(ctx: int, phase: int, loss_out: int, grad_out: int = 0) -> int:
    """Enqueue the loss (and gradient) on the staged target; returns the status code."""
    return lib().gs_loss_grad_prepared(_vp(ctx), _vp(phase), _vp(loss_out), _vp(grad_out or 0))


def gs_loss_adam_prepared(ctx: int, phase: int, m: int, v: int, state: int, lr: float, beta1: float, beta2: float,
                          eps: float, loss_out: int) -> int:
    """Enqueue one optimiser step (loss on the staged target, gradient, Adam update in place); returns the status code."""
    return lib().gs_loss_adam_prepared(_vp(ctx), _vp(phase), _vp(m), _vp(v), _vp(state), float(lr), float(beta1),
                                       float(beta2), float(eps), _vp(loss_out))


def gs_loss_adam_run(ctx: int, phase: int, m: int, v: int, state: int, lr: float, beta1: float, beta2: float,
                     eps: float, steps: int, loss_out: int) -> int:
    """Enqueue `steps` optimiser steps (up to 1024 per launch); loss_out[k] is the loss before step k."""
    return lib().gs_loss_adam_run(_vp(ctx), _vp(phase), _vp(m), _vp(v), _vp(state), float(lr), float(beta1),
                                  float(beta2), float(eps), int(steps), _vp(loss_out))


def gs_physical_error(ctx: int, target_intensity: int, phase: int, error_out: int) -> int:
    """Enqueue the physical error (E_l, E_d) into a device double[2]; returns the status code."""
    return lib().gs_physical_error(_vp(ctx), _vp(target_intensity), _vp(phase), _vp(error_out))


def gs_status(ctx: int) -> int:
    return lib().gs_status(_vp(ctx))


def gs_set_slm_amplitude(ctx: int, amplitude: int) -> int:
    """Set (device pointer) or clear (0) the SLM amplitude p; returns the status code."""
    return lib().gs_set_slm_amplitude(_vp(ctx), _vp(amplitude or 0))


def gs_test_barrier_timeout(ctx: int, enable: bool) -> int:
    """Test hook: make the grid barriers of later runs time out (enable) or not."""
    return lib().gs_test_barrier_timeout(_vp(ctx), 1 if enable else 0)


def gs_set_grid(ctx: int, ctas: int) -> int:
    return lib().gs_set_grid(_vp(ctx), int(ctas))


def gs_get_grid(ctx: int) -> int:
    out = _c_int(0)
    rc = lib().gs_get_grid(_vp(ctx), ctypes.byref(out))
    if rc != GS_OK:
        raise GSError(rc, "gs_get_grid")
    return out.value


def gs_run_noalloc(nx: int, ny: int, flags: int, stream: int, target_intensity: int, phase_in: int, iters: int,
                   phase_out: int, residual_out: int = 0, object_gap_out: int = 0, device_status: int = 0) -> int:
    """gs_run on the library's static scratch (no allocation); returns the status code."""
    return lib().gs_run_noalloc(int(nx), int(ny), int(flags), _vp(stream or 0), _vp(target_intensity),
                                _vp(phase_in), int(iters), _vp(phase_out), _vp(residual_out or 0),
                                _vp(object_gap_out or 0), _vp(device_status or 0))


def gs_fp32_peak(stream: int | None = None) -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s (synchronous). Raises GSError."""
    out = ctypes.c_double(0.0)
    rc = lib().gs_fp32_peak(ctypes.byref(out), _vp(stream or 0))
    if rc != GS_OK:
        raise GSError(rc, "gs_fp32_peak")
    return out.value


def gs_stream_notify(stream: int | None, fd: int) -> int:
    """Enqueue a write of 1 to ``fd`` once ``stream`` reaches it; returns the status code."""
    return lib().gs_stream_notify(_vp(stream or 0), int(fd))


def gs_serve_create(max_n: int, slots: int, grid: int = 0, stream: int | None = None) -> int:
    """A persistent server for masks up to max_n x max_n with `slots` request slots; returns its handle."""
    h = _vp()
    rc = lib().gs_serve_create(ctypes.byref(h), int(max_n), int(slots), int(grid), _vp(stream or 0))
    if rc != GS_OK:
        raise GSError(rc, "gs_serve_create")
    return h.value


def gs_serve_submit(srv: int, slot: int, n: int, target: int, phase_in: int, iters: int, phase_out: int,
                    r_out: int = 0, g_out: int = 0):
    """Post a request for an n x n mask (pinned host pointers); returns (status code, sequence number)."""
    seq = _c_uint(0)
    rc = lib().gs_serve_submit(_vp(srv), int(slot), int(n), _vp(target), _vp(phase_in), int(iters), _vp(phase_out),
                               _vp(r_out or None), _vp(g_out or None), ctypes.byref(seq))
    return rc, seq.value


def gs_serve_poll(srv: int, slot: int):
    """(server status, last done sequence number of the slot, that request's status)."""
    d, st = _c_uint(0), _c_int(0)
    rc = lib().gs_serve_poll(_vp(srv), int(slot), ctypes.byref(d), ctypes.byref(st))
    return rc, d.value, st.value


def gs_serve_stop(srv: int) -> int:
    return lib().gs_serve_stop(_vp(srv))


def gs_serve_grid(srv: int) -> int:
    return lib().gs_serve_grid(_vp(srv))


def gs_serve_test_tick_limit(srv: int, ticks: int) -> int:
    """Test hook: launches leave after `ticks` iterations; returns the status code."""
    return lib().gs_serve_test_tick_limit(_vp(srv), int(ticks))


def gs_serve_destroy(srv: int) -> None:
    lib().gs_serve_destroy(_vp(srv))


def gs_destroy(ctx: int) -> int:
    return lib().gs_destroy(_vp(ctx))
