"""Torch-facing wrapper of the C ABI: device memory and streams come from torch.

Every step of the method runs in the CUDA library; this module only checks
tensor shapes and dtypes, allocates outputs and passes pointers.
"""

from __future__ import annotations

import numpy as np

from . import _binding as B


class GerchbergSaxton:
    """A Gerchberg-Saxton context for nx x ny grids (C: gs_create).

    Runs are enqueued on ``stream`` (default: torch's current stream at
    construction). Arrays are [ny, nx] float32, target intensity in DFT order.
    """

    def __init__(self, nx: int, ny: int, final_residual: bool = True, stream=None, max_batch: int = 1,
                 init_from_target: bool = False, tensor_core: bool = False, bf16: bool = False,
                 mma_sync: bool = False):
        """``tensor_core`` runs the DFTs as FP16 tensor-core products (1024 x
        1024 on tcgen05 unless ``mma_sync``; ``bf16`` for BF16 operands there)."""
        import torch

        if stream is None:
            stream = torch.cuda.current_stream()
        self.nx, self.ny = int(nx), int(ny)
        self.final_residual = bool(final_residual)
        self.stream = stream
        self.max_batch = int(max_batch)
        flags = ((B.GS_FINAL_RESIDUAL if final_residual else 0) | (B.GS_INIT_FROM_TARGET if init_from_target else 0)
                 | (B.GS_TENSOR_CORE if tensor_core else 0) | (B.GS_BF16 if bf16 else 0)
                 | (B.GS_TC_MMA_SYNC if mma_sync else 0))
        self.tensor_core = bool(tensor_core)
        self.init_from_target = bool(init_from_target)
        self._p = None
        self.handle = B.gs_create_batched(self.nx, self.ny, self.max_batch, flags, stream.cuda_stream)

    # -- helpers
    def _check(self, x, name):
        import torch

        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
        if tuple(x.shape) != (self.ny, self.nx):
            raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {(self.ny, self.nx)}")

    def run(self, target, phase_in, iters: int, phase_out=None, residuals: bool = True, object_gap: bool = True):
        """Enqueue ``iters`` iterations (C: gs_run). Returns (phase_out, r, g);
        r and g are float64 CUDA tensors or None. Call ``status()`` (or sync the
        stream) before reading them."""
        import torch

        self._check(target, "target")
        if phase_in is not None or not self.init_from_target:
            self._check(phase_in, "phase_in")
        with torch.cuda.stream(self.stream):
            if phase_out is None:
                phase_out = torch.empty_like(target)
            else:
                self._check(phase_out, "phase_out")
            nr = iters + (1 if self.final_residual else 0)
            r = torch.empty(max(nr, 1), dtype=torch.float64, device=target.device) if residuals else None
            g = torch.empty(max(iters, 1), dtype=torch.float64, device=target.device) if object_gap else None
        rc = B.gs_run(self.handle, target.data_ptr(), phase_in.data_ptr() if phase_in is not None else 0, int(iters),
                      phase_out.data_ptr(),
                      r.data_ptr() if r is not None else 0, g.data_ptr() if g is not None else 0)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_run")
        if r is not None:
            r = r[:nr]
        if g is not None:
            g = g[:iters]
        return phase_out, r, g

    def run_batched(self, target, phase_in, iters: int, phase_out=None, residuals: bool = True,
                    object_gap: bool = True):
        """Enqueue ``iters`` iterations for a batch of masks (C: gs_run_batched).
        Arrays are [batch, ny, nx]; returns (phase_out, r [batch, K(+1)], g [batch, K])."""
        import torch

        for x, name in ((target, "target"), (phase_in, "phase_in")):
            if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
                raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
            if x.dim() != 3 or tuple(x.shape[1:]) != (self.ny, self.nx):
                raise ValueError(f"{name} has shape {tuple(x.shape)}, expected (batch, {self.ny}, {self.nx})")
        nb = target.shape[0]
        if phase_in.shape[0] != nb or not 1 <= nb <= self.max_batch:
            raise ValueError(f"batch {nb} outside 1..{self.max_batch} or mismatched")
        nr = iters + (1 if self.final_residual else 0)
        with torch.cuda.stream(self.stream):
            if phase_out is None:
                phase_out = torch.empty_like(phase_in)
            r = torch.empty((nb, max(nr, 1)), dtype=torch.float64, device=target.device) if residuals else None
            g = torch.empty((nb, max(iters, 1)), dtype=torch.float64, device=target.device) if object_gap else None
        if residuals and nr == 0:
            r = r[:, :0]
        rc = B.gs_run_batched(self.handle, nb, target.data_ptr(), phase_in.data_ptr(), int(iters), phase_out.data_ptr(),
                              r.data_ptr() if r is not None else 0, g.data_ptr() if g is not None else 0)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_run_batched")
        return phase_out, r, (g[:, :iters] if g is not None else None)

    def run_host(self, target: np.ndarray, phase_in: np.ndarray, iters: int):
        """End-to-end run on host arrays (C: gs_run_host). Returns numpy
        (phase, r, g); raises GSError on a device-side error."""
        target = np.ascontiguousarray(target, dtype=np.float32)
        phase_in = np.ascontiguousarray(phase_in, dtype=np.float32)
        out = np.empty_like(phase_in)
        nr = iters + (1 if self.final_residual else 0)
        r = np.empty(max(nr, 1), np.float64)
        g = np.empty(max(iters, 1), np.float64)
        rc = B.gs_run_host(self.handle, target.ctypes.data, phase_in.ctypes.data, int(iters), out.ctypes.data,
                           r.ctypes.data, g.ctypes.data)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_run_host")
        return out, r[:nr], g[:iters]

    def set_slm_amplitude(self, p) -> None:
        """Use the laser amplitude ``p`` (float32 CUDA tensor [ny, nx], kept
        alive by this object) on the SLM, or ``None`` for p = 1 (C: gs_set_slm_amplitude)."""
        if p is not None:
            self._check(p, "p")
        rc = B.gs_set_slm_amplitude(self.handle, p.data_ptr() if p is not None else 0)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_set_slm_amplitude")
        self._p = p

    def status(self) -> int:
        """Synchronise the stream and return (and clear) the device status (C: gs_status)."""
        return B.gs_status(self.handle)

    def set_grid(self, ctas: int) -> None:
        rc = B.gs_set_grid(self.handle, int(ctas))
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_set_grid")

    def set_mask_group(self, masks: int) -> None:
        """Masks of a batch iterated together (0: automatic, C: gs_set_mask_group)."""
        rc = B.gs_set_mask_group(self.handle, int(masks))
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_set_mask_group")

    @property
    def grid(self) -> int:
        return B.gs_get_grid(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            B.gs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class MixedGerchbergSaxton:
    """Batches of square masks of sizes 256, 512 and 1024 iterated together
    in one persistent launch (C: gs_create_mixed, gs_run_mixed).

    ``max_batch`` maps each size (256, 512, 1024) to the most masks of that
    size per run (total 1..64)."""

    SIZES = (256, 512, 1024)

    def __init__(self, max_batch: dict, final_residual: bool = True, stream=None, tensor_core: bool = False,
                 init_from_target: bool = False, bf16: bool = False, mma_sync: bool = False):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.final_residual = bool(final_residual)
        self.init_from_target = bool(init_from_target)
        self.max_batch = {n: int(max_batch.get(n, 0)) for n in self.SIZES}
        flags = ((B.GS_FINAL_RESIDUAL if final_residual else 0) | (B.GS_INIT_FROM_TARGET if init_from_target else 0)
                 | (B.GS_TENSOR_CORE if tensor_core else 0) | (B.GS_BF16 if bf16 else 0)
                 | (B.GS_TC_MMA_SYNC if mma_sync else 0))
        self.handle = B.gs_create_mixed([self.max_batch[n] for n in self.SIZES], flags, stream.cuda_stream)

    def run(self, targets: dict, phases: dict | None, iters: int):
        """Enqueue ``iters`` iterations for every size present in ``targets``
        (size -> [batch, n, n] float32 CUDA tensor; ``phases`` likewise, or
        None with init_from_target). Returns size -> (phase_out, r, g)."""
        import torch

        batch, tp, pp, op, rp, gp, out = [], [], [], [], [], [], {}
        nr = iters + (1 if self.final_residual else 0)
        for n in self.SIZES:
            t = targets.get(n)
            if t is None:
                batch.append(0)
                for lst in (tp, pp, op, rp, gp):
                    lst.append(0)
                continue
            ph = None if phases is None else phases.get(n)
            for x, name in ((t, "target"), (ph, "phase")):
                if x is None and name == "phase" and self.init_from_target:
                    continue
                if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
                        and x.dim() == 3 and tuple(x.shape[1:]) == (n, n)):
                    raise TypeError(f"{name} for size {n} must be a contiguous float32 CUDA tensor [batch, {n}, {n}]")
            nb = t.shape[0]
            if not 1 <= nb <= self.max_batch[n] or (ph is not None and ph.shape[0] != nb):
                raise ValueError(f"batch {nb} of size {n} outside 1..{self.max_batch[n]} or mismatched")
            with torch.cuda.stream(self.stream):
                o = torch.empty_like(t)
                r = torch.empty((nb, max(nr, 1)), dtype=torch.float64, device=t.device)
                g = torch.empty((nb, max(iters, 1)), dtype=torch.float64, device=t.device)
            out[n] = (o, r[:, :nr], g[:, :iters])
            batch.append(nb)
            tp.append(t.data_ptr())
            pp.append(ph.data_ptr() if ph is not None else 0)
            op.append(o.data_ptr())
            rp.append(r.data_ptr())
            gp.append(g.data_ptr())
        rc = B.gs_run_mixed(self.handle, batch, tp, None if self.init_from_target and phases is None else pp,
                            int(iters), op, rp, gp)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_run_mixed")
        return out

    def status(self) -> int:
        return B.gs_status(self.handle)

    @property
    def grid(self) -> int:
        return B.gs_get_grid(self.handle)

    def set_grid(self, ctas: int) -> None:
        rc = B.gs_set_grid(self.handle, int(ctas))
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_set_grid")

    def set_mask_group(self, masks: int) -> None:
        rc = B.gs_set_mask_group(self.handle, int(masks))
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_set_mask_group")

    def close(self) -> None:
        if getattr(self, "handle", None):
            B.gs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
