"""Differentiable form: the intensity loss with a hand-written adjoint, as a
``torch.autograd.Function``, and a gradient-descent phase optimiser.

    L(phi) = sum_k (|F exp(i phi)|_k^2 / N - I_k)^2

Both the loss and its gradient come from one launch of the library
(gs_loss_grad): the gradient is produced by the adjoint passes in the forward
call and scaled by the incoming gradient in ``backward``. Adam itself is
torch's optimiser acting on the phase tensor there; ``optimize_phase``
runs the library's own optimiser steps instead (loss, gradient and Adam
update, many steps per launch).
"""

from __future__ import annotations

from . import _binding as B


class LossContext:
    """Workspace for the loss of n x n phase masks (C: gs_create + gs_loss_grad)."""

    def __init__(self, n: int, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream()
        self.n = int(n)
        self.stream = stream
        self.handle = B.gs_create(self.n, self.n, B.GS_FINAL_RESIDUAL, stream.cuda_stream)

    def loss_grad(self, target, phase, want_grad: bool = True):
        """Enqueue the loss (float64 tensor [1]) and the gradient (float32 like
        ``phase``, or None)."""
        import torch

        for x, nm in ((target, "target"), (phase, "phase")):
            if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and tuple(x.shape) == (self.n, self.n)):
                raise ValueError(f"{nm} must be a contiguous float32 CUDA tensor of shape ({self.n}, {self.n})")
        # The launch runs on the context's stream: it waits for the work the
        # caller queued on its current stream (the writes of target and
        # phase), and the caller's stream waits for the launch before it
        # touches loss and grad (or overwrites phase, as an optimiser step does).
        cur = torch.cuda.current_stream(phase.device)
        loss = torch.empty(1, dtype=torch.float64, device=phase.device)
        grad = torch.empty_like(phase) if want_grad else None
        self.stream.wait_stream(cur)
        rc = B.gs_loss_grad(self.handle, target.data_ptr(), phase.data_ptr(), loss.data_ptr(),
                            grad.data_ptr() if grad is not None else 0)
        cur.wait_stream(self.stream)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_loss_grad")
        return loss, grad

    def prepare(self, target):
        """Stage ``target`` once (C: gs_loss_prepare) for ``loss_grad_prepared``."""
        import torch

        if not (target.is_cuda and target.dtype == torch.float32 and target.is_contiguous()
                and tuple(target.shape) == (self.n, self.n)):
            raise ValueError(f"target must be a contiguous float32 CUDA tensor of shape ({self.n}, {self.n})")
        self.stream.wait_stream(torch.cuda.current_stream(target.device))
        rc = B.gs_loss_prepare(self.handle, target.data_ptr())
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_loss_prepare")

    def loss_grad_prepared(self, phase, want_grad: bool = True):
        """The loss and gradient on the staged target (C: gs_loss_grad_prepared)."""
        import torch

        if not (phase.is_cuda and phase.dtype == torch.float32 and phase.is_contiguous()
                and tuple(phase.shape) == (self.n, self.n)):
            raise ValueError(f"phase must be a contiguous float32 CUDA tensor of shape ({self.n}, {self.n})")
        cur = torch.cuda.current_stream(phase.device)
        loss = torch.empty(1, dtype=torch.float64, device=phase.device)
        grad = torch.empty_like(phase) if want_grad else None
        self.stream.wait_stream(cur)
        rc = B.gs_loss_grad_prepared(self.handle, phase.data_ptr(), loss.data_ptr(),
                                     grad.data_ptr() if grad is not None else 0)
        cur.wait_stream(self.stream)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_loss_grad_prepared")
        return loss, grad

    def status(self) -> int:
        return B.gs_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.gs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _function():
    import torch

    class IntensityLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phase, target, lctx):
            loss, grad = lctx.loss_grad(target, phase, want_grad=phase.requires_grad)
            ctx.save_for_backward(grad if grad is not None else phase.new_empty(0))
            return loss[0]

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            return grad * grad_out.to(grad.dtype), None, None

    return IntensityLoss


_IL = None


def intensity_loss(phase, target, lctx: LossContext):
    """L(phase) as a differentiable float64 scalar tensor."""
    global _IL
    if _IL is None:
        _IL = _function()
    return _IL.apply(phase, target, lctx)


def optimize_phase(target, phase0, steps: int = 200, lr: float = 0.05, betas=(0.9, 0.999), eps: float = 1e-8,
                   lctx: LossContext | None = None, record_every: int = 1, fused: bool = True):
    """Adam on the phase. Returns (phase, losses) with losses[k] the loss
    before step k (and the final loss last).

    With ``fused`` (the default) the target is staged once (gs_loss_prepare)
    and the library runs every step (gs_loss_adam_run: the loss and the
    gradient on the staged target with the Adam update of gs_adam_step
    applied in the gradient pass, all steps in one launch of up to 1024),
    writing each step's loss into the record on the device. Otherwise every
    step goes through the autograd function above and torch's Adam."""
    import torch

    if steps < 0 or record_every < 1:
        raise ValueError("steps must be >= 0 and record_every >= 1")
    if lctx is None:
        lctx = LossContext(phase0.shape[-1])
    if not fused:
        return _optimize_eager(target, phase0, steps, lr, betas, eps, lctx, record_every)
    s = lctx.stream
    cur = torch.cuda.current_stream(phase0.device)
    s.wait_stream(cur)
    with torch.cuda.stream(s):
        phase = phase0.detach().clone()
        m = torch.zeros_like(phase)
        v = torch.zeros_like(phase)
        state = torch.zeros(2, dtype=torch.int32, device=phase.device)
        record = torch.zeros(steps + 1, dtype=torch.float64, device=phase.device)
        # the target is validated and staged once; every step runs only the
        # transform passes on it
        rc = B.gs_loss_prepare(lctx.handle, target.data_ptr())
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_loss_prepare")
        if steps > 0:
            rc = B.gs_loss_adam_run(lctx.handle, phase.data_ptr(), m.data_ptr(), v.data_ptr(), state.data_ptr(),
                                    lr, betas[0], betas[1], eps, steps, record.data_ptr())
            if rc != B.GS_OK:
                raise B.GSError(rc, "gs_loss_adam_run")
        rc = B.gs_loss_grad_prepared(lctx.handle, phase.data_ptr(), record.data_ptr() + 8 * steps, 0)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_loss_grad_prepared")
    cur.wait_stream(s)
    phase.record_stream(cur)  # allocated on the context's stream, used on the caller's
    keep = list(range(0, steps, record_every)) + [steps]
    return phase.detach(), record.cpu().numpy()[keep]


def _optimize_eager(target, phase0, steps, lr, betas, eps, lctx, record_every):
    import torch

    phase = phase0.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([phase], lr=lr, betas=betas, eps=eps)
    losses = []
    for k in range(steps):
        opt.zero_grad(set_to_none=True)
        loss = intensity_loss(phase, target, lctx)
        loss.backward()
        opt.step()
        if k % record_every == 0:
            losses.append(loss.detach())
    with torch.no_grad():
        losses.append(intensity_loss(phase.detach(), target, lctx))
    return phase.detach(), torch.stack(losses).cpu().numpy()
