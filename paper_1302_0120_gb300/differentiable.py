"""Differentiable form: the intensity loss with a hand-written adjoint, as a
``torch.autograd.Function``, and a gradient-descent phase optimiser.

    L(phi) = sum_k (|F exp(i phi)|_k^2 / N - I_k)^2

Both the loss and its gradient come from one launch of the library
(gs_loss_grad): the gradient is produced by the adjoint passes in the forward
call and scaled by the incoming gradient in ``backward``. Adam itself is
torch's optimiser acting on the phase tensor.
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
        with torch.cuda.stream(self.stream):
            loss = torch.empty(1, dtype=torch.float64, device=phase.device)
            grad = torch.empty_like(phase) if want_grad else None
        rc = B.gs_loss_grad(self.handle, target.data_ptr(), phase.data_ptr(), loss.data_ptr(),
                            grad.data_ptr() if grad is not None else 0)
        if rc != B.GS_OK:
            raise B.GSError(rc, "gs_loss_grad")
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
                   lctx: LossContext | None = None, record_every: int = 1):
    """Adam on the phase. Returns (phase, losses) with losses[k] the loss
    before step k (and the final loss last)."""
    import torch

    lctx = lctx or LossContext(phase0.shape[-1])
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
