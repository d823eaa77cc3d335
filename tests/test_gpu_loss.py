"""The differentiable form on the GPU against the FP64 oracle.

Loss: relative error <= 1e-4; gradient (hand-written adjoint): relative L2
error <= 1e-3 against the oracle's analytic gradient, which is itself pinned
to central finite differences in FP64 (tests/test_oracle_pins.py)."""

import numpy as np
import pytest

import oracle.gs_oracle as O
from paper_1302_0120_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def normalized_target(seed, n, nspots):
    I = S.spot_target(seed, n, n, nspots, (0.5, 1.0)).astype(np.float64)
    I *= I.size / I.sum()  # sum I = N
    return I.astype(np.float32)


def gpu_loss_grad(I, phi, want_grad=True):
    import torch

    from paper_1302_0120_gb300 import build_lib
    from paper_1302_0120_gb300.differentiable import LossContext

    build_lib.build()
    lc = LossContext(I.shape[0])
    loss, grad = lc.loss_grad(torch.from_numpy(I).cuda(), torch.from_numpy(phi).cuda(), want_grad)
    st = lc.status()
    out = (float(loss.item()), grad.cpu().numpy() if grad is not None else None, st)
    lc.close()
    return out


@pytest.mark.parametrize("n,nspots", [(32, 4), (64, 6), (256, 30), (1024, 100)])
def test_loss_and_gradient_match_oracle(n, nspots):
    I = normalized_target(n, n, nspots)
    phi = S.random_phase(n + 1, n, n)
    loss, grad, st = gpu_loss_grad(I, phi)
    assert st == 0
    ref_l = O.intensity_loss(phi, I)
    ref_g = O.intensity_loss_grad(phi, I)
    assert abs(loss - ref_l) <= 1e-4 * ref_l, (loss, ref_l)
    err = np.linalg.norm(grad - ref_g) / np.linalg.norm(ref_g)
    assert err <= 1e-3, err
    loss_only, none, st = gpu_loss_grad(I, phi, want_grad=False)
    assert st == 0 and none is None and loss_only == loss


def test_autograd_and_adam():
    import torch

    from paper_1302_0120_gb300.differentiable import LossContext, intensity_loss, optimize_phase

    n = 256
    I = torch.from_numpy(normalized_target(5, n, 30)).cuda()
    phi0 = torch.from_numpy(S.random_phase(6, n, n)).cuda()
    lc = LossContext(n)
    phase = phi0.clone().requires_grad_(True)
    loss = intensity_loss(phase, I, lc)
    (2.5 * loss).backward()
    _, g = lc.loss_grad(I, phi0)
    assert torch.allclose(phase.grad, 2.5 * g, rtol=1e-6, atol=0)
    ph, losses = optimize_phase(I, phi0, steps=60, lr=0.05, lctx=lc)
    assert lc.status() == 0
    assert losses[-1] < 0.5 * losses[0], losses[[0, -1]]
    lc.close()


def test_nonfinite_target():
    from paper_1302_0120_gb300 import GS_ENUMERIC

    I = normalized_target(1, 64, 4)
    I[3, 3] = np.inf
    loss, grad, st = gpu_loss_grad(I, S.random_phase(2, 64, 64))
    assert st == GS_ENUMERIC and np.isnan(loss)
