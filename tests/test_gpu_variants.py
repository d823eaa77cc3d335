"""Paper variants on the GPU against the oracle: a Gaussian laser amplitude p
on the SLM (Eq. slm-constraint) and the target-based initial condition of
Sec. IV. Same tolerances as tests/test_gpu_parity.py."""

import numpy as np
import pytest

import oracle.gs_oracle as O
from paper_1302_0120_gb300 import synthetic as S
from tests.gpu_util import aligned_rel_err

pytestmark = pytest.mark.gpu


def gpu_run(I, phi0, iters, p=None, init_from_target=False):
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton, build_lib

    build_lib.build()
    ny, nx = I.shape
    with GerchbergSaxton(nx, ny, init_from_target=init_from_target) as gs:
        pt = None
        if p is not None:
            pt = torch.from_numpy(p).cuda()
            gs.set_slm_amplitude(pt)
        It = torch.from_numpy(I).cuda()
        Pt = torch.from_numpy(phi0).cuda() if phi0 is not None else None
        ph, r, g = gs.run(It, Pt, iters)
        st = gs.status()
        return ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy(), st


@pytest.mark.parametrize("ny,nx,iters", [(64, 64, 20), (512, 512, 30), (256, 512, 10)])
def test_laser_amplitude(ny, nx, iters):
    I = S.spot_target(31, ny, nx, 20, (0.5, 1.0))
    phi0 = S.random_phase(31, ny, nx)
    p = S.laser_amplitude(ny, nx)
    ph, r, g, st = gpu_run(I, phi0, iters, p=p)
    assert st == 0
    ref = O.gs_run(I, phi0, iters, p=p)
    assert np.max(np.abs(r - ref["r"]) / ref["r"]) <= 1e-3
    assert np.max(np.abs(g - ref["g"]) / ref["g"]) <= 1e-3
    assert np.all(r[:-1] - g >= -1e-6) and np.all(g - r[1:] >= -1e-6)
    # one step from the GPU's own iterate
    ph1, _, _, _ = gpu_run(I, ph, 1, p=p)
    m = O.target_amplitude(I, energy=float(np.sum(p.astype(np.float64) ** 2)))
    u = p.astype(np.float64) * np.exp(1j * ph.astype(np.float64))
    u1, _, _ = O.gs_step(u, m, p.astype(np.float64))
    assert aligned_rel_err(ph1, u1 / np.abs(u1)) <= 1e-5


def test_laser_amplitude_rejects_negative():
    from paper_1302_0120_gb300 import GS_ENUMERIC

    I, phi0, _ = S.workload("spots64")
    p = S.laser_amplitude(64, 64)
    p[10, 10] = -0.5
    ph, r, g, st = gpu_run(I, phi0, 3, p=p)
    assert st == GS_ENUMERIC and np.all(np.isnan(r))


@pytest.mark.parametrize("n,iters", [(64, 10), (1024, 5)])
def test_target_start(n, iters):
    """The start is conjugate-symmetric (real target), an invariant subspace of
    the iteration that is unstable: rounding breaks the symmetry and the
    difference grows about tenfold per iteration (an FP32 run of the oracle
    already differs from the FP64 one by 2e-4 after one step and 3e-3 after
    two at 1024^2). Trajectories are therefore compared at the start and after
    the first step only; the chain holds throughout."""
    I = S.spot_target(41, n, n, 20 if n == 64 else 50, (0.5, 1.0))
    ph, r, g, st = gpu_run(I, None, iters, init_from_target=True)
    assert st == 0
    ref = O.gs_run(I, None, iters, init="target")
    assert np.max(np.abs(r[:2] - ref["r"][:2]) / ref["r"][:2]) <= 1e-3
    assert np.all(r[:-1] - g >= -1e-6) and np.all(g - r[1:] >= -1e-6)
    # the start itself (zero iterations): u0 = P_S(F^{-1} m). v/|v| is
    # ill-conditioned where F^{-1} m nearly vanishes, so the phase is gated at
    # three times the error an FP32 run of the oracle itself makes.
    ph0, r0, _, st = gpu_run(I, None, 0, init_from_target=True)
    ref0 = O.gs_run(I, None, 0, init="target")
    fp32 = O.gs_run(I, None, 0, init="target", dtype=np.float32)
    tol = max(1e-5, 3 * aligned_rel_err(fp32["phase"].astype(np.float32), ref0["u"]))
    assert st == 0 and aligned_rel_err(ph0, ref0["u"]) <= tol
    assert abs(r0[0] - ref0["r"][0]) <= 1e-4 * ref0["r"][0]
