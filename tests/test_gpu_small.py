"""Small grids (power-of-two sides >= 32, at most 8192 pixels): by default a
run takes one block per mask with the whole field in shared memory; a fixed
grid (gs_set_grid) selects the persistent kernel instead. Both transform every
row and column with the same group FFT and the same projection arithmetic, so
the phases agree bit for bit and the gaps to FP64 rounding (their partial
sums are grouped differently). Parity with the oracle for the small kernel:
the 64 x 64 parity tests at the default grid, and the shapes below."""

import numpy as np
import pytest

from paper_1302_0120_gb300 import synthetic as S
from tests.gpu_util import gpu_gs, GROUPING_RTOL
from tests.test_gpu_parity import check_run

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32), (64, 64), (32, 64), (64, 32), (128, 64), (64, 128), (32, 256), (256, 32), (32, 128),
          (128, 32)]


def _inputs(ny, nx, seed=0):
    I = S.spot_target(seed, ny, nx, nspots=6, amp_range=(0.5, 1.0))
    phi0 = S.random_phase(seed + 1, ny, nx)
    return I, phi0


def _same(a, b):
    assert np.array_equal(a[0], b[0]), np.max(np.abs(a[0] - b[0]))
    np.testing.assert_allclose(a[1], b[1], rtol=GROUPING_RTOL, atol=0)
    np.testing.assert_allclose(a[2], b[2], rtol=GROUPING_RTOL, atol=0)
    assert a[3] == 0 and b[3] == 0


@pytest.mark.parametrize("ny,nx", SHAPES)
def test_small_kernel_matches_persistent_kernel(ny, nx):
    I, phi0 = _inputs(ny, nx)
    _same(gpu_gs(I, phi0, 20), gpu_gs(I, phi0, 20, grid=3))


@pytest.mark.parametrize("iters", [0, 1, 300])
def test_small_kernel_iteration_counts(iters):
    # zero iterations (the phase of exp(i phi0) and r^0), one, and more than
    # one persistent launch holds (the small kernel runs them in one launch)
    I, phi0 = _inputs(64, 64, seed=5)
    _same(gpu_gs(I, phi0, iters), gpu_gs(I, phi0, iters, grid=2))


def test_small_kernel_without_final_residual():
    I, phi0 = _inputs(64, 32, seed=7)
    a = gpu_gs(I, phi0, 9, final_residual=False)
    b = gpu_gs(I, phi0, 9, grid=5, final_residual=False)
    _same(a, b)
    assert a[1].shape == (9,)


@pytest.mark.parametrize("ny,nx", [(128, 64), (32, 256), (256, 32)])
def test_small_kernel_oracle_parity(ny, nx):
    I, phi0 = _inputs(ny, nx, seed=11)
    check_run(I, phi0, 12, one_step_at=(0, 11))


def test_small_kernel_batch_of_64():
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton

    I = np.stack([S.spot_target(300 + k, 64, 64, 5) for k in range(64)])
    P = np.stack([S.random_phase(400 + k, 64, 64) for k in range(64)])
    with GerchbergSaxton(64, 64, max_batch=64) as gs:
        ph, r, g = gs.run_batched(torch.from_numpy(I).cuda(), torch.from_numpy(P).cuda(), 20)
        assert gs.status() == 0
        ph, r, g = ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy()
    for k in (0, 17, 63):
        one = gpu_gs(I[k], P[k], 20)
        _same((ph[k], r[k], g[k], 0), one)


def test_small_kernel_without_gap_outputs():
    # null residual and gap pointers: the phase is unchanged and nothing is written
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton

    I, phi0 = _inputs(64, 64, seed=13)
    with GerchbergSaxton(64, 64) as gs:
        It, Pt = torch.from_numpy(I).cuda(), torch.from_numpy(phi0).cuda()
        ph, r, g = gs.run(It, Pt, 11, residuals=False, object_gap=False)
        assert r is None and g is None
        assert gs.status() == 0
        ph = ph.cpu().numpy()
    assert np.array_equal(ph, gpu_gs(I, phi0, 11)[0])
