"""Batched runs (gs_run_batched): several independent masks of the same grid
in one launch give exactly the phases of separate runs (the masks share the
launch and its barriers, not their arithmetic) and the same gaps to FP64
rounding (the FP64 partial sums are grouped by each block's share of the
batch, which differs from a single mask's share), and an invalid target only
takes its own mask out."""

import numpy as np
import pytest

from paper_1302_0120_gb300 import synthetic as S
from tests.gpu_util import gpu_gs, GROUPING_RTOL

pytestmark = pytest.mark.gpu


def same_gaps(a, b):
    """Gaps summed in a different grouping of lines into blocks: equal to the
    rounding of the FP32 per-block partial sums (the sum across blocks is
    FP64)."""
    return np.allclose(a, b, rtol=GROUPING_RTOL, atol=0)


def make_batch(n_masks, ny, nx, iters_seed=0, nspots=20):
    I = np.stack([S.spot_target(100 + iters_seed + k, ny, nx, nspots, (0.5, 1.0)) for k in range(n_masks)])
    P = np.stack([S.random_phase(200 + iters_seed + k, ny, nx) for k in range(n_masks)])
    return I, P


def run_batched(I, P, iters, grid=None, final_residual=True):
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton, build_lib

    build_lib.build()
    nb, ny, nx = I.shape
    with GerchbergSaxton(nx, ny, final_residual=final_residual, max_batch=nb) as gs:
        if grid:
            gs.set_grid(grid)
        ph, r, g = gs.run_batched(torch.from_numpy(I).cuda(), torch.from_numpy(P).cuda(), iters)
        st = gs.status()
        from paper_1302_0120_gb300 import _binding as B

        assert B.gs_check_workspace(gs.handle) == B.GS_OK
        return ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy(), st


@pytest.mark.parametrize("n,ny,nx,iters,grid", [
    (4, 512, 512, 20, None),
    (3, 1024, 1024, 5, None),
    (2, 256, 512, 8, None),
    (5, 64, 64, 130, 4),   # more iterations than one launch holds
    (3, 128, 128, 6, 7),   # ragged shares
])
def test_batch_equals_separate_runs(n, ny, nx, iters, grid):
    I, P = make_batch(n, ny, nx)
    ph, r, g, st = run_batched(I, P, iters, grid=grid)
    assert st == 0
    for k in range(n):
        ph1, r1, g1, st1 = gpu_gs(I[k], P[k], iters, grid=grid)
        assert st1 == 0
        assert np.array_equal(ph[k], ph1), k
        assert same_gaps(r[k], r1), k
        assert same_gaps(g[k], g1), k


def test_batch_with_an_invalid_target():
    import torch

    from paper_1302_0120_gb300 import GS_ENUMERIC, GerchbergSaxton

    I, P = make_batch(3, 64, 64)
    I[1, 5, 7] = np.nan
    with GerchbergSaxton(64, 64, max_batch=3) as gs:
        sentinel = torch.full((3, 64, 64), 9.0, device="cuda")
        ph, r, g = gs.run_batched(torch.from_numpy(I).cuda(), torch.from_numpy(P).cuda(), 10, phase_out=sentinel)
        assert gs.status() == GS_ENUMERIC
        ph, r, g = ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy()
    assert np.all(ph[1] == 9.0) and np.all(np.isnan(r[1])) and np.all(np.isnan(g[1]))
    for k in (0, 2):
        ph1, r1, g1, st1 = gpu_gs(I[k], P[k], 10)
        assert np.array_equal(ph[k], ph1) and same_gaps(r[k], r1) and same_gaps(g[k], g1)


def test_batch_with_an_invalid_target_across_launches():
    import torch

    from paper_1302_0120_gb300 import GS_ENUMERIC, GerchbergSaxton

    I, P = make_batch(2, 64, 64)
    I[0] = 0.0
    with GerchbergSaxton(64, 64, max_batch=2) as gs:
        sentinel = torch.full((2, 64, 64), 9.0, device="cuda")
        ph, r, g = gs.run_batched(torch.from_numpy(I).cuda(), torch.from_numpy(P).cuda(), 140, phase_out=sentinel)
        assert gs.status() == GS_ENUMERIC
        ph, r = ph.cpu().numpy(), r.cpu().numpy()
    assert np.all(ph[0] == 9.0) and np.all(np.isnan(r[0]))
    ph1, r1, _, _ = gpu_gs(I[1], P[1], 140)
    assert np.array_equal(ph[1], ph1) and same_gaps(r[1], r1)
