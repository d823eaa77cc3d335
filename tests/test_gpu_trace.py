"""Pass timestamps (gs_set_trace): the record has the launch's shape, every
block's stamps advance pass by pass, and tracing does not change results."""

import numpy as np
import pytest

from paper_1302_0120_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def test_trace_shape_order_and_results():
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton, build_lib
    from paper_1302_0120_gb300 import _binding as B

    build_lib.build()
    I, phi0, _ = S.workload("spots512")
    It, Pt = torch.from_numpy(I).cuda(), torch.from_numpy(phi0).cuda()
    iters = 10
    with GerchbergSaxton(512, 512) as gs:
        ph0, r0, _ = gs.run(It, Pt, iters)
        assert gs.status() == 0
        assert B.gs_set_trace(gs.handle, True) == 0
        ph1, r1, _ = gs.run(It, Pt, iters)
        assert gs.status() == 0
        tr = B.gs_get_trace(gs.handle)
        grid = gs.grid
    assert torch.equal(ph0, ph1) and torch.equal(r0, r1)
    passes = 1 + 2 * iters + 1  # init, (column, row) x K, final residual
    assert tr.shape == (passes + 1, grid, 2)
    t = tr.astype(np.int64)
    assert np.all(t > 0)
    seq = t.transpose(0, 2, 1).reshape(-1, grid)  # per block: start, start, done_1, released_1, ...
    assert np.all(np.diff(seq, axis=0) >= 0), "stamps must not go back in time"
    work, barrier = B.pass_times(tr)
    assert work.shape == (passes,) and np.all(work > 0) and np.all(barrier > -1.0)


def test_workspace_canaries():
    """The canary words survive runs of every kind on one context and
    report an overwrite."""
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton, build_lib
    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300.differentiable import LossContext

    build_lib.build()
    I, phi0, _ = S.workload("spots64")
    It, Pt = torch.from_numpy(I).cuda(), torch.from_numpy(phi0).cuda()
    with GerchbergSaxton(64, 64, max_batch=2) as gs:
        gs.run(It, Pt, 7)
        gs.run_batched(torch.stack([It, It]), torch.stack([Pt, Pt]), 3)
        assert gs.status() == 0
        assert B.gs_check_workspace(gs.handle) == B.GS_OK
        assert B.gs_test_corrupt_workspace(gs.handle) == B.GS_OK
        assert B.gs_check_workspace(gs.handle) == B.GS_ECORRUPT
    lc = LossContext(64)
    lc.loss_grad(It, Pt)
    assert lc.status() == 0 and B.gs_check_workspace(lc.handle) == B.GS_OK
    lc.close()
