"""Failure detection on the GPU without a GPU fault: a grid barrier that can
never complete (it waits for one arrival more than the grid has) gives up
after its bounded wait, the run reports GS_ETIMEOUT through gs_status, and the
same context then runs normally."""

import time

import numpy as np
import pytest

import oracle.gs_oracle as O
from paper_1302_0120_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def test_barrier_wait_gives_up_and_context_recovers():
    import torch

    from paper_1302_0120_gb300 import GS_ETIMEOUT, GerchbergSaxton, build_lib
    from paper_1302_0120_gb300 import _binding as B

    build_lib.build()
    I, phi0, _ = S.workload("spots64")
    with GerchbergSaxton(64, 64) as gs:
        gs.set_grid(4)  # a multi-block grid, so runs use grid barriers
        It, Pt = torch.from_numpy(I).cuda(), torch.from_numpy(phi0).cuda()
        assert B.gs_test_barrier_timeout(gs.handle, True) == 0
        t0 = time.perf_counter()
        gs.run(It, Pt, 5)
        st = gs.status()
        waited = time.perf_counter() - t0
        assert st == GS_ETIMEOUT
        assert 0.5 < waited < 30.0
        assert B.gs_test_barrier_timeout(gs.handle, False) == 0
        ph, r, g = gs.run(It, Pt, 5)
        assert gs.status() == 0
        ref = O.gs_run(I, phi0, 5)
        assert np.allclose(r.cpu().numpy(), ref["r"], rtol=1e-3, atol=0)
