"""Serving on the GPU: every request served in the mix (batched with others,
on concurrent lanes, from a warm start) gives the same mask as the same
request run alone, and a 1 kHz stream of 512^2/1024^2 requests stays within
the 10 ms interspike budget (Sec. I, IV.A)."""

import numpy as np
import pytest

from tests.gpu_util import aligned_rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sizes,rate,seconds,budget", [((128, 256), 4000.0, 0.08, 256 << 20),
                                                        ((512, 1024), 2000.0, 0.15, None)])
def test_each_result_same_alone_and_in_the_mix(sizes, rate, seconds, budget):
    """Small sizes at a high rate (many shared launches), and the 512^2 /
    1024^2 sizes the service runs at."""
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton
    from paper_1302_0120_gb300 import serving as SV

    kw = {} if budget is None else {"budget_bytes": budget}
    summ, sch, ex = SV.run_service(rate_hz=rate, seconds=seconds, sizes=sizes, lanes=(1, 2), iters=30,
                                   record=True, warmup_s=0.0, max_batch_cap=6, **kw)
    try:
        done = sorted(sch.done, key=lambda r: r.rid)
        assert len(done) == summ["requests"] > 50
        assert max(r.slot for r in done) > 0  # some requests shared a launch
        assert {r.n for r in done} == set(sizes)
        picks = done[:: max(1, len(done) // 12)]
        for r in picks:
            with GerchbergSaxton(r.n, r.n) as gs:
                ph, res, _ = gs.run(torch.from_numpy(r.target).cuda(), torch.from_numpy(r.warm_in).cuda(), 30)
                assert gs.status() == 0
                ph = ph.cpu().numpy()
                res = res.cpu().numpy()
            assert aligned_rel_err(r.phase, np.exp(1j * ph.astype(np.float64))) <= 1e-5, r.rid
            assert abs(r.residual - res[-1]) <= 1e-3 * res[-1], r.rid
    finally:
        ex.close()


def test_stream_of_512_and_1024_meets_interspike_budget():
    from paper_1302_0120_gb300 import serving as SV

    summ, sch, ex = SV.run_service(rate_hz=1000.0, seconds=1.0, sizes=(512, 1024), lanes=(1, 2), iters=30,
                                   warmup_s=0.3)
    ex.close()
    assert summ["requests"] > 800
    assert summ["p99_ms"] < 10.0, summ
