"""The persistent server (gs_serve_*): requests posted while others run join
them between iterations, and each result is the result of the same request
run alone (gs_run from the same start), within the serving tolerances of
tests/test_gpu_serving.py; a bad target or a busy slot is reported, the
server leaves when idle and comes back on the next request, and a 1 kHz
stream of 512^2 / 1024^2 requests stays within the 10 ms interspike budget
(Sec. I, IV.A)."""

import time

import numpy as np
import pytest

from paper_1302_0120_gb300 import synthetic as S
from tests.gpu_util import aligned_rel_err

pytestmark = pytest.mark.gpu


def _pinned(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


class _Req:
    def __init__(self, n, seed, K, target=None):
        import torch

        self.n, self.K = n, K
        self.I = _pinned(S.spot_target(seed, n, n, 30, (0.5, 1.0)) if target is None else target.astype(np.float32))
        self.phi0 = S.random_phase(seed, n, n)
        self.phase = _pinned(self.phi0.copy())  # start phase, overwritten by the result
        self.r = torch.zeros(K, dtype=torch.float64).pin_memory()
        self.g = torch.zeros(K, dtype=torch.float64).pin_memory()
        self.seq = 0

    def submit(self, B, srv, slot):
        rc, seq = B.gs_serve_submit(srv, slot, self.n, self.I.data_ptr(), self.phase.data_ptr(), self.K,
                                    self.phase.data_ptr(), self.r.data_ptr(), self.g.data_ptr())
        if rc == B.GS_OK:
            self.seq = seq
        return rc


def _wait(B, srv, slot, seq, timeout=20.0):
    t0 = time.perf_counter()
    while True:
        rc, done, st = B.gs_serve_poll(srv, slot)
        assert rc == B.GS_OK, B.gs_strerror(rc)
        if done == seq:
            return st
        assert time.perf_counter() - t0 < timeout, "request not done"
        time.sleep(1e-4)


def _check_alone(req):
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton

    with GerchbergSaxton(req.n, req.n) as gs:
        ph, r, g = gs.run(req.I.cuda(), torch.from_numpy(req.phi0).cuda(), req.K)
        assert gs.status() == 0
        ph, r, g = ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy()
    assert aligned_rel_err(req.phase.numpy(), np.exp(1j * ph.astype(np.float64))) <= 1e-5
    assert np.allclose(req.r.numpy(), r[: req.K], rtol=1e-3, atol=0)
    assert np.allclose(req.g.numpy(), g, rtol=1e-3, atol=0)


@pytest.mark.parametrize("sizes", [(256, 256, 256), (512, 512, 512), (1024, 1024, 1024), (1024, 256, 512)])
def test_requests_joining_mid_run_match_runs_alone(sizes):
    """Three requests, the third posted while the first two run; one server
    for one size, and one serving three sizes at once."""
    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300 import build_lib

    build_lib.build()
    srv = B.gs_serve_create(max(sizes), 4, 0, None)
    try:
        a, b, c = _Req(sizes[0], 1, 40), _Req(sizes[1], 2, 6), _Req(sizes[2], 3, 9)
        assert a.submit(B, srv, 0) == B.GS_OK
        assert b.submit(B, srv, 1) == B.GS_OK
        time.sleep(3e-4)  # a and b are running: c joins them
        assert c.submit(B, srv, 3) == B.GS_OK
        for req, slot in ((a, 0), (b, 1), (c, 3)):
            assert _wait(B, srv, slot, req.seq) == B.GS_OK
        assert B.gs_serve_stop(srv) == B.GS_OK
        for req in (a, b, c):
            _check_alone(req)
    finally:
        B.gs_serve_destroy(srv)


def test_launches_leaving_mid_request_resume():
    """Launches that leave every 5 ticks with requests running (the tick limit
    that keeps the barrier counter in range, lowered by a test hook): the next
    launch resumes the slots, and every result is the result of the run alone."""
    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300 import build_lib

    build_lib.build()
    srv = B.gs_serve_create(512, 3, 0, None)
    try:
        assert B.gs_serve_test_tick_limit(srv, 5) == B.GS_OK
        a, b, c = _Req(512, 11, 23), _Req(256, 12, 17), _Req(512, 13, 9)
        assert a.submit(B, srv, 0) == B.GS_OK
        assert b.submit(B, srv, 1) == B.GS_OK
        assert c.submit(B, srv, 2) == B.GS_OK
        for req, slot in ((a, 0), (b, 1), (c, 2)):
            assert _wait(B, srv, slot, req.seq) == B.GS_OK
        assert B.gs_serve_stop(srv) == B.GS_OK
        for req in (a, b, c):
            _check_alone(req)
    finally:
        B.gs_serve_destroy(srv)


def test_bad_target_busy_slot_and_idle_relaunch():
    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300 import build_lib

    build_lib.build()
    n = 256
    srv = B.gs_serve_create(n, 2, 0, None)
    try:
        bad_target = S.spot_target(5, n, n, 10, (0.5, 1.0))
        bad_target[3, 4] = -1.0
        bad, good = _Req(n, 5, 4, target=bad_target), _Req(n, 6, 20)
        assert good.submit(B, srv, 1) == B.GS_OK
        assert good.submit(B, srv, 1) == B.GS_EINVAL  # slot 1 is busy
        big = _Req(512, 8, 3)
        assert big.submit(B, srv, 0) == B.GS_EINVAL  # larger than the server's grids
        assert bad.submit(B, srv, 0) == B.GS_OK
        assert _wait(B, srv, 0, bad.seq) == B.GS_ENUMERIC
        assert np.array_equal(bad.phase.numpy(), bad.phi0)  # untouched
        assert _wait(B, srv, 1, good.seq) == B.GS_OK
        _check_alone(good)
        time.sleep(0.2)  # the launch leaves after 20 ms without work
        again = _Req(n, 7, 7)
        assert again.submit(B, srv, 0) == B.GS_OK  # relaunches
        assert _wait(B, srv, 0, again.seq) == B.GS_OK
        _check_alone(again)
        assert B.gs_serve_stop(srv) == B.GS_OK
    finally:
        B.gs_serve_destroy(srv)


def test_stream_same_alone_and_in_the_mix():
    """A Poisson stream of 512^2 and 1024^2 requests through one server:
    sampled results against the same requests alone."""
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton
    from paper_1302_0120_gb300 import serving as SV

    summ, sch, ex = SV.run_persistent_service(rate_hz=2000.0, seconds=0.15, sizes=(512, 1024), slots=(4, 4),
                                              iters=30, record=True, warmup_s=0.0)
    ex.close()  # the server leaves before the runs alone
    done = sorted(sch.done, key=lambda r: r.rid)
    assert len(done) == summ["requests"] > 100
    assert {r.n for r in done} == {512, 1024}
    for r in done[:: max(1, len(done) // 10)]:
        with GerchbergSaxton(r.n, r.n) as gs:
            ph, res, _ = gs.run(torch.from_numpy(r.target).cuda(), torch.from_numpy(r.warm_in).cuda(), 30)
            assert gs.status() == 0
            ph, res = ph.cpu().numpy(), res.cpu().numpy()
        assert aligned_rel_err(r.phase, np.exp(1j * ph.astype(np.float64))) <= 1e-5, r.rid
        assert abs(r.residual - res[29]) <= 1e-3 * res[29], r.rid


def test_persistent_stream_meets_interspike_budget():
    from paper_1302_0120_gb300 import serving as SV

    summ, sch, ex = SV.run_persistent_service(rate_hz=1000.0, seconds=1.0, sizes=(512, 1024), slots=(8, 8),
                                              iters=30, warmup_s=0.2)
    ex.close()
    assert summ["requests"] > 800
    assert summ["p99_ms"] < 10.0, summ
