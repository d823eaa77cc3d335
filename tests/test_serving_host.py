"""Host-side logic of the serving loop, on CPU with a simulated device:
memory-based lane planning, admission of waiting requests as lanes free up,
FIFO order within a size class, overlap of lanes, and latency accounting."""

import numpy as np
import pytest

from paper_1302_0120_gb300 import serving as SV


def fake_workspace(nx, ny, b):
    return b * nx * ny * 24 + 600_000


class FakeExecutor:
    """A lane finishes `cost(n, b)` seconds after its launch."""

    def __init__(self, cost):
        self.cost = cost
        self.busy = {}
        self.batches = []

    def idle(self, p):
        return p.name not in self.busy

    def launch(self, p, reqs, now):
        self.busy[p.name] = (now + self.cost(p.n, len(reqs)), reqs)
        self.batches.append((p.name, now, [r.rid for r in reqs]))

    def poll(self, p, now):
        if p.name in self.busy and self.busy[p.name][0] <= now:
            t, reqs = self.busy.pop(p.name)
            for r in reqs:
                r.finish = t
            return reqs
        return []


class StepClock:
    def __init__(self, dt):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_plan_lanes_respects_budget_and_sms():
    plans = SV.plan_lanes([512, 1024], [1, 2], sm_count=152, budget_bytes=2 << 30, iters=30,
                          workspace_bytes=fake_workspace, max_batch_cap=16)
    assert [p.n for p in plans] == [512, 1024, 1024]
    assert sum(p.grid for p in plans) == 152
    assert plans[1].grid > plans[0].grid  # more SMs for the larger grids
    assert sum(p.bytes for p in plans) <= 2 << 30
    for p in plans:
        assert 1 <= p.max_batch <= 16
        assert p.bytes == SV.lane_bytes(p.n, p.max_batch, 30, fake_workspace)


def test_plan_lanes_shrinks_batches_with_budget():
    big = SV.plan_lanes([1024], [1], 152, 4 << 30, 30, fake_workspace)
    small = SV.plan_lanes([1024], [1], 152, 200 << 20, 30, fake_workspace)
    assert small[0].max_batch < big[0].max_batch
    with pytest.raises(ValueError):
        SV.plan_lanes([1024], [1], 152, 1 << 20, 30, fake_workspace)


def test_requests_join_as_lanes_free_up_and_lanes_overlap():
    plans = [SV.LanePlan("512/0", 512, 2, 40, 0), SV.LanePlan("1024/0", 1024, 3, 112, 0)]
    ex = FakeExecutor(lambda n, b: 1e-3 * (n / 512) * (1 + 0.25 * b))
    reqs = [SV.Request(i, 512 if i % 2 else 1024, np.zeros((1, 1), np.float32), arrival=0.0002 * i)
            for i in range(40)]
    sch = SV.serve(reqs, plans, ex, clock=StepClock(1e-5))
    assert len(sch.done) == 40 and all(r.finish is not None and r.finish >= r.arrival for r in sch.done)
    # FIFO within a size class and batch limits per lane
    for name, _, ids in ex.batches:
        assert len(ids) <= (2 if name.startswith("512") else 3)
    for n in (512, 1024):
        order = [rid for name, _, ids in ex.batches if name.startswith(str(n)) for rid in ids]
        assert order == sorted(order)
    # a request never waits while its lane is idle: it starts at its first tick
    first = min(sch.done, key=lambda r: r.arrival)
    assert first.start - first.arrival < 1e-4
    # the two lanes worked at the same time
    spans = {name: [(t, t + ex.cost(int(name.split('/')[0]), len(ids))) for nm, t, ids in ex.batches if nm == name]
             for name in ("512/0", "1024/0")}
    overlap = any(a0 < b1 and b0 < a1 for a0, a1 in spans["512/0"] for b0, b1 in spans["1024/0"])
    assert overlap
    s = SV.latency_summary(sch.done)
    assert s["requests"] == 40 and s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]


def test_poisson_stream_recipe():
    reqs = SV.poisson_stream(1000.0, 0.2, [64, 128], seed=3, neurons=50, subset=(5, 20))
    assert 120 < len(reqs) < 280
    t = [r.arrival for r in reqs]
    assert t == sorted(t) and t[-1] <= 0.2
    for r in reqs:
        assert r.target.shape == (r.n, r.n) and r.target.dtype == np.float32 and r.target.max() > 0
        assert r.target[0, 0] == 0  # DC kept dark


def test_plan_lanes_with_equal_weights_gives_every_lane_the_same_share():
    # the service's default: one 512 lane and two 1024 lanes, 152 SMs
    plans = SV.plan_lanes([512, 1024], [1, 2], sm_count=152, budget_bytes=2 << 30, iters=30,
                          workspace_bytes=fake_workspace, max_batch_cap=16, weights=[1.0, 1.0])
    grids = [p.grid for p in plans]
    assert sum(grids) == 152 and max(grids) - min(grids) <= 1


def test_plan_lanes_sharing_the_device():
    """Time-shared lanes: every grid is the whole device, batches still from
    the memory budget."""
    plans = SV.plan_lanes([512, 1024], [1, 2], sm_count=152, budget_bytes=2 << 30, iters=30,
                          workspace_bytes=fake_workspace, max_batch_cap=16, weights=[1.0, 1.0], share_sms=True)
    assert [p.grid for p in plans] == [152, 152, 152]
    split = SV.plan_lanes([512, 1024], [1, 2], sm_count=152, budget_bytes=2 << 30, iters=30,
                          workspace_bytes=fake_workspace, max_batch_cap=16, weights=[1.0, 1.0])
    assert [p.max_batch for p in plans] == [p.max_batch for p in split]
