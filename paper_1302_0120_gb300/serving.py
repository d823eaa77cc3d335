"""Continuous-batching request loop for phase masks.

The paper's use case is interactive: a new stimulation pattern must become a
phase mask within an interspike interval of 10-20 ms (Sec. I, IV.A). This
module serves a stream of such requests on one GPU:

* Requests carry a target intensity for an ``n x n`` grid. Each grid size is a
  *class*; a class has one or more *lanes*. A lane owns a batched context
  (gs_create_batched), a CUDA stream, device buffers for ``max_batch`` masks and
  a share of the SMs (its grid), so the lanes of all classes run concurrently.
* Admission is by memory: ``plan_lanes`` sizes every lane's batch from a device
  memory budget using the library's workspace size (gs_workspace_bytes_batched)
  plus the lane's own buffers.
* Whenever a lane is idle and requests of its class are waiting, the oldest
  ones (up to the lane's batch) are admitted and launched at once, while the
  other lanes keep working: requests that arrive while others are on the GPU
  join as soon as a lane frees up.
* Warm starts: every mask of a launch starts from the most recent mask of its
  lane (kept on the device, one warm-start buffer per lane); the last mask of
  a launch becomes that lane's next warm start. A class with several lanes
  therefore keeps one warm start per lane, not one for the class.
* Targets reach the lane from pinned host memory: a client renders each
  pattern into a buffer of a pinned pool before it submits the request (the
  loop stages upcoming requests this way while it has nothing else to do;
  a request staged late pays for the copy in its latency), and the launch
  copies it to the device on the lane's stream. The rest of the per-launch
  sequence (warm-start copies, the batched run, the warm-start update) is
  captured once per lane and batch size as a CUDA graph and replayed.
* The loop either spins on the lanes' completion events or sleeps until the
  next arrival or the next completion, which the library signals through an
  eventfd (gs_stream_notify) from the end of each launch.

``PersistentExecutor`` and ``run_persistent_service`` serve through the
library's persistent server instead (gs_serve_create): one launch on the
whole device keeps iterating, and a request posted to a free slot joins the
running ones at their next iteration, with no launch per request.

Every step of the method runs in the CUDA library; this module only moves
buffers and decides what to launch when.
"""

from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    n: int                      # grid is n x n
    target: np.ndarray          # float32 [n, n] intensity, DFT order
    arrival: float              # seconds, server clock
    start: Optional[float] = None
    finish: Optional[float] = None
    lane: Optional[str] = None
    launch_id: int = -1
    slot: int = -1
    warm_in: Optional[np.ndarray] = None   # kept when the server records inputs
    phase: Optional[np.ndarray] = None     # kept when the server records results
    residual: Optional[float] = None
    pinned: Optional[object] = None        # the target in a pinned host buffer of the client's pool

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclasses.dataclass
class LanePlan:
    name: str
    n: int
    max_batch: int
    grid: int
    bytes: int


def lane_bytes(n: int, max_batch: int, iters: int, workspace_bytes: Callable[[int, int, int], int]) -> int:
    """Device bytes of one lane: library workspace + the lane's own buffers
    (targets, phases: 4 B/px each per slot; residuals; one warm-start mask)."""
    px = n * n
    own = max_batch * (8 * px + 16 * (iters + 1)) + 4 * px
    return int(workspace_bytes(n, n, max_batch)) + own


def plan_lanes(sizes: Sequence[int], lanes_per_size: Sequence[int], sm_count: int, budget_bytes: int, iters: int,
               workspace_bytes: Callable[[int, int, int], int], max_batch_cap: int = 16,
               weights: Optional[Sequence[float]] = None, share_sms: bool = False) -> List[LanePlan]:
    """Split the SMs and the memory budget among the lanes.

    SMs go to each size in proportion to its expected work (``weights``,
    default n^2 log n per request, equal request rates) and then evenly to its
    lanes. Each lane gets the largest batch (<= max_batch_cap) whose bytes fit
    its share of the budget, which is split in the same proportion. Raises
    ValueError when a lane cannot hold even one mask. With ``share_sms`` every
    lane's grid is the whole device instead: the lanes' launches time-share
    the SMs (a launch starts when the previous one leaves room for all its
    blocks) instead of running side by side on disjoint shares.
    """
    if weights is None:
        weights = [n * n * math.log2(n) for n in sizes]
    tot_w = float(sum(w * k for w, k in zip(weights, lanes_per_size)))
    plans = []
    sm_left = sm_count
    nl_total = sum(lanes_per_size)
    for si, (n, nl) in enumerate(zip(sizes, lanes_per_size)):
        for li in range(nl):
            share = weights[si] / tot_w
            grid = max(1, int(sm_count * share))
            mem = int(budget_bytes * share)
            b = max_batch_cap
            while b >= 1 and lane_bytes(n, b, iters, workspace_bytes) > mem:
                b -= 1
            if b < 1:
                raise ValueError(f"memory budget too small for one {n}x{n} mask")
            plans.append(LanePlan(f"{n}/{li}", n, b, grid, lane_bytes(n, b, iters, workspace_bytes)))
            sm_left -= grid
    if share_sms:
        for p in plans:
            p.grid = sm_count
        return plans
    # hand SMs lost to rounding to the largest lanes, never exceeding the device
    i = 0
    while sm_left > 0 and plans:
        plans[i % len(plans)].grid += 1
        sm_left -= 1
        i += 1
    assert sum(p.grid for p in plans) <= sm_count or nl_total > sm_count
    return plans


class Scheduler:
    """Admission and dispatch, independent of the device.

    ``executor`` has ``idle(lane) -> bool``, ``launch(lane, reqs, now)`` and
    ``poll(lane, now) -> list of finished requests``.
    """

    def __init__(self, plans: Sequence[LanePlan], executor):
        self.plans = list(plans)
        self.ex = executor
        self.pending: Dict[int, collections.deque] = collections.defaultdict(collections.deque)
        self.done: List[Request] = []
        self.launches = 0

    def submit(self, req: Request):
        self.pending[req.n].append(req)

    def tick(self, now: float) -> int:
        """Collect finished work, then admit waiting requests to idle lanes.
        Returns the number of requests admitted."""
        for p in self.plans:
            self.done.extend(self.ex.poll(p, now))
        admitted = 0
        for p in self.plans:
            q = self.pending[p.n]
            if q and self.ex.idle(p):
                take = [q.popleft() for _ in range(min(p.max_batch, len(q)))]
                for r in take:
                    r.start = now
                    r.lane = p.name
                self.ex.launch(p, take, now)
                self.launches += 1
                admitted += len(take)
        return admitted

    def busy(self) -> bool:
        return any(self.pending[n] for n in self.pending) or any(not self.ex.idle(p) for p in self.plans)


class GpuExecutor:
    """Runs lanes on the GPU through the C ABI (batched runs, graph replay).

    ``notify=True`` creates an eventfd (``self.fd``) that the end of every
    launch writes through gs_stream_notify, for loops that sleep."""

    def __init__(self, plans: Sequence[LanePlan], iters: int, device=None, use_graphs: bool = True,
                 record: bool = False, warm_seed: int = 7, notify: bool = False, pool_extra: int = 16):
        import os

        import torch

        from . import _binding as B
        from .synthetic import random_phase

        self.torch = torch
        self.B = B
        self.iters = iters
        self.record = record
        self.use_graphs = use_graphs
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.fd = os.eventfd(0, os.EFD_NONBLOCK) if notify else None
        self.lanes = {}
        slots = collections.Counter()
        for p in plans:
            n, mb = p.n, p.max_batch
            slots[n] += mb
            st = torch.cuda.Stream(device=self.device)
            h = B.gs_create_batched(n, n, mb, B.GS_FINAL_RESIDUAL, st.cuda_stream)
            rc = B.gs_set_grid(h, p.grid)
            if rc != B.GS_OK:
                raise B.GSError(rc, "gs_set_grid")
            L = {
                "plan": p,
                "stream": st,
                "handle": h,
                "I": torch.empty((mb, n, n), dtype=torch.float32, device=self.device),
                "P": torch.empty((mb, n, n), dtype=torch.float32, device=self.device),
                "R": torch.empty((mb, iters + 1), dtype=torch.float64, device=self.device),
                "G": torch.empty((mb, max(iters, 1)), dtype=torch.float64, device=self.device),
                "hI": torch.empty((mb, n, n), dtype=torch.float32).pin_memory(),
                "warm": torch.from_numpy(random_phase(warm_seed, n, n)).to(self.device),
                "graphs": {},
                "busy": None,
                "launch_id": 0,
            }
            self.lanes[p.name] = L
        # the clients' pinned buffers: enough for every lane's batch plus the
        # requests staged ahead of their arrival
        self.pool = {n: [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(k + pool_extra)]
                     for n, k in slots.items()}
        self.graph_ok = use_graphs

    # -- the launch sequence of one lane for b masks (targets already in L["I"])
    def _enqueue(self, L, b):
        n = L["plan"].n
        L["P"][:b].copy_(L["warm"].expand(b, n, n))
        rc = self.B.gs_run_batched(L["handle"], b, L["I"].data_ptr(), L["P"].data_ptr(), self.iters,
                                   L["P"].data_ptr(), L["R"].data_ptr(), L["G"].data_ptr())
        if rc != self.B.GS_OK:
            raise self.B.GSError(rc, "gs_run_batched")
        L["warm"].copy_(L["P"][b - 1])

    def _graph(self, L, b):
        torch = self.torch
        g = L["graphs"].get(b)
        if g is None and self.graph_ok:
            try:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=L["stream"]):
                    self._enqueue(L, b)
                L["graphs"][b] = g
            except Exception:
                self.graph_ok = False  # capture unsupported here: launch directly
                torch.cuda.synchronize(self.device)
                g = None
        return g

    def stage(self, r: Request) -> bool:
        """Copy a request's target into a pinned buffer of the pool (the
        client's side of a submission). False when the pool is empty."""
        if r.pinned is not None:
            return True
        pool = self.pool.get(r.n)
        if not pool:
            return False
        buf = pool.pop()
        buf.copy_(self.torch.from_numpy(r.target))
        r.pinned = buf
        return True

    def idle(self, p: LanePlan) -> bool:
        return self.lanes[p.name]["busy"] is None

    def launch(self, p: LanePlan, reqs: List[Request], now: float):
        torch = self.torch
        L = self.lanes[p.name]
        b = len(reqs)
        srcs = []
        for k, r in enumerate(reqs):
            if not self.stage(r):  # no pinned buffer left: through the lane's own
                L["hI"][k].copy_(torch.from_numpy(r.target))
            srcs.append(r.pinned if r.pinned is not None else L["hI"][k])
            r.slot = k
            r.launch_id = L["launch_id"]
        if self.record:  # the lane is idle, so its warm start is final
            warm = L["warm"].cpu().numpy()
            for r in reqs:
                r.warm_in = warm
        with torch.cuda.stream(L["stream"]):
            for k, src in enumerate(srcs):
                L["I"][k].copy_(src, non_blocking=True)
            g = self._graph(L, b)
            if g is not None:
                g.replay()
            else:
                self._enqueue(L, b)
            ev = torch.cuda.Event()
            ev.record(L["stream"])
        if self.fd is not None:
            rc = self.B.gs_stream_notify(L["stream"].cuda_stream, self.fd)
            if rc != self.B.GS_OK:
                raise self.B.GSError(rc, "gs_stream_notify")
        L["busy"] = (ev, reqs)
        L["launch_id"] += 1

    def poll(self, p: LanePlan, now: float) -> List[Request]:
        L = self.lanes[p.name]
        if L["busy"] is None:
            return []
        ev, reqs = L["busy"]
        if not ev.query():
            return []
        L["busy"] = None
        st = self.B.gs_status(L["handle"])
        if st != self.B.GS_OK:
            raise self.B.GSError(st, "serving launch")
        if self.record:
            P = L["P"][: len(reqs)].cpu().numpy()
            R = L["R"][: len(reqs), self.iters].cpu().numpy()
            for k, r in enumerate(reqs):
                r.phase = P[k].copy()
                r.residual = float(R[k])
        for r in reqs:
            r.finish = now
            if r.pinned is not None:  # the copy to the device is done: back to the pool
                self.pool[r.n].append(r.pinned)
                r.pinned = None
        return reqs

    def wait(self, timeout: float):
        """Sleep until a launch completes (its notification) or `timeout` s."""
        import os
        import select

        if timeout > 0:
            select.select([self.fd], [], [], timeout)
        try:
            os.eventfd_read(self.fd)
        except BlockingIOError:
            pass

    def close(self):
        import os

        for L in self.lanes.values():
            L["graphs"].clear()
            self.B.gs_destroy(L["handle"])
        self.lanes = {}
        if self.fd is not None:
            self.torch.cuda.synchronize(self.device)  # every notification has run
            os.close(self.fd)
            self.fd = None


class PersistentExecutor:
    """Serves through one persistent server (gs_serve_create) on the whole
    device: its slots are dedicated to the sizes (``slots[i]`` slots for
    ``sizes[i]``), each slot a lane of one request. A request posted to a free
    slot joins the server's running requests, of every size, at its next
    iteration; the host only writes the request table and reads completions.
    The target and the phase stay in pinned host memory that the server reads
    and writes in place; every slot warm-starts from its own last mask."""

    def __init__(self, sizes: Sequence[int], slots: Sequence[int], iters: int, grid: int = 0, device=None,
                 record: bool = False, warm_seed: int = 7, pool_extra: int = 16):
        import torch

        from . import _binding as B
        from .synthetic import random_phase

        self.torch = torch
        self.B = B
        self.iters = iters
        self.record = record
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.Stream(device=self.device)
        self.server = B.gs_serve_create(max(sizes), sum(slots), grid, self.stream.cuda_stream)
        self.grid = B.gs_serve_grid(self.server)
        self.lanes = {}
        self.plans: List[LanePlan] = []
        k = 0
        for n, s in zip(sizes, slots):
            for _ in range(s):
                p = LanePlan(f"{n}/{k}", n, 1, self.grid, 12 * n * n)
                self.plans.append(p)
                self.lanes[p.name] = {
                    "plan": p, "slot": k,
                    "warm": torch.from_numpy(random_phase(warm_seed, n, n)).pin_memory(),
                    "hI": torch.empty((n, n), dtype=torch.float32).pin_memory(),
                    "R": torch.zeros(max(iters, 1), dtype=torch.float64).pin_memory(),
                    "G": torch.zeros(max(iters, 1), dtype=torch.float64).pin_memory(),
                    "busy": None,
                }
                k += 1
        self.pool = {n: [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(s + pool_extra)]
                     for n, s in zip(sizes, slots)}
        self.graph_ok = False

    def stage(self, r: Request) -> bool:
        if r.pinned is not None:
            return True
        pool = self.pool.get(r.n)
        if not pool:
            return False
        buf = pool.pop()
        buf.copy_(self.torch.from_numpy(r.target))
        r.pinned = buf
        return True

    def idle(self, p: LanePlan) -> bool:
        return self.lanes[p.name]["busy"] is None

    def launch(self, p: LanePlan, reqs: List[Request], now: float):
        L = self.lanes[p.name]
        (r,) = reqs
        if not self.stage(r):
            L["hI"].copy_(self.torch.from_numpy(r.target))
        src = r.pinned if r.pinned is not None else L["hI"]
        if self.record:
            r.warm_in = L["warm"].numpy().copy()
        r.slot = L["slot"]
        rc, seq = self.B.gs_serve_submit(self.server, L["slot"], r.n, src.data_ptr(), L["warm"].data_ptr(), self.iters,
                                         L["warm"].data_ptr(), L["R"].data_ptr(), L["G"].data_ptr())
        if rc != self.B.GS_OK:
            raise self.B.GSError(rc, "gs_serve_submit")
        L["busy"] = (seq, r)

    def poll(self, p: LanePlan, now: float) -> List[Request]:
        L = self.lanes[p.name]
        if L["busy"] is None:
            return []
        seq, r = L["busy"]
        rc, done, st = self.B.gs_serve_poll(self.server, L["slot"])
        if rc != self.B.GS_OK:
            raise self.B.GSError(rc, "persistent server")
        if done != seq:
            return []
        if st != self.B.GS_OK:
            raise self.B.GSError(st, f"request {r.rid}")
        L["busy"] = None
        r.finish = now
        if self.record:
            r.phase = L["warm"].numpy().copy()
            r.residual = float(L["R"][self.iters - 1])
        if r.pinned is not None:
            self.pool[r.n].append(r.pinned)
            r.pinned = None
        return [r]

    def close(self):
        if self.server:
            self.B.gs_serve_destroy(self.server)
            self.server = None


def serve(arrivals: Sequence[Request], plans: Sequence[LanePlan], executor, clock=time.perf_counter,
          t0: Optional[float] = None, lookahead_s: float = 0.002, wait: str = "spin") -> Scheduler:
    """Run the request loop until every request in ``arrivals`` (sorted by
    arrival time, relative to ``t0``) is finished. Returns the scheduler; the
    finished requests are in ``scheduler.done`` with their times.

    While it has nothing else to do, the loop plays the clients' part for the
    requests due within ``lookahead_s``: their targets go into pinned buffers
    (``executor.stage``) before they are submitted. ``wait="event"`` sleeps
    between events (``executor.wait``: a completion, or the next arrival)
    instead of spinning."""
    sch = Scheduler(plans, executor)
    t0 = clock() if t0 is None else t0
    i = 0
    total = len(arrivals)
    stage = getattr(executor, "stage", None)
    sleep = wait == "event" and getattr(executor, "fd", None) is not None
    staged = 0
    while len(sch.done) < total:
        now = clock() - t0
        while i < total and arrivals[i].arrival <= now:
            sch.submit(arrivals[i])
            i += 1
        sch.tick(now)
        if stage is not None:
            staged = max(staged, i)
            while staged < total and arrivals[staged].arrival <= now + lookahead_s and stage(arrivals[staged]):
                staged += 1
        if sleep and not any(sch.pending[p.n] and executor.idle(p) for p in plans):
            # nothing to launch: sleep until a completion or the next arrival
            nxt = arrivals[i].arrival - (clock() - t0) if i < total else 0.05
            executor.wait(min(max(nxt, 0.0), 0.05))
    return sch


def poisson_stream(rate_hz: float, seconds: float, sizes: Sequence[int], seed: int, neurons: int = 200,
                   subset=(5, 100), amp_range=(0.5, 1.0)) -> List[Request]:
    """Requests at Poisson times; each picks a size uniformly and a random
    subset of a fixed set of neuron positions of that size, rendered as spots."""
    from . import synthetic as S

    rng = np.random.default_rng(seed)
    pos = {n: S.neuron_positions(seed, neurons, n, n) for n in sizes}
    t = 0.0
    out = []
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > seconds:
            break
        n = sizes[int(rng.integers(0, len(sizes)))]
        k = int(rng.integers(subset[0], subset[1] + 1))
        pick = rng.choice(neurons, size=k, replace=False)
        amps = rng.uniform(amp_range[0], amp_range[1], size=k)
        out.append(Request(rid, n, S.render_spots(pos[n][pick], amps, n, n), t))
        rid += 1
    return out


def latency_summary(done: Sequence[Request]) -> dict:
    lat = np.array([r.latency for r in done]) * 1e3
    by_n = collections.defaultdict(list)
    for r in done:
        by_n[r.n].append(r.latency * 1e3)
    return {
        "requests": len(done),
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "max_ms": float(lat.max()),
        "by_size": {str(n): {"requests": len(v), "p50_ms": float(np.percentile(v, 50)),
                             "p99_ms": float(np.percentile(v, 99))} for n, v in sorted(by_n.items())},
    }


def run_service(rate_hz: float = 1000.0, seconds: float = 10.0, sizes=(512, 1024), lanes=(1, 2), iters: int = 30,
                budget_bytes: int = 2 << 30, seed: int = 0, max_batch_cap: int = 16, record: bool = False,
                use_graphs: bool = True, warmup_s: float = 0.5, weights=None, wait: str = "spin",
                share_sms: bool = True):
    """Serve a Poisson stream on the current GPU; returns (summary, scheduler, executor).

    By default every lane's launches use the whole device and time-share it
    (``share_sms``): at 512^2 and 1024^2 a mask's latency is set by the fixed
    cost of each pass, which a share of the SMs stretches (about 1.3 ms for a
    1024^2 mask on a third of the device against 0.5 ms on all of it), while
    at 1 kHz the device is busy less than half the time. On one GB300 (1 kHz,
    50/50 sizes, 30 iterations, one 512 lane and two 1024 lanes): p50 / p99
    0.59 / 2.11 ms time-sharing, 1.22 / 3.08 ms on disjoint equal shares (and
    1.54 / 2.60 ms with three 1024 lanes). ``weights`` splits the SMs among the
    sizes when the lanes do not share them (see plan_lanes)."""
    import torch

    from . import _binding as B
    from . import build_lib

    build_lib.build()
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    if weights is None:
        weights = [1.0] * len(sizes)
    plans = plan_lanes(list(sizes), list(lanes), sm, budget_bytes, iters,
                       lambda nx, ny, b: B.gs_workspace_bytes_batched(nx, ny, b, B.GS_FINAL_RESIDUAL),
                       max_batch_cap=max_batch_cap, weights=weights, share_sms=share_sms)
    ex = GpuExecutor(plans, iters, use_graphs=use_graphs, record=record, notify=(wait == "event"))
    if warmup_s > 0:  # capture every graph and warm the lanes, untimed
        warm = poisson_stream(rate_hz, warmup_s, sizes, seed + 1)
        serve(warm, plans, ex, wait=wait)
        for p in plans:
            for b in range(1, p.max_batch + 1):
                ex._graph(ex.lanes[p.name], b)
        torch.cuda.synchronize()
    reqs = poisson_stream(rate_hz, seconds, sizes, seed)
    sch = serve(reqs, plans, ex, wait=wait)
    summ = latency_summary(sch.done)
    summ.update({
        "rate_hz": rate_hz, "seconds": seconds, "iters": iters, "launches": sch.launches,
        "lanes": [dataclasses.asdict(p) for p in plans], "graphs": ex.graph_ok, "wait": wait, "share_sms": share_sms,
        "throughput_masks_per_s": len(sch.done) / max(max(r.finish for r in sch.done), 1e-9),
    })
    return summ, sch, ex


def run_persistent_service(rate_hz: float = 1000.0, seconds: float = 10.0, sizes=(512, 1024), slots=(8, 8),
                           iters: int = 30, seed: int = 0, record: bool = False, warmup_s: float = 0.5, grid: int = 0):
    """Serve a Poisson stream through one persistent server on the whole
    device (``grid`` blocks; 0: one per SM); returns (summary, scheduler,
    executor)."""
    from . import build_lib

    build_lib.build()
    ex = PersistentExecutor(sizes, slots, iters, grid=grid, record=record)
    if warmup_s > 0:
        serve(poisson_stream(rate_hz, warmup_s, sizes, seed + 1), ex.plans, ex)
    reqs = poisson_stream(rate_hz, seconds, sizes, seed)
    sch = serve(reqs, ex.plans, ex)
    summ = latency_summary(sch.done)
    summ.update({
        "rate_hz": rate_hz, "seconds": seconds, "iters": iters, "mode": "persistent",
        "slots": {str(n): s for n, s in zip(sizes, slots)}, "grid": ex.grid,
        "throughput_masks_per_s": len(sch.done) / max(max(r.finish for r in sch.done), 1e-9),
    })
    return summ, sch, ex


def persistent_tick_us(sizes=(512, 1024), k_short: int = 10, k_long: int = 70, reps: int = 12, seed: int = 1):
    """Time of one server iteration (tick) per size, from lone requests of
    k_short and k_long iterations timed from post to observed completion:
    (t_long - t_short) / (k_long - k_short); also the lone latencies (ms).
    The server leaves before it returns."""
    import statistics

    import torch

    from . import _binding as B
    from . import build_lib
    from . import synthetic as S

    build_lib.build()
    out = {}
    srv = B.gs_serve_create(max(sizes), 1, 0, None)
    try:
        for n in sizes:
            I = torch.from_numpy(S.spot_target(seed, n, n, 30, (0.5, 1.0))).pin_memory()
            ph = torch.from_numpy(S.random_phase(seed, n, n)).pin_memory()
            r = torch.zeros(k_long, dtype=torch.float64).pin_memory()
            g = torch.zeros(k_long, dtype=torch.float64).pin_memory()
            lat = {}
            for K in (k_short, k_long):
                ts = []
                for _ in range(reps):
                    t0 = time.perf_counter()
                    rc, seq = B.gs_serve_submit(srv, 0, n, I.data_ptr(), ph.data_ptr(), K, ph.data_ptr(),
                                                r.data_ptr(), g.data_ptr())
                    if rc != B.GS_OK:
                        raise B.GSError(rc, "gs_serve_submit")
                    while True:
                        rc, done, st = B.gs_serve_poll(srv, 0)
                        if rc != B.GS_OK:
                            raise B.GSError(rc, "gs_serve_poll")
                        if done == seq:
                            break
                    ts.append((time.perf_counter() - t0) * 1e3)
                    time.sleep(0.002)
                lat[K] = statistics.median(ts[2:])
            out[str(n)] = {"tick_us": round((lat[k_long] - lat[k_short]) / (k_long - k_short) * 1e3, 2),
                           f"lone_ms_k{k_short}": round(lat[k_short], 4), f"lone_ms_k{k_long}": round(lat[k_long], 4)}
    finally:
        B.gs_serve_destroy(srv)
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="serve a Poisson stream of phase-mask requests")
    ap.add_argument("--rate", type=float, default=1000.0)
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--wait", choices=["spin", "event"], default="spin")
    ap.add_argument("--lanes", default="1,2", help="lanes per size (512, 1024)")
    ap.add_argument("--split-sms", action="store_true", help="lanes on disjoint shares of the SMs")
    a = ap.parse_args()
    s, _, ex = run_service(a.rate, a.seconds, iters=a.iters, use_graphs=not a.no_graphs, wait=a.wait,
                           lanes=tuple(int(x) for x in a.lanes.split(",")), share_sms=not a.split_sms)
    ex.close()
    print(json.dumps(s))
