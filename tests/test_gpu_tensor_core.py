"""The tensor-core form (GS_TENSOR_CORE: FP16 DFT-matrix products with FP32
accumulation) against the FP64 oracle.

Gates, from the reduced-precision arithmetic (unit roundoff 2^-11 per FP16
operand, about 3e-4 relative L2 per transform, five transforms per step):
  * one step u -> u^{+1} from the same start: relative L2 <= 3e-3 (global
    phase removed);
  * the final residual r^K within 2% of the oracle's, and r^0 within 3e-3;
  * the chain r^nu >= g^nu >= r^{nu+1} to a relative slack of 5e-3 (the
    transforms are no longer exact, so neither are the projections).
"""

import numpy as np
import pytest

import oracle.gs_oracle as O
from paper_1302_0120_gb300 import synthetic as S
from tests.gpu_util import aligned_rel_err, GROUPING_RTOL

pytestmark = pytest.mark.gpu

STEP_TOL = 3e-3
FINAL_TOL = 0.02
CHAIN_SLACK = 5e-3


# Engines of the tensor-core form: tcgen05 with FP16 or BF16 operands, and
# the warp-level mma.sync products.
ENGINES = {"tcgen05-f16": {}, "tcgen05-bf16": {"bf16": True}, "mma-sync": {"mma_sync": True}}


def tc_run(I, phi0, iters, p=None, engine="tcgen05-f16"):
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton, build_lib

    build_lib.build()
    ny, nx = I.shape
    kw = ENGINES[engine]
    with GerchbergSaxton(nx, ny, tensor_core=True, **kw) as gs:
        pt = None
        if p is not None:
            pt = torch.from_numpy(p).cuda()
            gs.set_slm_amplitude(pt)
        ph, r, g = gs.run(torch.from_numpy(I).cuda(), torch.from_numpy(phi0).cuda(), iters)
        st = gs.status()
        from paper_1302_0120_gb300 import _binding as B

        assert B.gs_check_workspace(gs.handle) == B.GS_OK
        return ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy(), st


def check_chain(r, g):
    assert np.all(g <= r[:-1] * (1 + CHAIN_SLACK)), np.max(g / r[:-1])
    assert np.all(r[1:] <= g * (1 + CHAIN_SLACK)), np.max(r[1:] / g)


CASES = [(n, s, e) for n, s in ((256, 20), (512, 40), (1024, 50)) for e in ("tcgen05-f16", "tcgen05-bf16", "mma-sync")]


@pytest.mark.parametrize("n,nspots,engine", CASES)
def test_final_residual(n, nspots, engine):
    iters = 100 if n == 1024 else 50
    I = S.spot_target(70 + n, n, n, nspots, (0.5, 1.0))
    phi0 = S.random_phase(71 + n, n, n)
    ph, r, g, st = tc_run(I, phi0, iters, engine=engine)
    assert st == 0 and np.all(np.isfinite(ph)) and np.all(np.abs(ph) <= np.float32(np.pi))
    ref = O.gs_run(I, phi0, iters)
    assert abs(r[0] - ref["r"][0]) <= STEP_TOL * ref["r"][0], (r[0], ref["r"][0])
    assert abs(r[-1] - ref["r"][-1]) <= FINAL_TOL * ref["r"][-1], (r[-1], ref["r"][-1])
    check_chain(r, g)


@pytest.mark.parametrize("n,nspots,engine", CASES)
def test_one_step(n, nspots, engine):
    I = S.spot_target(80 + n, n, n, nspots, (0.5, 1.0))
    phi0 = S.random_phase(81 + n, n, n)
    start = O.gs_run(I, phi0, 5)["phase"].astype(np.float32)
    nxt, r, g, st = tc_run(I, start, 1, engine=engine)
    assert st == 0
    u_ref, r_ref, g_ref = O.gs_step(np.exp(1j * start.astype(np.float64)), O.target_amplitude(I))
    err = aligned_rel_err(nxt, u_ref)
    assert err <= STEP_TOL, err
    assert abs(r[0] - r_ref) <= STEP_TOL * r_ref and abs(g[0] - g_ref) <= STEP_TOL * g_ref


@pytest.mark.parametrize("n", [256, 512, 1024])
def test_batch_matches_single_runs(n):
    """Each mask of a batched launch has the single-mask run's phase, bit for
    bit, and its gaps to FP64 rounding (at 1024: tcgen05, whose products mix
    the lines of different masks in one M = 128 product)."""
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton, build_lib

    build_lib.build()
    nb, iters = 4, 12
    masks = [(S.spot_target(90 + k, n, n, 30, (0.5, 1.0)), S.random_phase(90 + k, n, n)) for k in range(nb)]
    It = torch.from_numpy(np.stack([m[0] for m in masks])).cuda()
    Pt = torch.from_numpy(np.stack([m[1] for m in masks])).cuda()
    with GerchbergSaxton(n, n, max_batch=nb, tensor_core=True) as gs:
        ph, r, g = gs.run_batched(It, Pt, iters)
        assert gs.status() == 0
        ph, r, g = ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy()
    for k, (I, phi0) in enumerate(masks):
        ph1, r1, g1, st = tc_run(I, phi0, iters)
        assert st == 0
        assert np.array_equal(ph[k], ph1)
        assert np.allclose(r[k], r1, rtol=GROUPING_RTOL, atol=0) and np.allclose(g[k], g1, rtol=GROUPING_RTOL, atol=0)


_ORACLE_FINAL = {}


def oracle_final_residual(k, I, phi0, iters):
    """The oracle's r^K of mask k of the mixed batch (computed once for the
    three engines)."""
    if k not in _ORACLE_FINAL:
        _ORACLE_FINAL[k] = O.gs_run(I, phi0, iters)["r"][-1]
    return _ORACLE_FINAL[k]


@pytest.mark.parametrize("engine", ["tcgen05-f16", "tcgen05-bf16", "mma-sync"])
def test_mixed_sizes_64_masks(engine):
    """64 masks drawn from 256, 512 and 1024 with 10..200 spots, 50 iterations
    in one persistent launch: every final residual within 2% of the oracle's
    (the oracle runs each mask at full size)."""
    import torch

    from paper_1302_0120_gb300 import MixedGerchbergSaxton, build_lib

    build_lib.build()
    iters = 50
    masks = S.mixed_batch(4)
    by_size = {}
    for k, (I, phi0) in enumerate(masks):
        by_size.setdefault(I.shape[0], []).append(k)
    assert len(by_size) == 3
    T = {n: torch.from_numpy(np.stack([masks[k][0] for k in ks])).cuda() for n, ks in by_size.items()}
    P = {n: torch.from_numpy(np.stack([masks[k][1] for k in ks])).cuda() for n, ks in by_size.items()}
    with MixedGerchbergSaxton({n: len(ks) for n, ks in by_size.items()}, tensor_core=True, **ENGINES[engine]) as gs:
        out = gs.run(T, P, iters)
        assert gs.status() == 0
    r_final = {}
    for n, ks in by_size.items():
        r, g = out[n][1].cpu().numpy(), out[n][2].cpu().numpy()
        for j, k in enumerate(ks):
            check_chain(r[j], g[j])
            r_final[k] = r[j][-1]
    worst = 0.0
    for k, (I, phi0) in enumerate(masks):
        ref = oracle_final_residual(k, I, phi0, iters)
        worst = max(worst, abs(r_final[k] - ref) / ref)
    assert worst <= FINAL_TOL, worst


def test_laser_amplitude():
    n, iters = 512, 30
    I = S.spot_target(95, n, n, 30, (0.5, 1.0))
    phi0 = S.random_phase(95, n, n)
    p = S.laser_amplitude(n, n)
    ph, r, g, st = tc_run(I, phi0, iters, p=p)
    assert st == 0
    ref = O.gs_run(I, phi0, iters, p=p)
    assert abs(r[-1] - ref["r"][-1]) <= FINAL_TOL * ref["r"][-1]
    check_chain(r, g)


@pytest.mark.parametrize("n,engine", [(n, e) for n in (256, 512, 1024) for e in ("tcgen05-f16", "tcgen05-bf16", "mma-sync")])
def test_large_laser_amplitude_is_rescaled(n, engine):
    """p = 100 everywhere: n sum p^2 = n^3 1e4 puts the raw transform inputs far
    beyond the FP16 range (65504); the per-mask power-of-two scale keeps the
    operands in range, and the run meets the one-step and final gates."""
    iters = 20
    I = S.spot_target(96, n, n, 20, (0.5, 1.0))
    phi0 = S.random_phase(96, n, n)
    p = np.full((n, n), 100.0, np.float32)
    ph, r, g, st = tc_run(I, phi0, iters, p=p, engine=engine)
    assert st == 0 and np.all(np.isfinite(r)) and np.all(np.isfinite(g))
    ref = O.gs_run(I, phi0, iters, p=p)
    assert abs(r[0] - ref["r"][0]) <= STEP_TOL * ref["r"][0], (r[0], ref["r"][0])
    assert abs(r[-1] - ref["r"][-1]) <= FINAL_TOL * ref["r"][-1], (r[-1], ref["r"][-1])
    check_chain(r, g)
    start = ref["phase"].astype(np.float32)
    nxt, _, _, st = tc_run(I, start, 1, p=p, engine=engine)
    assert st == 0
    u_ref, _, _ = O.gs_step(100.0 * np.exp(1j * start.astype(np.float64)), O.target_amplitude(I, energy=float(n * n) * 1e4),
                            p.astype(np.float64))
    assert aligned_rel_err(nxt, u_ref / 100.0) <= STEP_TOL
