"""One launch over masks of three sizes (gs_run_mixed) against one batched
launch per size: every mask takes the single-size path, so its phase is
bit-identical; its gaps agree to FP64 rounding (the per-block partial sums
are grouped by the launch's block count)."""

import numpy as np
import pytest

from paper_1302_0120_gb300 import synthetic as S
from tests.gpu_util import GROUPING_RTOL

pytestmark = pytest.mark.gpu


def masks_by_size(counts, seed):
    out = {}
    for n, cnt in counts.items():
        out[n] = [(S.spot_target(seed + 7 * k + n, n, n, 20 + 5 * k, (0.5, 1.0)), S.random_phase(seed + 7 * k + n, n, n))
                  for k in range(cnt)]
    return out


def stacked(ms, idx, init_from_target=False):
    import torch

    if idx == 1 and init_from_target:
        return None
    return {n: torch.from_numpy(np.stack([m[idx] for m in lst])).cuda() for n, lst in ms.items()}


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("counts,iters,from_target", [
    ({256: 3, 512: 2, 1024: 2}, 12, False),
    ({256: 2, 1024: 1}, 130, False),   # two chunks; no 512 class
    ({512: 2}, 5, False),              # one class only
    ({256: 1, 512: 1, 1024: 1}, 6, True),
])
def test_mixed_matches_per_size_launches(tc, counts, iters, from_target):
    from paper_1302_0120_gb300 import GerchbergSaxton, MixedGerchbergSaxton, build_lib

    build_lib.build()
    ms = masks_by_size(counts, 3)
    T, P = stacked(ms, 0), stacked(ms, 1, from_target)
    with MixedGerchbergSaxton(counts, tensor_core=tc, init_from_target=from_target) as gs:
        out = gs.run(T, P, iters)
        assert gs.status() == 0
        from paper_1302_0120_gb300 import _binding as B

        assert B.gs_check_workspace(gs.handle) == B.GS_OK
        out = {n: tuple(x.cpu().numpy() for x in v) for n, v in out.items()}
    for n in counts:
        with GerchbergSaxton(n, n, max_batch=counts[n], tensor_core=tc, init_from_target=from_target) as gs1:
            if from_target:
                import torch

                ph, r, g = gs1.run_batched(T[n], torch.zeros_like(T[n]), iters)  # phase_in ignored
            else:
                ph, r, g = gs1.run_batched(T[n], P[n], iters)
            assert gs1.status() == 0
            ph, r, g = ph.cpu().numpy(), r.cpu().numpy(), g.cpu().numpy()
        assert np.array_equal(out[n][0], ph), n
        assert np.allclose(out[n][1], r, rtol=GROUPING_RTOL, atol=0) and np.allclose(out[n][2], g, rtol=GROUPING_RTOL, atol=0), n


def test_mixed_rejects_one_mask():
    """A mask with an invalid target gets NaN gaps and GS_ENUMERIC; the
    others of every size are unaffected."""
    from paper_1302_0120_gb300 import GS_ENUMERIC, MixedGerchbergSaxton, build_lib

    build_lib.build()
    counts = {256: 2, 512: 2}
    ms = masks_by_size(counts, 5)
    T, P = stacked(ms, 0), stacked(ms, 1)
    T[512][1, 3, 3] = float("nan")
    with MixedGerchbergSaxton(counts) as gs:
        out = gs.run(T, P, 4)
        assert gs.status() == GS_ENUMERIC
        r = {n: v[1].cpu().numpy() for n, v in out.items()}
    assert np.all(np.isnan(r[512][1])) and np.all(np.isfinite(r[512][0])) and np.all(np.isfinite(r[256]))


@pytest.mark.parametrize("group", [1, 2])
def test_mask_groups_do_not_change_results(group):
    """gs_set_mask_group only reorders the work: phases bit-identical, gaps
    to FP64 rounding."""
    from paper_1302_0120_gb300 import GerchbergSaxton, MixedGerchbergSaxton, build_lib

    build_lib.build()
    counts = {256: 3, 512: 2}
    ms = masks_by_size(counts, 9)
    T, P = stacked(ms, 0), stacked(ms, 1)
    res = {}
    for g in (0, group):
        with MixedGerchbergSaxton(counts) as gs:
            gs.set_mask_group(g)
            out = gs.run(T, P, 7)
            assert gs.status() == 0
            res[g] = {n: tuple(x.cpu().numpy() for x in v) for n, v in out.items()}
        with GerchbergSaxton(512, 512, max_batch=2) as gs1:
            gs1.set_mask_group(g)
            ph, r, _ = gs1.run_batched(T[512], P[512], 7)
            assert gs1.status() == 0
            res[("single", g)] = (ph.cpu().numpy(), r.cpu().numpy())
    for n in counts:
        assert np.array_equal(res[0][n][0], res[group][n][0])
        assert np.allclose(res[0][n][1], res[group][n][1], rtol=GROUPING_RTOL, atol=0)
    assert np.array_equal(res[("single", 0)][0], res[("single", group)][0])
    assert np.allclose(res[("single", 0)][1], res[("single", group)][1], rtol=GROUPING_RTOL, atol=0)
