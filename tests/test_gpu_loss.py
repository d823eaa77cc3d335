"""The differentiable form on the GPU against the FP64 oracle.

Loss: relative error <= 1e-4; gradient (hand-written adjoint): relative L2
error <= 1e-3 against the oracle's analytic gradient, which is itself pinned
to central finite differences in FP64 (tests/test_oracle_pins.py)."""

import numpy as np
import pytest

import oracle.gs_oracle as O
from paper_1302_0120_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def normalized_target(seed, n, nspots):
    I = S.spot_target(seed, n, n, nspots, (0.5, 1.0)).astype(np.float64)
    I *= I.size / I.sum()  # sum I = N
    return I.astype(np.float32)


def gpu_loss_grad(I, phi, want_grad=True):
    import torch

    from paper_1302_0120_gb300 import build_lib
    from paper_1302_0120_gb300.differentiable import LossContext

    build_lib.build()
    lc = LossContext(I.shape[0])
    loss, grad = lc.loss_grad(torch.from_numpy(I).cuda(), torch.from_numpy(phi).cuda(), want_grad)
    st = lc.status()
    out = (float(loss.item()), grad.cpu().numpy() if grad is not None else None, st)
    lc.close()
    return out


@pytest.mark.parametrize("n,nspots", [(32, 4), (64, 6), (256, 30), (1024, 100)])
def test_loss_and_gradient_match_oracle(n, nspots):
    I = normalized_target(n, n, nspots)
    phi = S.random_phase(n + 1, n, n)
    loss, grad, st = gpu_loss_grad(I, phi)
    assert st == 0
    ref_l = O.intensity_loss(phi, I)
    ref_g = O.intensity_loss_grad(phi, I)
    assert abs(loss - ref_l) <= 1e-4 * ref_l, (loss, ref_l)
    err = np.linalg.norm(grad - ref_g) / np.linalg.norm(ref_g)
    assert err <= 1e-3, err
    loss_only, none, st = gpu_loss_grad(I, phi, want_grad=False)
    assert st == 0 and none is None and loss_only == loss


@pytest.mark.parametrize("n,nspots", [(64, 6), (1024, 100)])
def test_prepared_target_matches_fused_call(n, nspots):
    """gs_loss_prepare + gs_loss_grad_prepared give the fused call's loss and
    gradient bit for bit (the same passes on the same staged target), call
    after call, and both match the oracle; a new phase needs no new prepare."""
    import torch

    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300.differentiable import LossContext

    I = normalized_target(40 + n, n, nspots)
    It = torch.from_numpy(I).cuda()
    lc = LossContext(n)
    lc.prepare(It)
    for k in range(3):
        phi = S.random_phase(41 + n + k, n, n)
        Pt = torch.from_numpy(phi).cuda()
        l_p, g_p = lc.loss_grad_prepared(Pt)
        l_p, g_p = float(l_p.item()), g_p.cpu().numpy()
        assert lc.status() == 0
        lc2 = LossContext(n)
        l_f, g_f = lc2.loss_grad(It, Pt)
        assert lc2.status() == 0
        assert l_p == float(l_f.item()) and np.array_equal(g_p, g_f.cpu().numpy())
        lc2.close()
        ref_l = O.intensity_loss(phi, I)
        assert abs(l_p - ref_l) <= 1e-4 * ref_l
        if n <= 64:
            ref_g = O.intensity_loss_grad(phi, I)
            assert np.linalg.norm(g_p - ref_g) / np.linalg.norm(ref_g) <= 1e-3
    # an iteration run on the same context overwrites the staged target
    from paper_1302_0120_gb300 import GerchbergSaxton  # noqa: F401

    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    out = torch.empty_like(It)
    r = torch.empty(3, dtype=torch.float64, device="cuda")
    assert B.gs_run(lc.handle, It.data_ptr(), Pt.data_ptr(), 2, out.data_ptr(), r.data_ptr(), 0) == 0
    assert lc.status() == 0
    assert B.gs_loss_grad_prepared(lc.handle, Pt.data_ptr(), loss.data_ptr(), 0) == B.GS_EINVAL
    lc.close()


def test_prepared_nonfinite_target():
    import torch

    from paper_1302_0120_gb300 import GS_ENUMERIC
    from paper_1302_0120_gb300.differentiable import LossContext

    n = 64
    I = normalized_target(44, n, 6)
    I[5, 7] = np.nan
    lc = LossContext(n)
    lc.prepare(torch.from_numpy(I).cuda())
    assert lc.status() == GS_ENUMERIC
    loss, _ = lc.loss_grad_prepared(torch.from_numpy(S.random_phase(45, n, n)).cuda())
    assert lc.status() == GS_ENUMERIC and np.isnan(loss.item())
    lc.close()


def test_autograd_and_adam():
    import torch

    from paper_1302_0120_gb300.differentiable import LossContext, intensity_loss, optimize_phase

    n = 256
    I = torch.from_numpy(normalized_target(5, n, 30)).cuda()
    phi0 = torch.from_numpy(S.random_phase(6, n, n)).cuda()
    lc = LossContext(n)
    phase = phi0.clone().requires_grad_(True)
    loss = intensity_loss(phase, I, lc)
    (2.5 * loss).backward()
    _, g = lc.loss_grad(I, phi0)
    assert torch.allclose(phase.grad, 2.5 * g, rtol=1e-6, atol=0)
    ph, losses = optimize_phase(I, phi0, steps=60, lr=0.05, lctx=lc)
    assert lc.status() == 0
    assert losses[-1] < 0.5 * losses[0], losses[[0, -1]]
    lc.close()


def test_adam_step_matches_torch_adam():
    """gs_adam_step against torch's Adam (single-tensor form) on the same
    gradients over five steps."""
    import torch

    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300 import build_lib

    build_lib.build()
    n = 300_001  # not a multiple of the block size
    gen = torch.Generator(device="cuda").manual_seed(3)
    p0 = torch.rand(n, device="cuda", generator=gen) * 6.0
    ours = p0.clone()
    m = torch.zeros_like(ours)
    v = torch.zeros_like(ours)
    state = torch.zeros(2, dtype=torch.int32, device="cuda")
    ref = p0.clone().requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=0.05, betas=(0.9, 0.999), eps=1e-8, foreach=False)
    for k in range(5):
        g = torch.randn(n, device="cuda", generator=gen) * (10.0 ** (k - 2))
        assert B.gs_adam_step(ours.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), n, state.data_ptr(),
                              0.05, 0.9, 0.999, 1e-8, torch.cuda.current_stream().cuda_stream) == 0
        ref.grad = g.clone()
        opt.step()
    torch.cuda.synchronize()
    assert state.tolist() == [5, 0]
    assert torch.allclose(ours, ref.detach(), rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("n", [256, 1024])
def test_fused_adam_step_matches_separate_launches(n):
    """gs_loss_adam_prepared (the update in the gradient pass) against
    gs_loss_grad_prepared followed by gs_adam_step, over six steps from the
    same start: the same losses, moments, step count and phases."""
    import torch

    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300 import build_lib

    build_lib.build()
    I = torch.from_numpy(normalized_target(5, n, 40)).cuda()
    phi0 = torch.from_numpy(S.random_phase(6, n, n)).cuda()
    h1, h2 = B.gs_create(n, n), B.gs_create(n, n)
    try:
        assert B.gs_loss_prepare(h1, I.data_ptr()) == 0 and B.gs_loss_prepare(h2, I.data_ptr()) == 0
        ph1, ph2 = phi0.clone(), phi0.clone()
        m1, v1, m2, v2 = (torch.zeros_like(phi0) for _ in range(4))
        st1 = torch.zeros(2, dtype=torch.int32, device="cuda")
        st2 = torch.zeros(2, dtype=torch.int32, device="cuda")
        l1 = torch.zeros(6, dtype=torch.float64, device="cuda")
        l2 = torch.zeros(6, dtype=torch.float64, device="cuda")
        g = torch.empty_like(phi0)
        stream = torch.cuda.current_stream().cuda_stream
        for k in range(6):
            assert B.gs_loss_adam_prepared(h1, ph1.data_ptr(), m1.data_ptr(), v1.data_ptr(), st1.data_ptr(),
                                           0.05, 0.9, 0.999, 1e-8, l1[k:].data_ptr()) == 0
            assert B.gs_loss_grad_prepared(h2, ph2.data_ptr(), l2[k:].data_ptr(), g.data_ptr()) == 0
            assert B.gs_adam_step(ph2.data_ptr(), g.data_ptr(), m2.data_ptr(), v2.data_ptr(), n * n, st2.data_ptr(),
                                  0.05, 0.9, 0.999, 1e-8, stream) == 0
        torch.cuda.synchronize()
        assert B.gs_status(h1) == 0 and B.gs_status(h2) == 0
        assert st1.tolist() == st2.tolist() == [6, 0]
        assert torch.allclose(l1, l2, rtol=1e-6, atol=0)
        assert torch.allclose(m1, m2, rtol=1e-6, atol=1e-12) and torch.allclose(v1, v2, rtol=1e-6, atol=1e-20)
        assert torch.allclose(ph1, ph2, rtol=0, atol=1e-6)
        assert l1[5] < l1[0]
    finally:
        B.gs_destroy(h1)
        B.gs_destroy(h2)


def single_launch_steps(h, I, phi0, steps, n):
    """`steps` gs_loss_adam_prepared launches from phi0 on the staged target I,
    then the final loss: (losses, phase, m, v, state) on the host."""
    import torch

    from paper_1302_0120_gb300 import _binding as B

    assert B.gs_loss_prepare(h, I.data_ptr()) == 0
    ph = phi0.clone()
    m, v = torch.zeros_like(ph), torch.zeros_like(ph)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    rec = torch.zeros(steps + 1, dtype=torch.float64, device="cuda")
    for k in range(steps):
        assert B.gs_loss_adam_prepared(h, ph.data_ptr(), m.data_ptr(), v.data_ptr(), st.data_ptr(),
                                       0.05, 0.9, 0.999, 1e-8, rec[k:].data_ptr()) == 0
    assert B.gs_loss_grad_prepared(h, ph.data_ptr(), rec[steps:].data_ptr(), 0) == 0
    assert B.gs_status(h) == 0
    return rec.cpu().numpy(), ph, m, v, st.tolist()


@pytest.mark.parametrize("n,steps", [(256, 1), (256, 2), (256, 40), (1024, 12)])
def test_fused_run_matches_single_launches(n, steps):
    """optimize_phase (gs_loss_adam_run: all steps in one launch, each step's
    gradient pass forming the next step's row transforms) against the same
    steps as single gs_loss_adam_prepared launches: bit-identical losses and
    phase."""
    import torch

    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300.differentiable import LossContext, optimize_phase

    I = torch.from_numpy(normalized_target(27, n, 30)).cuda()
    phi0 = torch.from_numpy(S.random_phase(28, n, n)).cuda()
    lc = LossContext(n, stream=torch.cuda.Stream())
    ph_f, loss_f = optimize_phase(I, phi0, steps=steps, lr=0.05, lctx=lc)
    assert lc.status() == 0
    h = B.gs_create(n, n)
    try:
        rec, ph, _, _, st = single_launch_steps(h, I, phi0, steps, n)
        assert st == [steps, 0]
        assert np.array_equal(loss_f, rec)
        assert torch.equal(ph_f, ph)
    finally:
        B.gs_destroy(h)
        lc.close()


def test_adam_run_splits_long_runs():
    """gs_loss_adam_run over more steps than one launch takes (1024): the
    same losses, phase, moments and step count as single launches, bit for
    bit; a second run continues from the state the first left."""
    import torch

    from paper_1302_0120_gb300 import _binding as B

    n, steps = 64, 1030
    I = torch.from_numpy(normalized_target(29, n, 6)).cuda()
    phi0 = torch.from_numpy(S.random_phase(30, n, n)).cuda()
    h1, h2 = B.gs_create(n, n), B.gs_create(n, n)
    try:
        rec, ph, m, v, st = single_launch_steps(h1, I, phi0, steps, n)
        assert B.gs_loss_prepare(h2, I.data_ptr()) == 0
        ph2 = phi0.clone()
        m2, v2 = torch.zeros_like(ph2), torch.zeros_like(ph2)
        st2 = torch.zeros(2, dtype=torch.int32, device="cuda")
        rec2 = torch.zeros(steps + 1, dtype=torch.float64, device="cuda")
        args = (ph2.data_ptr(), m2.data_ptr(), v2.data_ptr(), st2.data_ptr(), 0.05, 0.9, 0.999, 1e-8)
        assert B.gs_loss_adam_run(h2, *args, 1000, rec2.data_ptr()) == 0
        assert B.gs_loss_adam_run(h2, *args, 30, rec2[1000:].data_ptr()) == 0
        assert B.gs_loss_grad_prepared(h2, ph2.data_ptr(), rec2[steps:].data_ptr(), 0) == 0
        assert B.gs_status(h2) == 0
        assert st2.tolist() == st == [steps, 0]
        assert np.array_equal(rec2.cpu().numpy(), rec)
        assert torch.equal(ph2, ph) and torch.equal(m2, m) and torch.equal(v2, v)
        assert rec[-1] < 0.5 * rec[0]
        # the same steps as one call, split by the library into two launches
        ph3, m3, v3 = phi0.clone(), torch.zeros_like(ph2), torch.zeros_like(ph2)
        st3 = torch.zeros(2, dtype=torch.int32, device="cuda")
        rec3 = torch.zeros(steps, dtype=torch.float64, device="cuda")
        assert B.gs_loss_adam_run(h2, ph3.data_ptr(), m3.data_ptr(), v3.data_ptr(), st3.data_ptr(), 0.05, 0.9, 0.999,
                                  1e-8, steps, rec3.data_ptr()) == 0
        assert B.gs_status(h2) == 0
        assert st3.tolist() == [steps, 0]
        assert np.array_equal(rec3.cpu().numpy(), rec[:steps]) and torch.equal(ph3, ph)
        # arguments the call refuses
        assert B.gs_loss_adam_run(h2, *args, 0, rec2.data_ptr()) == B.GS_EINVAL
        assert B.gs_loss_adam_run(h2, *args, 3, 0) == B.GS_EINVAL
    finally:
        B.gs_destroy(h1)
        B.gs_destroy(h2)


def test_adam_run_nonfinite_target():
    """A staged target with a NaN: every loss of the run is NaN, the phase,
    moments and step count are left as they were, and the status says so."""
    import torch

    from paper_1302_0120_gb300 import _binding as B

    n = 64
    I = normalized_target(31, n, 6)
    I[3, 9] = np.nan
    It = torch.from_numpy(I).cuda()
    phi0 = torch.from_numpy(S.random_phase(32, n, n)).cuda()
    h = B.gs_create(n, n)
    try:
        assert B.gs_loss_prepare(h, It.data_ptr()) == 0
        ph = phi0.clone()
        m, v = torch.zeros_like(ph), torch.zeros_like(ph)
        st = torch.tensor([5, 0], dtype=torch.int32, device="cuda")
        rec = torch.zeros(7, dtype=torch.float64, device="cuda")
        assert B.gs_loss_adam_run(h, ph.data_ptr(), m.data_ptr(), v.data_ptr(), st.data_ptr(), 0.05, 0.9, 0.999,
                                  1e-8, 7, rec.data_ptr()) == 0
        assert B.gs_status(h) == B.GS_ENUMERIC
        assert np.all(np.isnan(rec.cpu().numpy()))
        assert torch.equal(ph, phi0) and not m.any() and not v.any() and st.tolist() == [5, 0]
    finally:
        B.gs_destroy(h)


def test_fused_adam_matches_eager():
    """The library's fused steps (its own Adam) follow the eager autograd
    path with torch's Adam: same losses to 1e-2 over 30 steps, and the loss
    falls."""
    import torch

    from paper_1302_0120_gb300.differentiable import LossContext, optimize_phase

    n = 256
    I = torch.from_numpy(normalized_target(7, n, 30)).cuda()
    phi0 = torch.from_numpy(S.random_phase(8, n, n)).cuda()
    lc_g = LossContext(n, stream=torch.cuda.Stream())
    ph_g, loss_g = optimize_phase(I, phi0, steps=30, lr=0.05, lctx=lc_g)
    lc_e = LossContext(n)
    ph_e, loss_e = optimize_phase(I, phi0, steps=30, lr=0.05, lctx=lc_e, fused=False)
    assert lc_g.status() == 0 and lc_e.status() == 0
    assert loss_g.shape == loss_e.shape == (31,)
    assert np.allclose(loss_g, loss_e, rtol=1e-2, atol=0), np.max(np.abs(loss_g / loss_e - 1))
    assert loss_g[-1] < 0.7 * loss_g[0]
    lc_g.close()
    lc_e.close()


def test_side_stream_eager_steps_match_current_stream():
    """The eager path on a context with its own stream, while torch's Adam
    writes the phase on the current stream: the two are ordered, so the
    result equals an eager run whose context uses the current stream. The
    fused path on a side stream equals the fused path on the current one. A
    user-built context on a side stream gives the same loss as one on the
    current stream."""
    import torch

    from paper_1302_0120_gb300.differentiable import LossContext, intensity_loss, optimize_phase

    n = 256
    I = torch.from_numpy(normalized_target(17, n, 30)).cuda()
    phi0 = torch.from_numpy(S.random_phase(18, n, n)).cuda()
    lc_s = LossContext(n, stream=torch.cuda.Stream())
    ph_side, loss_side = optimize_phase(I, phi0, steps=3, lr=0.05, lctx=lc_s, fused=False)
    lc_cur = LossContext(n)
    ph_cur, loss_cur = optimize_phase(I, phi0, steps=3, lr=0.05, lctx=lc_cur, fused=False)
    assert lc_cur.status() == 0 and lc_s.status() == 0
    assert np.array_equal(loss_side, loss_cur)
    assert torch.equal(ph_side, ph_cur)
    ph_fs, loss_fs = optimize_phase(I, phi0, steps=5, lr=0.05, lctx=lc_s)
    ph_fc, loss_fc = optimize_phase(I, phi0, steps=5, lr=0.05)  # lctx None: the current stream
    assert lc_s.status() == 0
    assert np.array_equal(loss_fs, loss_fc) and torch.equal(ph_fs, ph_fc)
    lc_s.close()
    lc_side = LossContext(n, stream=torch.cuda.Stream())
    for _ in range(3):
        phi = phi0 * 1.01  # written on the current stream just before the call
        a = intensity_loss(phi, I, lc_side)
        b = intensity_loss(phi, I, lc_cur)
        assert float(a) == float(b)
    assert lc_side.status() == 0
    lc_side.close()
    lc_cur.close()


def gpu_physical_error(I, phi, p=None):
    import torch

    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300 import build_lib
    from paper_1302_0120_gb300.differentiable import LossContext

    build_lib.build()
    lc = LossContext(I.shape[0])
    pt = None
    if p is not None:
        pt = torch.from_numpy(p).cuda()
        assert B.gs_set_slm_amplitude(lc.handle, pt.data_ptr()) == 0
    e = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    It, Pt = torch.from_numpy(I).cuda(), torch.from_numpy(phi).cuda()
    assert B.gs_physical_error(lc.handle, It.data_ptr(), Pt.data_ptr(), e.data_ptr()) == 0
    st = lc.status()
    out = e.cpu().numpy()
    lc.close()
    return out, st


@pytest.mark.parametrize("n,iters", [(64, 20), (256, 30), (1024, 20)])
def test_physical_error_of_gs_masks(n, iters):
    """E (Eq. phys-error) of a GPU Gerchberg-Saxton mask, against the oracle's
    E of the same mask; E is continuous in the field, so FP32 stays close."""
    from tests.gpu_util import gpu_gs

    I = S.spot_target(50 + n, n, n, 10 if n == 64 else 40, (0.5, 1.0))
    ph, _, _, st = gpu_gs(I, S.random_phase(51 + n, n, n), iters)
    assert st == 0
    e, st = gpu_physical_error(I, ph)
    assert st == 0
    ref = O.physical_error(I, np.exp(1j * ph.astype(np.float64)))
    assert ref[0] > 0 and ref[1] > 0
    assert np.allclose(e, ref, rtol=2e-3, atol=0), (e, ref)


def test_physical_error_consistent_target_is_zero():
    n = 64
    rng = np.random.default_rng(8)
    phi = (rng.random((n, n)) * 2 * np.pi).astype(np.float32)
    I = O.consistent_target(phi).astype(np.float32)  # no dark pixel, exact reconstruction
    e, st = gpu_physical_error(I, phi)
    assert st == 0 and e[0] == 0.0 and e[1] == 0.0


def test_loss_and_physical_error_with_laser_amplitude():
    import torch

    from paper_1302_0120_gb300 import _binding as B
    from paper_1302_0120_gb300.differentiable import LossContext

    n = 128
    I = normalized_target(60, n, 10)
    phi = S.random_phase(61, n, n)
    p = S.laser_amplitude(n, n)
    lc = LossContext(n)
    pt = torch.from_numpy(p).cuda()
    assert B.gs_set_slm_amplitude(lc.handle, pt.data_ptr()) == 0
    loss, grad = lc.loss_grad(torch.from_numpy(I).cuda(), torch.from_numpy(phi).cuda())
    assert lc.status() == 0
    ref_l = O.intensity_loss(phi, I, p)
    ref_g = O.intensity_loss_grad(phi, I, p)
    assert abs(loss.item() - ref_l) <= 1e-4 * ref_l
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g) <= 1e-3
    lc.close()
    e, st = gpu_physical_error(I, phi, p)
    ref = O.physical_error(I, p.astype(np.float64) * np.exp(1j * phi.astype(np.float64)))
    assert st == 0 and np.allclose(e, ref, rtol=2e-3, atol=0), (e, ref)


def test_nonfinite_target():
    from paper_1302_0120_gb300 import GS_ENUMERIC

    I = normalized_target(1, 64, 4)
    I[3, 3] = np.inf
    loss, grad, st = gpu_loss_grad(I, S.random_phase(2, 64, 64))
    assert st == GS_ENUMERIC and np.isnan(loss)
