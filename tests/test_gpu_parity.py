"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the field is FP32, the oracle FP64.
  * one step u^nu -> u^{nu+1} from the same start: relative L2 <= 1e-5
    (after removing a global phase, to which the iteration is equivariant);
  * the normalised residuals r^nu, g^nu: relative error <= 1e-3, and the final
    r^K within 0.1% of the oracle's;
  * the chain r^nu >= g^nu >= r^{nu+1} holds on the GPU's FP64-reduced gaps to
    a slack of 1e-6 (FP32 rounding of the field).
Sizes span several blocks and ragged shares (grids that do not divide the
number of rows or columns), non-square grids and the size limits.
"""

import numpy as np
import pytest

import oracle.gs_oracle as O
from paper_1302_0120_gb300 import synthetic as S
from tests.gpu_util import aligned_rel_err, gpu_gs

pytestmark = pytest.mark.gpu

ONE_STEP_TOL = 1e-5
RES_TOL = 1e-3


def check_run(I, phi0, iters, grid=None, one_step_at=(0,), final_resid_tol=1e-3):
    ph, r, g, st = gpu_gs(I, phi0, iters, grid=grid)
    assert st == 0
    ref = O.gs_run(I, phi0, iters)
    assert r.shape == ref["r"].shape and g.shape == ref["g"].shape
    rel_r = np.abs(r - ref["r"]) / ref["r"]
    rel_g = np.abs(g - ref["g"]) / ref["g"]
    assert np.max(rel_r) <= RES_TOL, (np.argmax(rel_r), np.max(rel_r))
    if iters:
        assert np.max(rel_g) <= RES_TOL, (np.argmax(rel_g), np.max(rel_g))
    assert abs(r[-1] - ref["r"][-1]) <= final_resid_tol * ref["r"][-1]
    assert np.all(r[:-1] - g >= -1e-6) and np.all(g - r[1:] >= -1e-6)
    m = O.target_amplitude(I)
    for nu in one_step_at:
        if nu >= iters:
            continue
        start = phi0 if nu == 0 else gpu_gs(I, phi0, nu, grid=grid)[0]
        nxt, _, _, st = gpu_gs(I, start, 1, grid=grid)
        assert st == 0
        u_ref, _, _ = O.gs_step(np.exp(1j * start.astype(np.float64)), m)
        err = aligned_rel_err(nxt, u_ref)
        assert err <= ONE_STEP_TOL, (nu, err)
    return ph, r, g, ref


def test_spots64_20_iterations():
    I, phi0, iters = S.workload("spots64")
    ph, r, g, ref = check_run(I, phi0, iters, one_step_at=range(iters))
    # trajectory from the same start, global phase removed
    err = aligned_rel_err(ph, ref["u"])
    assert err <= 1e-4, err


@pytest.mark.parametrize("grid", [1, 3, 7, 64])
def test_spots64_grids(grid):
    I, phi0, _ = S.workload("spots64")
    check_run(I, phi0, 6, grid=grid, one_step_at=(0, 5))


def test_spots512_100_iterations():
    I, phi0, iters = S.workload("spots512")
    check_run(I, phi0, iters, one_step_at=(0, 1, 50, 99))


def test_spots1024_100_iterations():
    I, phi0, iters = S.workload("spots1024")
    check_run(I, phi0, iters, one_step_at=(0, 1, 10, 50, 99))


@pytest.mark.parametrize("grid", [5, 100, 151])
def test_spots1024_ragged_grids(grid):
    I, phi0, _ = S.workload("spots1024")
    check_run(I, phi0, 3, grid=grid, one_step_at=(0,))


@pytest.mark.parametrize("ny,nx", [(64, 256), (256, 64), (512, 1024), (1024, 512), (32, 4096), (4096, 32), (32, 32)])
def test_nonsquare_and_extreme_shapes(ny, nx):
    I = S.spot_target(7, ny, nx, 12, (0.5, 1.0))
    phi0 = S.random_phase(7, ny, nx)
    check_run(I, phi0, 5, one_step_at=(0, 4))


@pytest.mark.parametrize("n", [128, 256, 2048])
def test_other_square_sizes(n):
    I = S.spot_target(8, n, n, 20, (0.5, 1.0))
    phi0 = S.random_phase(8, n, n)
    check_run(I, phi0, 4, one_step_at=(0,))


def test_max_size_4096():
    I = S.spot_target(9, 4096, 4096, 100, (0.5, 1.0))
    phi0 = S.random_phase(9, 4096, 4096)
    check_run(I, phi0, 2, one_step_at=(0,))


def test_chunked_run_crosses_launches():
    # more iterations than one persistent launch holds (128)
    I, phi0, _ = S.workload("spots64")
    check_run(I, phi0, 130, grid=4, one_step_at=())


@pytest.mark.parametrize("n", [512, 1024])
def test_consistent_target_fixed_point(n):
    rng = np.random.default_rng(3)
    phi_t = (rng.random((n, n)) * 2 * np.pi).astype(np.float32)
    I = O.consistent_target(phi_t).astype(np.float32)
    ph, r, g, st = gpu_gs(I, phi_t, 3)
    assert st == 0
    # FP32 floor: the gap of an exact solution stays at the rounding level
    assert r[0] < 1e-5 and np.all(r < 1e-5) and np.all(g < 1e-5)
    assert aligned_rel_err(ph, np.exp(1j * phi_t.astype(np.float64))) < 1e-5


@pytest.mark.parametrize("n", [512, 1024])
def test_consistent_target_local_convergence(n):
    rng = np.random.default_rng(4)
    phi_t = (rng.random((n, n)) * 2 * np.pi).astype(np.float32)
    I = O.consistent_target(phi_t).astype(np.float32)
    start = (phi_t + 0.1 * rng.standard_normal(phi_t.shape)).astype(np.float32)
    ph, r, g, ref = check_run(I, start, 30, one_step_at=(0, 29))
    assert r[-1] < 0.2 * r[0]


@pytest.mark.parametrize("ny,nx,iters", [(512, 512, 100), (600, 800, 25)])
def test_siemens_star(ny, nx, iters):
    """The paper's second target (Sec. IV, the Siemens star of its precision
    comparison): half the disc dark (m = 0 on whole sectors), the rest of the
    grid dark too. The FP32 path keeps every gate of the spot targets, and its
    final residual lands within 0.1% of the FP64 oracle's limit value (Sec.
    IV.B: single and double precision reach the same limits)."""
    I = S.siemens_star(ny, nx)
    phi0 = S.random_phase(31 + nx, ny, nx)
    ph, r, g, ref = check_run(I, phi0, iters, one_step_at=(0, iters - 1))
    print(f"siemens star {ny}x{nx}, {iters} iterations: r^K FP32 GPU {r[-1]:.7f}, FP64 oracle {ref['r'][-1]:.7f}, "
          f"relative difference {abs(r[-1] - ref['r'][-1]) / ref['r'][-1]:.2e}")


def test_zero_iterations():
    I, phi0, _ = S.workload("spots64")
    ph, r, g, st = gpu_gs(I, phi0, 0)
    assert st == 0 and r.shape == (1,) and g.shape == (0,)
    ref = O.gs_run(I, phi0, 0)
    assert abs(r[0] - ref["r"][0]) <= 1e-4 * ref["r"][0]
    assert np.max(np.abs(np.exp(1j * ph.astype(np.float64)) - np.exp(1j * phi0.astype(np.float64)))) < 1e-6
    assert np.all(ph > -np.pi - 1e-6) and np.all(ph <= np.pi + 1e-6)


def test_warm_start_aliasing_and_resume():
    """phase_in may alias phase_out; 5 + 5 iterations from the saved mask
    match 10 iterations (up to re-exponentiating the stored phase)."""
    I, phi0, _ = S.workload("spots64")
    ph10, r10, _, _ = gpu_gs(I, phi0, 10)
    ph5, _, _, _ = gpu_gs(I, phi0, 5)
    ph55, r55, _, st = gpu_gs(I, ph5.copy(), 5, aliased=True)
    assert st == 0
    assert aligned_rel_err(ph55, np.exp(1j * ph10.astype(np.float64))) < 1e-4
    assert abs(r55[-1] - r10[-1]) <= 1e-4 * r10[-1]


def test_no_final_residual_and_null_outputs():
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton

    I, phi0, _ = S.workload("spots64")
    ref = O.gs_run(I, phi0, 4)
    with GerchbergSaxton(64, 64, final_residual=False) as gs:
        It, Pt = torch.from_numpy(I).cuda(), torch.from_numpy(phi0).cuda()
        ph, r, g = gs.run(It, Pt, 4)
        assert gs.status() == 0
        assert r.shape == (4,)
        assert np.allclose(r.cpu().numpy(), ref["r"][:4], rtol=1e-3)
        ph2, r2, g2 = gs.run(It, Pt, 4, residuals=False, object_gap=False)
        assert gs.status() == 0 and r2 is None and g2 is None
        assert torch.equal(ph, ph2)


def test_deterministic():
    I, phi0, iters = S.workload("spots512")
    a = gpu_gs(I, phi0, 10)
    b = gpu_gs(I, phi0, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("bad", ["nan", "neg", "zero", "inf"])
def test_bad_target_reports_enumeric(bad):
    import torch

    from paper_1302_0120_gb300 import GS_ENUMERIC, GerchbergSaxton

    I, phi0, _ = S.workload("spots64")
    I = I.copy()
    if bad == "nan":
        I[3, 5] = np.nan
    elif bad == "neg":
        I[1, 1] = -1.0
    elif bad == "inf":
        I[2, 2] = np.inf
    else:
        I[:] = 0
    with GerchbergSaxton(64, 64) as gs:
        It, Pt = torch.from_numpy(I).cuda(), torch.from_numpy(phi0).cuda()
        sentinel = torch.full_like(Pt, 7.0)
        ph, r, g = gs.run(It, Pt, 3, phase_out=sentinel)
        assert gs.status() == GS_ENUMERIC
        assert torch.all(ph == 7.0)
        assert torch.all(torch.isnan(r)) and torch.all(torch.isnan(g))
        # the context stays usable
        I2, _, _ = S.workload("spots64")
        ph, r, g = gs.run(torch.from_numpy(I2).cuda(), Pt, 3)
        assert gs.status() == 0 and torch.all(torch.isfinite(r))


def test_run_host_matches_device_run():
    from paper_1302_0120_gb300 import GerchbergSaxton

    I, phi0, _ = S.workload("spots512")
    dev = gpu_gs(I, phi0, 5)
    with GerchbergSaxton(512, 512) as gs:
        ph, r, g = gs.run_host(I, phi0, 5)
    assert np.array_equal(ph, dev[0]) and np.array_equal(r, dev[1]) and np.array_equal(g, dev[2])


@pytest.mark.parametrize("iters", [0, 5, 130])
def test_run_host_pinned_buffers(iters):
    """Pinned host buffers (the asynchronous-copy path of the bench's e2e
    figure): the results are those of a device run, call after call,
    including zero iterations and a run of two launches."""
    import torch

    from paper_1302_0120_gb300 import GerchbergSaxton
    from paper_1302_0120_gb300 import _binding as B

    I, phi0, _ = S.workload("spots512")
    dev = gpu_gs(I, phi0, iters)
    pI = torch.from_numpy(I).pin_memory()
    pP = torch.from_numpy(phi0).pin_memory()
    pO = torch.full_like(pP, 7.0).pin_memory()
    r = np.empty(iters + 1)
    g = np.empty(max(iters, 1))
    with GerchbergSaxton(512, 512) as gs:
        for _ in range(2):
            rc = B.gs_run_host(gs.handle, pI.data_ptr(), pP.data_ptr(), iters, pO.data_ptr(), r.ctypes.data,
                               g.ctypes.data)
            assert rc == 0
            assert np.array_equal(pO.numpy(), dev[0]) and np.array_equal(r, dev[1])
            if iters:
                assert np.array_equal(g[:iters], dev[2])
            pO.fill_(7.0)


def test_run_host_growing_runs_and_status():
    """One context, runs of growing and shrinking length (the staging of the
    gaps grows with them), then an invalid target: the status comes back as
    the return value and is cleared for the next call."""
    from paper_1302_0120_gb300 import GS_ENUMERIC, GerchbergSaxton
    from paper_1302_0120_gb300 import _binding as B

    I, phi0, _ = S.workload("spots64")
    with GerchbergSaxton(64, 64) as gs:
        for iters in (3, 140, 0, 7):
            dev = gpu_gs(I, phi0, iters)
            r = np.empty(iters + 1)
            g = np.empty(max(iters, 1))
            out = np.empty_like(phi0)
            rc = B.gs_run_host(gs.handle, I.ctypes.data, phi0.ctypes.data, iters, out.ctypes.data, r.ctypes.data,
                               g.ctypes.data)
            assert rc == 0
            assert np.array_equal(out, dev[0]) and np.array_equal(r, dev[1])
            if iters:
                assert np.array_equal(g[:iters], dev[2])
        bad = I.copy()
        bad[3, 5] = -1.0
        r = np.empty(6)
        out = np.empty_like(phi0)
        assert B.gs_run_host(gs.handle, bad.ctypes.data, phi0.ctypes.data, 5, out.ctypes.data, r.ctypes.data,
                             0) == GS_ENUMERIC
        assert np.all(np.isnan(r))
        rc = B.gs_run_host(gs.handle, I.ctypes.data, phi0.ctypes.data, 5, out.ctypes.data, r.ctypes.data, 0)
        assert rc == 0 and np.all(np.isfinite(r))
