"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these checks re-uses the oracle's own formula: the FFT is compared
with a direct DFT sum, the projections with their defining nearest-point
property (Sec. II: "the set of nearest points"), the iteration with the
interleaved gap chain that alternating projections must satisfy, consistent
problems with their known fixed point, and the gradient with finite
differences. tests/test_oracle_mutations.py plants mistakes in the oracle and
checks that these pins fail.
"""

import numpy as np
import pytest

import oracle.gs_oracle as O
from paper_1302_0120_gb300 import synthetic as S


def direct_dft2(x):
    """Unnormalised 2D DFT by direct summation over both axes."""
    ny, nx = x.shape
    out = np.zeros((ny, nx), dtype=np.complex128)
    ky = np.arange(ny)
    kx = np.arange(nx)
    for k2 in range(ny):
        ey = np.exp(-2j * np.pi * np.outer(ky, np.full(1, k2)) / ny)[:, 0]
        for k1 in range(nx):
            ex = np.exp(-2j * np.pi * kx * k1 / nx)
            out[k2, k1] = np.sum(x * ey[:, None] * ex[None, :])
    return out


def rand_complex(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- FFT step


def check_fft_direct(shape, seed=0):
    rng = np.random.default_rng(seed)
    x = rand_complex(rng, shape)
    ref = direct_dft2(x) / np.sqrt(x.size)
    got = O.fft2u(x)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, err
    back = O.ifft2u(ref)
    err2 = np.linalg.norm(back - x) / np.linalg.norm(x)
    assert err2 <= 1e-12, err2


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (32, 32), (8, 32), (32, 8), (6, 10), (15, 12), (24, 20), (45, 8),
                                   (72, 80), (96, 67)])
def test_fft_matches_direct_dft(shape):
    check_fft_direct(shape)


def direct_dft1(x):
    """Unnormalised DFT along the last axis by the defining sum, one output
    frequency at a time (angles reduced exactly in integers)."""
    n = x.shape[-1]
    j = np.arange(n)
    out = np.empty(x.shape, dtype=np.complex128)
    for k in range(n):
        a = 2 * np.pi * ((j * k) % n) / n
        out[..., k] = np.sum(x * (np.cos(a) - 1j * np.sin(a)), axis=-1)
    return out


def check_fft_long(n, seed=2):
    """Lengths above the direct-sum limit, which the oracle's FFT computes by
    the Cooley-Tukey factorisation (powers of two, 5-smooth SLM sides of
    Sec. V, a prime factor): against the defining sum."""
    from oracle import dft as D

    rng = np.random.default_rng(seed + n)
    x = rand_complex(rng, (2, n))
    ref = direct_dft1(x)
    err = np.linalg.norm(D.dft_last(x) - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, (n, err)
    back = D.idft_last(ref) / n
    assert np.linalg.norm(back - x) / np.linalg.norm(x) <= 1e-12


@pytest.mark.parametrize("n", [96, 128, 134, 600, 800, 1024, 1536, 4096])
def test_fft_long_lengths_match_direct_dft(n):
    check_fft_long(n)


def check_fft_identities(ny=32, nx=16, seed=1):
    rng = np.random.default_rng(seed)
    x = rand_complex(rng, (ny, nx))
    # Parseval (unitary transform)
    assert abs(np.linalg.norm(O.fft2u(x)) - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)
    # inverse
    assert np.allclose(O.ifft2u(O.fft2u(x)), x, rtol=0, atol=1e-12)
    # delta at the origin -> constant 1/sqrt(N)
    d = np.zeros((ny, nx), complex)
    d[0, 0] = 1.0
    assert np.allclose(O.fft2u(d), 1.0 / np.sqrt(ny * nx), rtol=0, atol=1e-14)
    # constant -> delta at DC with weight sqrt(N)
    c = np.ones((ny, nx), complex)
    Fc = O.fft2u(c)
    want = np.zeros((ny, nx), complex)
    want[0, 0] = np.sqrt(ny * nx)
    assert np.allclose(Fc, want, rtol=0, atol=1e-12)
    # shift -> linear phase (sign convention exp(-2 pi i ...))
    sy, sx = 3, 5
    xs = np.roll(x, (sy, sx), axis=(0, 1))
    k2 = np.arange(ny)[:, None]
    k1 = np.arange(nx)[None, :]
    ramp = np.exp(-2j * np.pi * (sx * k1 / nx + sy * k2 / ny))
    assert np.allclose(O.fft2u(xs), O.fft2u(x) * ramp, rtol=0, atol=1e-12)


def test_fft_identities():
    check_fft_identities()


# ---------------------------------------------------------------- target amplitude


def check_target_amplitude():
    I = S.spot_target(2, 32, 32, 4, (0.5, 1.0)).astype(np.float64)
    m = O.target_amplitude(I)
    assert abs(np.sum(m * m) - I.size) <= 1e-10 * I.size
    lit = I > 0
    ratio = m[lit] / np.sqrt(I[lit])
    assert np.ptp(ratio) <= 1e-12 * ratio.mean()
    assert np.all(m[~lit] == 0)
    assert np.allclose(O.target_amplitude(7.25 * I), m, rtol=1e-13, atol=0)


def test_target_amplitude():
    check_target_amplitude()


@pytest.mark.parametrize("bad", ["nan", "inf", "neg", "zero"])
def test_target_amplitude_rejects(bad):
    I = np.ones((8, 8))
    if bad == "nan":
        I[1, 2] = np.nan
    elif bad == "inf":
        I[0, 0] = np.inf
    elif bad == "neg":
        I[3, 3] = -1e-3
    else:
        I[:] = 0
    with pytest.raises(ValueError):
        O.target_amplitude(I)


# ---------------------------------------------------------------- projections


def check_proj_S(seed=3):
    rng = np.random.default_rng(seed)
    u = rand_complex(rng, (16, 8))
    p = rng.uniform(0.2, 2.0, size=u.shape)
    for pp in (None, p):
        pv = np.ones(u.shape) if pp is None else pp
        v = O.proj_S(u, pp)
        assert np.allclose(np.abs(v), pv, rtol=0, atol=1e-14)
        assert np.allclose(O.proj_S(v, pp), v, rtol=0, atol=1e-14)
        d0 = np.linalg.norm(u - v)
        for _ in range(200):  # no other point of S is closer (nearest point)
            y = pv * np.exp(2j * np.pi * rng.random(u.shape))
            assert d0 <= np.linalg.norm(u - y) + 1e-12
        for eps in (1e-3, -1e-3):  # nor any small rotation of the answer
            y = v * np.exp(1j * eps * rng.standard_normal(u.shape))
            assert d0 <= np.linalg.norm(u - y) + 1e-12
    # zero rule: arbitrary phase, theta = 0 chosen
    z = np.zeros((4, 4), complex)
    assert np.allclose(O.proj_S(z), 1.0)


def test_proj_S():
    check_proj_S()


def check_proj_M(seed=4):
    rng = np.random.default_rng(seed)
    I = S.spot_target(5, 16, 16, 3)
    m = O.target_amplitude(I)
    u = np.exp(2j * np.pi * rng.random((16, 16)))
    v = O.proj_M(u, m)
    assert np.allclose(np.abs(O.fft2u(v)), m, rtol=0, atol=1e-12)  # v in M
    assert np.allclose(O.proj_M(v, m), v, rtol=0, atol=1e-12)  # idempotent
    d0 = np.linalg.norm(u - v)
    for _ in range(200):  # nearest point of M (computed in the object domain)
        y = O.ifft2u(m * np.exp(2j * np.pi * rng.random(m.shape)))
        assert d0 <= np.linalg.norm(u - y) + 1e-12
    Fv = O.fft2u(v)
    for eps in (1e-3, -1e-3):
        y = O.ifft2u(Fv * np.exp(1j * eps * rng.standard_normal(m.shape)))
        assert d0 <= np.linalg.norm(u - y) + 1e-12
    # zero rule of Eq. (e:Mhat): where F u vanishes any phase is allowed; the
    # selection must still have amplitude m there (reading C1: phase 0). Exact
    # zeros are planted in the Fourier data: a transform of rounded inputs
    # leaves residues of order 1e-16 instead of exact zeros.
    Fz = rand_complex(rng, (8, 8))
    Fz[0, 1] = 0.0
    Fz[3, 5] = 0.0
    mm = rng.uniform(0.5, 2.0, (8, 8))
    sel = O._mhat(Fz, mm)
    assert np.allclose(np.abs(sel), mm, rtol=0, atol=1e-14)
    assert sel[0, 1] == mm[0, 1] and sel[3, 5] == mm[3, 5]


def test_proj_M():
    check_proj_M()


def check_gap_definitions(seed=6):
    rng = np.random.default_rng(seed)
    I = S.spot_target(6, 16, 32, 4, (0.5, 1.0))
    m = O.target_amplitude(I)
    u = np.exp(2j * np.pi * rng.random(m.shape))
    n = u.size
    # distance to M computed in the object domain, not through Parseval
    r_direct = np.linalg.norm(u - O.proj_M(u, m)) / np.sqrt(n)
    assert abs(O.gap_to_M(u, m) - r_direct) <= 1e-12
    v = O.proj_M(u, m)
    g_direct = np.linalg.norm(v - O.proj_S(v)) / np.sqrt(n)
    assert abs(O.gap_to_S(v) - g_direct) <= 1e-12
    u1, r, g = O.gs_step(u, m)
    assert abs(r - r_direct) <= 1e-12 and abs(g - g_direct) <= 1e-12
    assert np.allclose(u1, O.proj_S(O.proj_M(u, m)), rtol=0, atol=1e-14)


def test_gap_definitions():
    check_gap_definitions()


# ---------------------------------------------------------------- the iteration


def check_gap_chain(name="spots64", iters=30):
    """Alternating projections: r^nu >= g^nu >= r^{nu+1} (each step maps to a
    nearest point of a set that contains the previous iterate)."""
    I, phi0, _ = S.workload(name)
    res = O.gs_run(I, phi0, iters)
    r, g = res["r"], res["g"]
    assert len(r) == iters + 1 and len(g) == iters
    assert np.all(r[:-1] - g >= -1e-12), np.min(r[:-1] - g)
    assert np.all(g - r[1:] >= -1e-12), np.min(g - r[1:])
    assert r[-1] < r[0]


def test_gap_chain():
    check_gap_chain()


def test_gap_chain_nonsquare():
    I = S.spot_target(9, 32, 64, 6, (0.5, 1.0))
    phi0 = S.random_phase(9, 32, 64)
    res = O.gs_run(I, phi0, 25)
    r, g = res["r"], res["g"]
    assert np.all(r[:-1] - g >= -1e-12) and np.all(g - r[1:] >= -1e-12)


def test_gap_chain_not_power_of_two():
    """The 800 x 600 grid of Sec. V, scaled down to 40 x 30 (5-smooth sides)."""
    I = S.spot_target(10, 30, 40, 5, (0.5, 1.0))
    phi0 = S.random_phase(10, 30, 40)
    res = O.gs_run(I, phi0, 25)
    r, g = res["r"], res["g"]
    assert np.all(r[:-1] - g >= -1e-12) and np.all(g - r[1:] >= -1e-12) and r[-1] < r[0]


def test_consistent_fixed_point_not_power_of_two():
    check_consistent_fixed_point(shape=(30, 40))


def check_consistent_fixed_point(n=32, seed=1, shape=None):
    rng = np.random.default_rng(seed)
    phi_t = (rng.random(shape or (n, n)) * 2 * np.pi).astype(np.float32)
    I = O.consistent_target(phi_t)  # FP64, exact
    res = O.gs_run(I, phi_t, 1)
    assert res["r"][0] <= 1e-12 and res["r"][1] <= 1e-12 and res["g"][0] <= 1e-12
    u_t = np.exp(1j * phi_t.astype(np.float64))
    assert np.max(np.abs(res["u"] - u_t)) <= 1e-12


def test_consistent_fixed_point():
    check_consistent_fixed_point()


def test_consistent_local_convergence():
    """Near a solution of a consistent problem the gap falls towards zero
    (local convergence of alternating projections, Sec. II)."""
    rng = np.random.default_rng(1)
    phi_t = (rng.random((32, 32)) * 2 * np.pi).astype(np.float32)
    I = O.consistent_target(phi_t)
    start = (phi_t + 0.1 * rng.standard_normal(phi_t.shape)).astype(np.float32)
    res = O.gs_run(I, start, 300)
    r = res["r"]
    assert np.all(np.diff(r) <= 1e-14)
    assert r[-1] < 1e-2 * r[0]


def check_scale_invariance(seed=2):
    """Only phases survive P_S and P_M: rescaling m leaves every iterate unchanged."""
    I, phi0, _ = S.workload("spots64", seed)
    m = O.target_amplitude(I)
    u = np.exp(1j * phi0.astype(np.float64))
    a, _, _ = O.gs_step(u, m)
    b, _, _ = O.gs_step(u, 3.5 * m)
    assert np.max(np.abs(a - b)) <= 1e-12
    # equivariance under a global phase
    c, _, _ = O.gs_step(np.exp(0.7j) * u, m)
    assert np.max(np.abs(c - np.exp(0.7j) * a)) <= 1e-12


def test_scale_and_phase_invariance():
    check_scale_invariance()


def test_zero_iterations():
    I, phi0, _ = S.workload("spots64")
    res = O.gs_run(I, phi0, 0)
    assert res["r"].shape == (1,) and res["g"].shape == (0,)
    assert np.allclose(np.exp(1j * res["phase"]), np.exp(1j * phi0.astype(np.float64)), atol=1e-14)


def test_phase_range():
    I, phi0, _ = S.workload("spots64")
    ph = O.gs_run(I, phi0, 3)["phase"]
    assert np.all(ph > -np.pi) and np.all(ph <= np.pi)


# ---------------------------------------------------------------- SLM amplitude p and the target start


def laser_profile(ny, nx, seed=0):
    """A Gaussian beam on the SLM with a little seeded ripple, float32, > 0."""
    y = (np.arange(ny) - ny / 2)[:, None] / (0.45 * ny)
    x = (np.arange(nx) - nx / 2)[None, :] / (0.45 * nx)
    rng = np.random.default_rng(seed)
    p = np.exp(-(x * x + y * y)) * (1 + 0.05 * rng.standard_normal((ny, nx)))
    return np.abs(p).astype(np.float32) + 0.01


def check_slm_amplitude_chain(ny=32, nx=64, iters=25):
    p = laser_profile(ny, nx)
    I = S.spot_target(12, ny, nx, 6, (0.5, 1.0))
    phi0 = S.random_phase(12, ny, nx)
    res = O.gs_run(I, phi0, iters, p=p)
    r, g = res["r"], res["g"]
    assert np.all(r[:-1] - g >= -1e-12) and np.all(g - r[1:] >= -1e-12)
    assert np.allclose(np.abs(res["u"]), p.astype(np.float64), rtol=0, atol=1e-12)  # u^K in S
    m = O.target_amplitude(I, energy=float(np.sum(p.astype(np.float64) ** 2)))
    assert abs(np.sum(m * m) - np.sum(p.astype(np.float64) ** 2)) <= 1e-9 * np.sum(m * m)
    # the residual is the object-domain distance to M divided by ||p||
    u = res["u"]
    direct = np.linalg.norm(u - O.proj_M(u, m)) / np.linalg.norm(p.astype(np.float64))
    assert abs(res["r"][-1] - direct) <= 1e-12


def test_slm_amplitude_chain():
    check_slm_amplitude_chain()


def test_slm_amplitude_consistent_fixed_point():
    n = 32
    p = laser_profile(n, n, 3)
    rng = np.random.default_rng(8)
    phi_t = (rng.random((n, n)) * 2 * np.pi).astype(np.float32)
    I = np.abs(O.fft2u(p.astype(np.float64) * np.exp(1j * phi_t.astype(np.float64)))) ** 2
    res = O.gs_run(I, phi_t, 1, p=p)
    assert res["r"][0] <= 1e-12 and res["g"][0] <= 1e-12 and res["r"][1] <= 1e-12


def test_slm_amplitude_scale_invariance():
    """Only phases survive the projections: scaling p leaves the phases."""
    p = laser_profile(32, 32, 5)
    I, phi0, _ = S.workload("spots64")
    I, phi0 = I[:32, :32].copy(), phi0[:32, :32].copy()
    I[3, 3] = 1.0
    a = O.gs_run(I, phi0, 5, p=p)
    b = O.gs_run(I, phi0, 5, p=(4.0 * p).astype(np.float32))  # exact in float32
    assert np.max(np.abs(np.exp(1j * a["phase"]) - np.exp(1j * b["phase"]))) <= 1e-9
    assert np.allclose(a["r"], b["r"], rtol=1e-12, atol=0)


def test_target_start_is_hermitian():
    """u0 = P_S(F^{-1} m) with real m is conjugate-symmetric, u0(-x) = conj(u0(x)),
    so F u stays real along the iteration (the binary-phase Fourier plane of
    this start, a consequence of the reading)."""
    I, phi0, _ = S.workload("spots64")
    res0 = O.gs_run(I, phi0, 0, init="target")
    u0 = res0["u"]
    flip = np.roll(np.flip(u0, axis=(0, 1)), (1, 1), axis=(0, 1))  # u0[-y, -x]
    assert np.max(np.abs(flip - np.conj(u0))) <= 1e-9  # v/|v| amplifies rounding where |v| is tiny
    res1 = O.gs_run(I, phi0, 1, init="target")
    Fu = O.fft2u(res1["u"])
    # real up to rounding (amplified where |v| is tiny, so checked after one step)
    assert np.max(np.abs(Fu.imag)) <= 1e-7 * np.max(np.abs(Fu))
    res = O.gs_run(I, phi0, 4, init="target")
    r, g = res["r"], res["g"]
    assert np.all(r[:-1] - g >= -1e-12) and np.all(g - r[1:] >= -1e-12)


# ---------------------------------------------------------------- gradient (differentiable form)


def check_gradient_fd(n=32, seed=11, h=1e-6, p=None):
    rng = np.random.default_rng(seed)
    phi = rng.random((n, n)) * 2 * np.pi
    I = S.spot_target(seed, n, n, 4).astype(np.float64)
    I *= I.size / I.sum()  # sum I = N
    g = O.intensity_loss_grad(phi, I, p)
    idx = rng.choice(phi.size, size=48, replace=False)
    fd = np.empty(len(idx))
    for t, k in enumerate(idx):
        e = np.zeros(phi.size)
        e[k] = h
        e = e.reshape(phi.shape)
        fd[t] = (O.intensity_loss(phi + e, I, p) - O.intensity_loss(phi - e, I, p)) / (2 * h)
    ga = g.ravel()[idx]
    err = np.linalg.norm(ga - fd) / np.linalg.norm(fd)
    assert err <= 1e-6, err


def test_gradient_finite_differences():
    check_gradient_fd()


def test_gradient_finite_differences_with_laser_amplitude():
    check_gradient_fd(p=laser_profile(32, 32, 9).astype(np.float64))


def check_intensity_loss_closed_forms(seed=12):
    """The value of the intensity loss where the field's transform is known.

    A constant phase c gives x = e^{ic}, so y = F x = N e^{ic} at zero
    frequency and 0 elsewhere, |y|^2/N = N delta_0 and
    L = (N - I_0)^2 + sum_{k != 0} I_k^2. A plane-wave phase
    2 pi (a j/nx + b k/ny) moves the delta to frequency (a, b) (row b,
    column a). A constant laser amplitude p0 scales it to N p0^2."""
    rng = np.random.default_rng(seed)
    ny, nx = 8, 16
    n = nx * ny
    I = rng.uniform(0.0, 3.0, (ny, nx))
    c = 0.7
    want = (n - I[0, 0]) ** 2 + np.sum(I**2) - I[0, 0] ** 2
    got = O.intensity_loss(np.full((ny, nx), c), I)
    assert abs(got - want) <= 1e-10 * want, (got, want)
    a, b = 5, 3
    jj = np.arange(nx)[None, :]
    kk = np.arange(ny)[:, None]
    ramp = 2 * np.pi * (a * jj / nx + b * kk / ny) + c
    want = (n - I[b, a]) ** 2 + np.sum(I**2) - I[b, a] ** 2
    got = O.intensity_loss(ramp, I)
    assert abs(got - want) <= 1e-10 * want, (got, want)
    p0 = 1.5
    want = (n * p0**2 - I[0, 0]) ** 2 + np.sum(I**2) - I[0, 0] ** 2
    got = O.intensity_loss(np.full((ny, nx), c), I, np.full((ny, nx), p0))
    assert abs(got - want) <= 1e-10 * want, (got, want)


def test_intensity_loss_closed_forms():
    check_intensity_loss_closed_forms()


def test_gradient_single_pixel_is_zero():
    # N = 1: r is real and the loss does not depend on phi
    g = O.intensity_loss_grad(np.array([[0.3]]), np.array([[2.0]]))
    assert abs(g[0, 0]) <= 1e-15


# ---------------------------------------------------------------- physical error (parity unpinned)


def _field_with_intensity(I, Ir):
    """A field whose normalised reconstructed intensity is exactly Ir (Ir must
    carry the same total as I / max I: a field conserves its energy)."""
    n = I.size
    amp = np.sqrt(Ir * I.max() * n / I.sum())
    return O.ifft2u(amp.astype(complex))


def _moved(It, pix, new_value, peak):
    """It with pixel `pix` set to `new_value` and the difference taken from the
    peak pixel (kept within the lit tolerance), so the total is unchanged."""
    Ir = It.copy()
    delta = new_value - Ir[pix]
    Ir[pix] = new_value
    Ir[peak] -= delta
    assert abs(delta) / It[peak] < O.TL_LIT
    return Ir


def test_physical_error_special_cases():
    I = S.spot_target(4, 16, 16, 3)
    It = I.astype(np.float64) / I.max()
    peak = np.unravel_index(np.argmax(It), It.shape)
    # perfect reconstruction: no violation anywhere
    e_l, e_d = O.physical_error(I, _field_with_intensity(I, It))
    assert abs(e_l) < 1e-12 and abs(e_d) < 1e-12
    lit = tuple(np.argwhere((It > 0.05) & (It < 0.2))[0])
    dark = tuple(np.argwhere(It == 0)[0])
    # a lit pixel off by 3 t_l counts (3 - 1) t_d; one within t_l counts nothing
    Ir = _moved(It, lit, It[lit] * (1 + 3 * O.TL_LIT), peak)
    e_l, e_d = O.physical_error(I, _field_with_intensity(I, Ir))
    assert abs(e_l - 2 * O.TD_DARK) < 1e-9 and abs(e_d) < 1e-12
    Ir = _moved(It, lit, It[lit] * (1 + 0.5 * O.TL_LIT), peak)
    assert abs(O.physical_error(I, _field_with_intensity(I, Ir))[0]) < 1e-12
    # a dark pixel at 5 t_d counts 4 t_d
    Ir = _moved(It, dark, 5 * O.TD_DARK, peak)
    e_l, e_d = O.physical_error(I, _field_with_intensity(I, Ir))
    assert abs(e_d - 4 * O.TD_DARK) < 1e-10 and abs(e_l) < 1e-12
    # the energy normalisation: scaling the field changes nothing
    u = _field_with_intensity(I, Ir)
    assert np.allclose(O.physical_error(I, 3.0 * u), (e_l, e_d), rtol=1e-9, atol=1e-15)
