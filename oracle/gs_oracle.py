"""FP64 CPU oracle for the method of alternating projections (Gerchberg-Saxton).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

Every function cites the passage of the paper it restates (Kramer, Hagemann,
Luke, "Real-Time Phase Masks for Interactive Stimulation of Optogenetic
Neurons"). The code follows the paper's steps in its order and notation. The
Fourier transform is the oracle's own (oracle/dft.py: direct DFT sums and the
mixed-radix Cooley-Tukey factorisation), with no FFT library behind it.

Conventions (the paper fixes none of them; these are the readings used):
  * A grid is stored as an array ``[ny, nx]`` (row-major, element ``(j, k)``
    of the paper at ``[k, j]``), i.e. the paper's lexicographic pixel index.
  * ``F`` is the unnormalised 2D DFT with kernel
    ``exp(-2*pi*i*(j*k1/nx + k*k2/ny))``; ``F_u = F / sqrt(N)`` is unitary.
    The projections are computed with ``F_u`` so that the object and Fourier
    domains carry the same Euclidean norm.
  * The OSP amplitude is ``m = sqrt(I)`` rescaled so that ``sum m^2`` equals
    the energy ``sum p^2`` of an SLM field (``N`` for unit amplitude p = 1;
    Eq. pattern-constraint gives m as an amplitude; the scale is unstated and
    does not change the iterates).
  * Where the paper allows an arbitrary phase for a zero pixel (Eqs. e:PS and
    e:Mhat), theta = 0 is chosen, with an exact-zero test.
  * Both gaps are divided by ``||p||_2 = ||u||`` (``sqrt(N)`` for p = 1).
  * The initial condition ``P_M uhat^0`` of Sec. IV (garbled) is read as
    ``u0 = P_S(F^{-1} m)``; the default start is ``u0 = p exp(i phi0)``.

Parity status:
  fft2u / ifft2u (oracle/dft.py), target_amplitude, proj_S, proj_M, gap_to_M, gap_to_S,
  gs_step, gs_run, consistent_target, intensity_loss, intensity_loss_grad:
      pinned by the tests in tests/test_oracle_pins.py (brute-force DFT,
      Parseval, idempotence, nearest-point property, the interleaved gap chain,
      fixed points of consistent targets, scale invariance, finite
      differences, closed-form values of the loss for constant and
      plane-wave phases).
  physical_error: parity unpinned. The paper prints no value of E; its printed
      formula is restated under the reading documented on the function, and
      only special cases that follow from its definition are tested.
"""

from __future__ import annotations

import numpy as np

from . import dft as _dft

# Tolerances of the physical error, Sec. II (relative on lit pixels, absolute
# on dark pixels).
TL_LIT = 0.1
TD_DARK = 3e-4


def _complex_dtype(real_dtype):
    return np.complex64 if np.dtype(real_dtype) == np.float32 else np.complex128


def fft2u(x: np.ndarray) -> np.ndarray:
    """Unitary forward 2D DFT ``F_u x`` over the last two axes ([ny, nx]).

    The Fourier transform F of Sec. II that maps the SLM field to the
    stimulation pattern (Fraunhofer diffraction), with numpy's sign convention.
    """
    x = np.asarray(x)
    return _dft.dft2(x) / float(np.sqrt(x.shape[-1] * x.shape[-2]))  # a Python float keeps FP32 runs in FP32


def ifft2u(X: np.ndarray) -> np.ndarray:
    """Unitary inverse 2D DFT ``F_u^{-1} X`` (the ``F^{-1}`` of Eq. e:PM)."""
    X = np.asarray(X)
    return _dft.idft2(X) / float(np.sqrt(X.shape[-1] * X.shape[-2]))


def target_amplitude(I: np.ndarray, dtype=np.float64, energy: float | None = None) -> np.ndarray:
    """OSP amplitude m from a target intensity I (Eq. pattern-constraint).

    m is an amplitude, so ``m = sqrt(I)``; it is rescaled so that
    ``sum m^2`` equals the squared norm of every field in the SLM set S:
    ``energy = sum p^2`` (``N`` for unit amplitude, the default). Raises
    ValueError for a non-finite, negative or all-zero I.
    """
    I = np.asarray(I, dtype=np.float64)
    if not np.all(np.isfinite(I)):
        raise ValueError("target intensity has non-finite values")
    if np.any(I < 0):
        raise ValueError("target intensity has negative values")
    total = float(np.sum(I))
    if not total > 0.0:
        raise ValueError("target intensity sums to zero")
    e = float(I.size) if energy is None else float(energy)
    m = np.sqrt(I) * np.sqrt(e / total)
    return m.astype(dtype)


def proj_S(u: np.ndarray, p: np.ndarray | None = None) -> np.ndarray:
    """Projection onto S, Eq. (e:PS): ``v = p u/|u|``, and ``p`` where u = 0.

    ``p`` is the laser amplitude on the SLM (Eq. slm-constraint); it defaults
    to 1 everywhere (unit modulus, a phase-only mask).
    """
    if p is None:
        p = np.ones(u.shape, dtype=u.real.dtype)
    a = np.abs(u)
    nz = a != 0
    v = np.empty_like(u)
    v[nz] = p[nz] * (u[nz] / a[nz])
    v[~nz] = p[~nz]
    return v


def _mhat(Fu: np.ndarray, m: np.ndarray) -> np.ndarray:
    """The selection from Mhat(u), Eq. (e:Mhat): ``m Fu/|Fu|``, ``m`` where Fu = 0."""
    a = np.abs(Fu)
    nz = a != 0
    out = np.empty_like(Fu)
    out[nz] = m[nz] * (Fu[nz] / a[nz])
    out[~nz] = m[~nz]
    return out


def proj_M(u: np.ndarray, m: np.ndarray) -> np.ndarray:
    """Projection onto M, Eq. (e:PM): ``F^{-1} uhat`` with uhat from Eq. (e:Mhat)."""
    return ifft2u(_mhat(fft2u(u), m))


def _norm_S(shape, p):
    """||u|| for u in S: sqrt(sum p^2) (sqrt(N) for unit amplitude)."""
    return np.sqrt(float(np.prod(shape))) if p is None else float(np.sqrt(np.sum(np.asarray(p, np.float64) ** 2)))


def gap_to_M(u: np.ndarray, m: np.ndarray, p: np.ndarray | None = None) -> float:
    """Normalised distance of u to M, ``||u - P_M u||_2 / ||p||_2``.

    Computed in the Fourier domain, where (Parseval) it equals
    ``|| |F_u u| - m ||_2 / ||p||_2``; ``||p||_2 = sqrt(N)`` for unit
    amplitude. This is the normalised OSP residual r.
    """
    Fu = fft2u(u)
    return float(np.linalg.norm((np.abs(Fu) - m).ravel().astype(np.float64)) / _norm_S(u.shape, p))


def gap_to_S(v: np.ndarray, p: np.ndarray | None = None) -> float:
    """Normalised distance of v to S, ``||v - P_S v||_2 / ||p||_2 = || |v| - p ||_2 / ||p||_2``."""
    pp = 1.0 if p is None else p
    return float(np.linalg.norm((np.abs(v) - pp).ravel().astype(np.float64)) / _norm_S(v.shape, p))


def gs_step(u: np.ndarray, m: np.ndarray, p: np.ndarray | None = None):
    """One step of Eq. (e:AP), ``u' = P_S P_M u``, with both gaps of Eq. (gap-error).

    Returns ``(u_next, r, g)`` where ``r = ||u - P_M u|| / ||p||`` (the
    distance of the current iterate to M, the normalised OSP residual) and
    ``g = ||P_M u - P_S P_M u|| / ||p||`` (the distance of the M-iterate to
    S). Eq. (gap-error) writes the gap as ``||P_S u - P_M u||``; since the
    iterate alternates between the sets, both readings are reported.
    ``p`` is the SLM amplitude of Eq. (slm-constraint) (None: 1).
    """
    Fu = fft2u(u)
    r = float(np.linalg.norm((np.abs(Fu) - m).ravel().astype(np.float64)) / _norm_S(u.shape, p))
    v = ifft2u(_mhat(Fu, m))  # P_M u, Eq. (e:PM)
    g = gap_to_S(v, p)
    u_next = proj_S(v, p)  # Eq. (e:PS)
    return u_next, r, g


def gs_run(I, phi0, iters: int, final_residual: bool = True, dtype=np.float64, p=None, init: str = "phase"):
    """The method of alternating projections, Eq. (e:AP).

    Start ``init="phase"``: ``u0 = p exp(i phi0)``. Start ``init="target"``:
    the initial condition of Sec. IV, read as ``u0 = P_S(F^{-1} m)`` (the
    target amplitude brought to the SLM plane and adapted to the SLM
    constraint); ``phi0`` is then unused. ``p`` is the SLM amplitude of Eq.
    (slm-constraint), float32 [ny, nx] >= 0 (None: 1); the target amplitude
    carries the same energy, ``sum m^2 = sum p^2``.

    Inputs are the arrays the GPU receives; they are widened exactly to
    ``dtype`` (FP64 by default; FP32 reproduces the paper's single-precision
    runs, Sec. IV.B). Returns a dict with
      ``phase``  the final mask ``arg u^K`` in (-pi, pi],
      ``u``      the final iterate ``u^K``,
      ``r``      ``r^0..r^K`` (``r^K`` only if ``final_residual``),
      ``g``      ``g^0..g^{K-1}``.
    """
    if iters < 0:
        raise ValueError("iters must be >= 0")
    rdt = np.dtype(dtype)
    cdt = _complex_dtype(rdt)
    I = np.asarray(I)
    pw = None if p is None else np.asarray(p, dtype=np.float32).astype(rdt)
    energy = None if pw is None else float(np.sum(pw.astype(np.float64) ** 2))
    m = target_amplitude(I, dtype=rdt, energy=energy)
    if init == "phase":
        phi = np.asarray(phi0, dtype=np.float32).astype(rdt)
        u = np.exp(1j * phi).astype(cdt)
        if pw is not None:
            u = (pw * u).astype(cdt)
    elif init == "target":
        u = proj_S(ifft2u(m.astype(cdt)), pw).astype(cdt)
    else:
        raise ValueError("init must be 'phase' or 'target'")
    r_hist, g_hist = [], []
    for _ in range(iters):
        u, r, g = gs_step(u, m, pw)
        r_hist.append(r)
        g_hist.append(g)
    if final_residual:
        r_hist.append(gap_to_M(u, m, pw))
    phase = np.angle(u)
    phase = np.where(phase <= -np.pi, np.pi, phase)
    return {
        "phase": phase.astype(np.float64),
        "u": u,
        "r": np.asarray(r_hist, dtype=np.float64),
        "g": np.asarray(g_hist, dtype=np.float64),
    }


def consistent_target(phi_true) -> np.ndarray:
    """A consistent problem: ``I = |F exp(i phi_true)|^2`` (Eq. e:feas has a solution).

    ``exp(i phi_true)`` lies in S and, with ``m = sqrt(I)`` rescaled, in M, so
    S and M intersect. Returned in FP64 and unnormalised (any positive scale
    gives the same problem).
    """
    x = np.exp(1j * np.asarray(phi_true, dtype=np.float32).astype(np.float64))
    return np.abs(_dft.dft2(x)) ** 2


def physical_error(I, u, t_l: float = TL_LIT, t_d: float = TD_DARK):
    """Physical error ``E = E_l + E_d`` of Eq. (phys-error). PARITY UNPINNED.

    Reading of the garbled passage: both the target and the reconstruction are
    compared as intensities normalised to the target's peak,
      ``It = I / max I`` and
      ``Ir = |F_u u|^2 * (sum I / ||u||^2) / max I``
    (the reconstruction carries the target's total energy; ``||u||^2 = N``
    for a unit-amplitude field, ``sum p^2`` with a laser amplitude p). A pixel is lit if
    ``It > 0``. The formula is evaluated as printed:
      ``E_l = sum_lit (t_d |It - Ir| / (t_l It) - t_d) * Theta(|It - Ir|/It - t_l)``
      ``E_d = sum_dark (Ir - t_d) * Theta(Ir - t_d)``,  Theta(0) = 0.
    Returns ``(E_l, E_d)``.
    """
    I = np.asarray(I, dtype=np.float64)
    u = np.asarray(u, dtype=np.complex128)
    energy = float(np.sum(np.abs(u) ** 2))
    imax = float(I.max())
    It = I / imax
    Ir = np.abs(fft2u(u)) ** 2 * (float(I.sum()) / energy) / imax
    lit = It > 0
    rel = np.zeros_like(It)
    rel[lit] = np.abs(It[lit] - Ir[lit]) / It[lit]
    over_l = lit & (rel - t_l > 0)
    e_l = float(np.sum(t_d * rel[over_l] / t_l - t_d))
    dark = ~lit
    over_d = dark & (Ir - t_d > 0)
    e_d = float(np.sum(Ir[over_d] - t_d))
    return e_l, e_d


def intensity_loss(phi, I, p=None) -> float:
    """Intensity loss ``L = sum (|F x|^2 / N - I)^2``, ``x = p exp(i phi)``,
    with the unnormalised F (p = 1 by default).

    The differentiable form of the same inverse problem (fit |F u|^2 to the
    target intensity over u in S, Sec. II).
    """
    phi = np.asarray(phi, dtype=np.float64)
    I = np.asarray(I, dtype=np.float64)
    pw = 1.0 if p is None else np.asarray(p, dtype=np.float64)
    y = _dft.dft2(pw * np.exp(1j * phi))
    r = np.abs(y) ** 2 / phi.size - I
    return float(np.sum(r * r))


def intensity_loss_grad(phi, I, p=None) -> np.ndarray:
    """Analytic gradient of ``intensity_loss`` with respect to phi.

    With ``x = p exp(i phi)``, ``y = F x``, ``r = |y|^2/N - I``:
    ``dL/dphi = 4 Im(conj(x) * F^{-1}(r * y))`` (F^{-1} the normalised inverse),
    from ``d y_k / d phi_j = F_kj i x_j`` and the symmetry of F.
    """
    phi = np.asarray(phi, dtype=np.float64)
    I = np.asarray(I, dtype=np.float64)
    pw = 1.0 if p is None else np.asarray(p, dtype=np.float64)
    x = pw * np.exp(1j * phi)
    y = _dft.dft2(x)
    r = np.abs(y) ** 2 / phi.size - I
    z = _dft.idft2(r * y) / phi.size
    return 4.0 * np.imag(np.conj(x) * z)
