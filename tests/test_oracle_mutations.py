"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each case patches one function of oracle.gs_oracle for the duration of the
test and runs the pin that should catch it. A pin that still passes on the
mutated oracle would be too weak to trust.
"""

import numpy as np
import pytest
import scipy.fft as sfft

import oracle.dft as D
import oracle.gs_oracle as O
from tests import test_oracle_pins as P

_TWIDDLE = D._twiddle


def _wrong_sign_fft(x):
    return sfft.ifft2(x, norm="ortho")


def _unnormalised_fft(x):
    return sfft.fft2(x)


def _transposed_fft(x):
    return sfft.fft2(x.T, norm="ortho").T.reshape(x.shape) if x.shape[0] == x.shape[1] else sfft.fft2(
        x.reshape(x.shape[::-1]), norm="ortho"
    ).reshape(x.shape)


def _mhat_intensity(Fu, m):
    a = np.abs(Fu)
    return np.where(a != 0, m * m * Fu / np.where(a != 0, a, 1), m * m)


def _mhat_no_phase(Fu, m):
    return m.astype(Fu.dtype)


def _proj_S_ignores_p(u, p=None):
    a = np.abs(u)
    return np.where(a != 0, u / np.where(a != 0, a, 1), 1.0)


def _amp_is_intensity(I, dtype=np.float64):
    I = np.asarray(I, dtype=np.float64)
    return (I * np.sqrt(I.size / np.sum(I * I))).astype(dtype)


def _gs_step_late_residual(u, m):
    v = O.proj_M(u, m)
    u1 = O.proj_S(v)
    return u1, O.gap_to_M(u1, m), O.gap_to_S(v)


def _grad_wrong_sign(phi, I, p=None):
    x = np.exp(1j * phi)
    y = sfft.fft2(x)
    r = np.abs(y) ** 2 / phi.size - I
    return -4.0 * np.imag(np.conj(x) * sfft.ifft2(r * y))


def _grad_dropped_factor(phi, I, p=None):
    x = np.exp(1j * phi)
    y = sfft.fft2(x)
    r = np.abs(y) ** 2 / phi.size - I
    return 2.0 * np.imag(np.conj(x) * sfft.ifft2(r * y))


def _norm_S_ignores_p(shape, p):
    return np.sqrt(float(np.prod(shape)))


def _amp_unit_energy(I, dtype=np.float64, energy=None):
    I = np.asarray(I, dtype=np.float64)
    return (np.sqrt(I) * np.sqrt(I.size / I.sum())).astype(dtype)


def _loss_amplitude(phi, I, p=None):
    pw = 1.0 if p is None else np.asarray(p, dtype=np.float64)
    y = sfft.fft2(pw * np.exp(1j * np.asarray(phi, np.float64)))
    r = np.abs(y) / np.sqrt(phi.size) - I  # the amplitude |y|/sqrt(N) fitted instead of the intensity ...
    return float(np.sum(r * r))


def _grad_amplitude(phi, I, p=None):
    """... and the exact gradient of that wrong loss, so the pair stays
    consistent: d/dphi of sum (|y|/sqrt(N) - I)^2 = 2 sqrt(N) Im(conj(x) F^{-1}(r y/|y|))."""
    pw = 1.0 if p is None else np.asarray(p, dtype=np.float64)
    x = pw * np.exp(1j * np.asarray(phi, np.float64))
    y = sfft.fft2(x)
    r = np.abs(y) / np.sqrt(phi.size) - I
    return 2.0 * np.sqrt(phi.size) * np.imag(np.conj(x) * sfft.ifft2(r * y / np.abs(y)))


def _twiddle_conjugated(n1, n2, dtype):
    return np.conj(_TWIDDLE(n1, n2, dtype))


def _dft_no_reorder(x):
    """The Cooley-Tukey step with its output left in [k1][k2] order."""
    x = D._as_complex(x)
    n = x.shape[-1]
    n1 = D._split(n)
    if n <= D.DIRECT_MAX or n1 == 1:
        return x @ D._dft_matrix(n, x.dtype)
    n2 = n // n1
    a = x.reshape(x.shape[:-1] + (n1, n2))
    b = _dft_no_reorder(np.swapaxes(a, -1, -2))
    c = np.swapaxes(b, -1, -2) * D._twiddle(n1, n2, x.dtype)
    return _dft_no_reorder(c).reshape(x.shape)


MUTATIONS = [
    ("fft2u", _wrong_sign_fft, lambda: P.check_fft_direct((8, 32))),
    ("fft2u", _unnormalised_fft, P.check_fft_identities),
    ("fft2u", _transposed_fft, lambda: P.check_fft_direct((8, 32))),
    ("_mhat", _mhat_intensity, P.check_proj_M),
    ("_mhat", _mhat_no_phase, P.check_proj_M),
    ("proj_S", _proj_S_ignores_p, P.check_proj_S),
    ("target_amplitude", _amp_is_intensity, P.check_target_amplitude),
    ("gs_step", _gs_step_late_residual, P.check_gap_definitions),
    ("intensity_loss_grad", _grad_wrong_sign, P.check_gradient_fd),
    ("intensity_loss_grad", _grad_dropped_factor, P.check_gradient_fd),
    ("_norm_S", _norm_S_ignores_p, P.check_slm_amplitude_chain),
    ("target_amplitude", _amp_unit_energy, P.check_slm_amplitude_chain),
]


@pytest.mark.parametrize("name,bad,pin", MUTATIONS, ids=[f"{m[0]}:{m[1].__name__}" for m in MUTATIONS])
def test_pin_catches_mutation(monkeypatch, name, bad, pin):
    monkeypatch.setattr(O, name, bad)
    with pytest.raises(AssertionError):
        pin()


# Mistakes that span several functions or sit in the oracle's own FFT:
# (module, {name: replacement}, pin).
MULTI_MUTATIONS = [
    # the same slip in the loss and its gradient (amplitude fitted instead of
    # intensity): the finite-difference pin stays green, the closed-form
    # values do not
    ("loss-grad:amplitude-for-intensity", O,
     {"intensity_loss": _loss_amplitude, "intensity_loss_grad": _grad_amplitude},
     P.check_intensity_loss_closed_forms),
    ("dft:twiddle-conjugated", D, {"_twiddle": _twiddle_conjugated}, lambda: P.check_fft_long(1024)),
    ("dft:twiddle-conjugated-2d", D, {"_twiddle": _twiddle_conjugated}, lambda: P.check_fft_direct((72, 80))),
    ("dft:no-output-reorder", D, {"dft_last": _dft_no_reorder}, lambda: P.check_fft_long(800)),
]


def test_shared_slip_passes_the_fd_pin(monkeypatch):
    """The shared slip above is one the finite-difference pin cannot see."""
    monkeypatch.setattr(O, "intensity_loss", _loss_amplitude)
    monkeypatch.setattr(O, "intensity_loss_grad", _grad_amplitude)
    P.check_gradient_fd()


@pytest.mark.parametrize("case", MULTI_MUTATIONS, ids=[m[0] for m in MULTI_MUTATIONS])
def test_pin_catches_multi_mutation(monkeypatch, case):
    _, mod, patches, pin = case
    for name, bad in patches.items():
        monkeypatch.setattr(mod, name, bad)
    with pytest.raises(AssertionError):
        pin()
