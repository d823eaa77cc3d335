"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each case patches one function of oracle.gs_oracle for the duration of the
test and runs the pin that should catch it. A pin that still passes on the
mutated oracle would be too weak to trust.
"""

import numpy as np
import pytest
import scipy.fft as sfft

import oracle.gs_oracle as O
from tests import test_oracle_pins as P


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
