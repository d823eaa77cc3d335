"""The oracle's own discrete Fourier transform, FP64 (test infrastructure only).

The paper computes the Fourier transform F of Sec. II with an FFT (Sec. III:
cuFFT on the GPU, FFTW on the CPU). This module is the oracle's transform,
written from the definitions, with no FFT library behind it:

  * the DFT of length n is ``X[k] = sum_j x[j] W_n^{jk}``, ``W_n = exp(-2 pi i/n)``
    (unnormalised, numpy's sign convention);
  * short lengths (n <= 64) and prime lengths are computed by that sum
    directly, as a product with the n x n matrix ``W_n^{jk}`` whose entries
    are evaluated from cos/sin of ``2 pi (jk mod n)/n`` in FP64;
  * longer composite lengths use one step of the mixed-radix Cooley-Tukey
    factorisation n = n1 n2 (Cooley and Tukey, 1965): with ``j = n2 j1 + j2``
    and ``k = k1 + n1 k2``,
        ``X[k1 + n1 k2] = sum_j2 W_n2^{j2 k2} W_n^{j2 k1} sum_j1 W_n1^{j1 k1} x[n2 j1 + j2]``
    i.e. length-n1 transforms over j1, a twiddle ``W_n^{j2 k1}``, length-n2
    transforms over j2, each of which recurses the same way.

Any length works (the 5-smooth SLM sides of Sec. V included); accuracy is that
of sums of at most 64 terms per stage. The arithmetic is FP64 (complex128); a
single-precision input (float32, complex64) is transformed in single precision
with the same factors rounded once, to restate the paper's SP runs (Sec. IV.B).
The matrix products may run on several BLAS threads.
"""

from __future__ import annotations

import functools

import numpy as np

# Lengths up to this are transformed by the direct sum.
DIRECT_MAX = 64


@functools.lru_cache(maxsize=None)
def _smallest_factor(n: int) -> int:
    f = 2
    while f * f <= n:
        if n % f == 0:
            return f
        f += 1
    return n


@functools.lru_cache(maxsize=None)
def _split(n: int) -> int:
    """n1 of the factorisation n = n1 n2: the largest divisor of n not above
    sqrt(n) (1 for a prime n)."""
    best = 1
    d = 1
    while d * d <= n:
        if n % d == 0:
            best = d
        d += 1
    return best


def _roots(e: np.ndarray, n: int) -> np.ndarray:
    """W_n^e = exp(-2 pi i e / n) for integer exponents e, reduced mod n first
    so that the angle stays in [0, 2 pi)."""
    a = 2.0 * np.pi * (np.asarray(e, dtype=np.int64) % n) / n
    return np.cos(a) - 1j * np.sin(a)


@functools.lru_cache(maxsize=None)
def _dft_matrix(n: int, dtype) -> np.ndarray:
    j = np.arange(n)
    return _roots(np.outer(j, j), n).astype(dtype)  # symmetric: W_n^{jk}


@functools.lru_cache(maxsize=None)
def _twiddle(n1: int, n2: int, dtype) -> np.ndarray:
    """W_n^{j2 k1}, n = n1 n2, as an [n1 (k1), n2 (j2)] array."""
    return _roots(np.outer(np.arange(n1), np.arange(n2)), n1 * n2).astype(dtype)


def _as_complex(x) -> np.ndarray:
    x = np.asarray(x)
    single = x.dtype in (np.float32, np.complex64)
    return x.astype(np.complex64 if single else np.complex128, copy=False)


def dft_last(x: np.ndarray) -> np.ndarray:
    """Unnormalised forward DFT along the last axis (FP64, or FP32 for a
    single-precision input)."""
    x = _as_complex(x)
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    n1 = _split(n)
    if n <= DIRECT_MAX or n1 == 1:
        return x @ _dft_matrix(n, x.dtype)  # the defining sum
    n2 = n // n1
    a = x.reshape(x.shape[:-1] + (n1, n2))  # a[j1, j2] = x[n2 j1 + j2]
    b = dft_last(np.swapaxes(a, -1, -2))  # b[j2, k1] = sum_j1 W_n1^{j1 k1} a[j1, j2]
    c = np.swapaxes(b, -1, -2) * _twiddle(n1, n2, x.dtype)  # c[k1, j2] = W_n^{j2 k1} b[j2, k1]
    d = dft_last(c)  # d[k1, k2] = sum_j2 W_n2^{j2 k2} c[k1, j2]
    return np.swapaxes(d, -1, -2).reshape(x.shape)  # X[k1 + n1 k2] = d[k1, k2]


def idft_last(X: np.ndarray) -> np.ndarray:
    """Unnormalised inverse DFT along the last axis: ``sum_k X[k] W_n^{-jk}``,
    computed as ``conj(DFT(conj(X)))``."""
    return np.conj(dft_last(np.conj(_as_complex(X))))


def dft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised 2D DFT over the last two axes ([ny, nx]): rows, then
    columns. Returned C-contiguous (row-major), like its input layout."""
    rows = dft_last(x)
    return np.ascontiguousarray(np.swapaxes(dft_last(np.swapaxes(rows, -1, -2)), -1, -2))


def idft2(X: np.ndarray) -> np.ndarray:
    """Unnormalised 2D inverse DFT over the last two axes (no 1/N)."""
    return np.conj(dft2(np.conj(_as_complex(X))))
