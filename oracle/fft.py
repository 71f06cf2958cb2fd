"""The oracle's own discrete Fourier transform (test infrastructure only).

A plain mixed-radix Cooley-Tukey transform written from the definition
    X[k] = sum_{n<N} x[n] exp(-2 pi i n k / N)        (forward, unnormalised)
    x[n] = (1/N) sum_{k<N} X[k] exp(+2 pi i n k / N)  (inverse)
-- the convention of the discrete operator of Sec. 3, Eq. (18), which needs no cell-volume
factors. It shares nothing with the CUDA transforms (no tables, no plans, no common code).

One step of decimation in time, with a radix p dividing N and M = N / p:
    X[k1 + M k2] = sum_{r<p} exp(-2 pi i r k2 / p) [exp(-2 pi i r k1 / N) Y_r[k1]],
    Y_r = DFT_M of the subsequence x[r], x[r + p], x[r + 2p], ...
(Cooley and Tukey, 1965), applied recursively with p the largest divisor of N up to 32; a
length of at most 32, or a prime length, is the definition itself, summed as a product with
the dense DFT matrix. Every twiddle is exp(-2 pi i ((a b) mod N) / N) evaluated in FP64 from
the exact integer product, so no rounding accumulates through recurrences. The transform runs along
one axis at a time, vectorised over all the others; nothing is blocked or fused.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["fft", "ifft", "fftn", "ifftn", "fft2", "ifft2", "fftfreq", "dft_direct"]


def _radix(n: int) -> int:
    """The largest proper divisor of n that is at most 32 (1 when n is prime)."""
    for p in range(min(32, n - 1), 1, -1):
        if n % p == 0:
            return p
    return 1


def _roots(n: int, exps: np.ndarray, sign: float) -> np.ndarray:
    """exp(sign 2 pi i e / n) for integer exponents e, reduced modulo n first."""
    e = np.mod(exps, n).astype(np.float64)
    ang = sign * 2.0 * math.pi * e / n
    return np.cos(ang) + 1j * np.sin(ang)


def _dft_matrix(n: int, sign: float) -> np.ndarray:
    """W[k, j] = exp(sign 2 pi i j k / n)."""
    k = np.arange(n)
    return _roots(n, np.outer(k, k), sign)


def _dit(x: np.ndarray, sign: float) -> np.ndarray:
    """Unnormalised DFT of each row of a C-contiguous complex128 array of shape (B, n)."""
    b, n = x.shape
    p = _radix(n) if n > 32 else 1
    if p == 1:
        # short or prime length: the definition, X = x W^T, as one matrix product
        return x @ _dft_matrix(n, sign).T
    m = n // p
    # subsequences x[r + p j], j < m, for each r < p: rows of shape (B p, m)
    sub = np.ascontiguousarray(x.reshape(b, m, p).transpose(0, 2, 1)).reshape(b * p, m)
    Y = _dit(sub, sign).reshape(b, p, m)                              # DFT_m of each subsequence
    T = Y * _roots(n, np.arange(p)[:, None] * np.arange(m)[None, :], sign)  # exp(s 2 pi i r k1 / n)
    # p-point DFT over r for every (row, k1): X[k1 + m k2] = sum_r Wp[k2, r] T[r, k1]
    Tr = np.ascontiguousarray(T.transpose(0, 2, 1)).reshape(b * m, p)
    X = (Tr @ _dft_matrix(p, sign).T).reshape(b, m, p)
    return np.ascontiguousarray(X.transpose(0, 2, 1)).reshape(b, n)


def _along(x, axis: int, sign: float) -> np.ndarray:
    a = np.ascontiguousarray(np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1))
    out = _dit(a.reshape(-1, a.shape[-1]), sign).reshape(a.shape)
    return np.moveaxis(out, -1, axis)


def fft(x, axis: int = -1) -> np.ndarray:
    """Forward DFT along one axis (no normalisation)."""
    return _along(x, axis, -1.0)


def ifft(x, axis: int = -1) -> np.ndarray:
    """Inverse DFT along one axis (factor 1/N)."""
    n = np.shape(x)[axis]
    return _along(x, axis, +1.0) / n


def fftn(x, axes) -> np.ndarray:
    """Forward DFT along each of the given axes in turn."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        out = fft(out, ax)
    return out


def ifftn(x, axes) -> np.ndarray:
    """Inverse DFT along each of the given axes in turn."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        out = ifft(out, ax)
    return out


def fft2(x, axes=(-2, -1)) -> np.ndarray:
    return fftn(x, axes)


def ifft2(x, axes=(-2, -1)) -> np.ndarray:
    return ifftn(x, axes)


def fftfreq(n: int, d: float = 1.0) -> np.ndarray:
    """Frequencies of the DFT bins: k / (n d) with k = 0, 1, ..., ceil(n/2) - 1, then the
    negative ones -floor(n/2), ..., -1 (an even length's Nyquist bin is negative)."""
    k = np.arange(n)
    k = np.where(k < (n + 1) // 2, k, k - n)
    return k / (n * d)


def dft_direct(x, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """The definition as an explicit O(N^2) sum along one axis (for pinning the fast form)."""
    a = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = a.shape[-1]
    k = np.arange(n)
    jk = np.outer(k, k) % n  # the exponent j k reduced exactly, in integers
    ang = (1.0 if inverse else -1.0) * 2.0 * math.pi * jk / n
    W = np.cos(ang) + 1j * np.sin(ang)
    out = np.zeros_like(a)
    for j in range(n):  # X[k] = sum_j x[j] w^(j k), term by term
        out = out + a[..., j:j + 1] * W[:, j]
    if inverse:
        out = out / a.shape[-1]
    return np.moveaxis(out, -1, axis)
