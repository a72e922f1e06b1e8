"""The oracle's own discrete Fourier transform (test infrastructure).

The DFT of Sec. 2.2-2.3 written out as a plain mixed-radix Cooley-Tukey
transform, so that the oracle's FFT route can be checked against a transform
that shares no code with any FFT library:

    X[k] = sum_{j=0}^{n-1} x[j] exp(-2 pi i j k / n)          (forward)
    x[j] = (1/n) sum_{k=0}^{n-1} X[k] exp(+2 pi i j k / n)    (inverse)

A length n = r m (r = 2 or 3, the factors of the grids the paper's doubled
meshes use) splits into the r decimated subsequences x[q r + s], each
transformed with length m; output k + m t (t < r) is
sum_s w^{s (k + m t)} F_s[k] with w = exp(-2 pi i / n).  Lengths with another
prime factor fall back to the definition (a matrix product).  Every
transform runs along one axis of an array, vectorised over the others.  FP64
(complex128) throughout; no pruning, no symmetry.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n, inverse=False):
    """The n x n DFT matrix exp(-+2 pi i j k / n) (the definition)."""
    j = np.arange(n)
    sign = 1.0 if inverse else -1.0
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


def _fft_last(a, inverse):
    """Unnormalised DFT along the last axis of a complex array."""
    n = a.shape[-1]
    if n == 1:
        return a.copy()
    r = 2 if n % 2 == 0 else 3 if n % 3 == 0 else 0
    if r == 0:  # another prime factor: the definition
        return a @ dft_matrix(n, inverse).T
    m = n // r
    # F[s] = DFT_m of the subsequence x[q r + s], q < m
    F = np.stack([_fft_last(a[..., s::r], inverse) for s in range(r)])
    sign = 1.0 if inverse else -1.0
    k = np.arange(m)
    out = np.empty(a.shape, dtype=np.complex128)
    for t in range(r):
        acc = np.zeros(a.shape[:-1] + (m,), dtype=np.complex128)
        for s in range(r):
            acc = acc + F[s] * np.exp(sign * 2j * np.pi * s * (k + m * t) / n)
        out[..., m * t:m * (t + 1)] = acc
    return out


def fft_axis(a, axis, inverse=False):
    """DFT of a along one axis (inverse: with the 1/n normalisation)."""
    b = np.moveaxis(np.asarray(a, dtype=np.complex128), axis, -1)
    out = _fft_last(b, inverse)
    if inverse:
        out = out / b.shape[-1]
    return np.moveaxis(out, -1, axis)


def fftn(a):
    """Forward DFT over every axis (unnormalised)."""
    out = np.asarray(a, dtype=np.complex128)
    for ax in range(out.ndim):
        out = fft_axis(out, ax)
    return out


def ifftn(a):
    """Inverse DFT over every axis (1 / size normalisation)."""
    out = np.asarray(a, dtype=np.complex128)
    for ax in range(out.ndim):
        out = fft_axis(out, ax, inverse=True)
    return out
