"""Centred unitary DFT, sparsifying-filter weights and Hankel multiplicities.

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper used here:
* F^1D / F^2D (Sec. III-A, Eq. 2) are unnormalised in the paper.  The oracle
  uses the centred unitary DFT ``F x = fftshift(fft(ifftshift(x)))/sqrt(N)``
  (DC at index N/2), so that F* F = I as Eq. 15 requires.
* W (Sec. III-A, below Eq. 2) multiplies by "the Fourier transform of a 1D
  sparse transform filter" without naming the filter.  The oracle takes the
  circular first difference (Dx)[n] = x[n] - x[n-1], whose centred DFT gives
  w(k) = 1 - exp(-2*pi*i*(k - N/2)/N), so F(Dx) = w * F(x) exactly.
"""
from __future__ import annotations

import numpy as np


def fftc(x, axis=-1):
    """Centred unitary forward DFT along ``axis`` (library FFT as one step)."""
    x = np.fft.ifftshift(x, axes=axis)
    x = np.fft.fft(x, axis=axis, norm="ortho")
    return np.fft.fftshift(x, axes=axis)


def ifftc(x, axis=-1):
    """Centred unitary inverse DFT along ``axis``."""
    x = np.fft.ifftshift(x, axes=axis)
    x = np.fft.ifft(x, axis=axis, norm="ortho")
    return np.fft.fftshift(x, axes=axis)


def fft2c(x):
    return fftc(fftc(x, axis=-1), axis=-2)


def ifft2c(x):
    return ifftc(ifftc(x, axis=-1), axis=-2)


def filter_weights(N, kind=1):
    """Weights of W (Sec. III-A): kind 0 -> all ones (W = I); kind 1 -> the
    centred DFT of the circular first-difference filter."""
    if kind == 0:
        return np.ones(N, dtype=np.complex128)
    k = np.arange(N)
    return 1.0 - np.exp(-2j * np.pi * (k - N / 2) / N)


def hankel_multiplicity(N, p):
    """c[k] = number of Hankel entries (i, c), 0<=i<N-p+1, 0<=c<p, with i+c = k.

    H* H = diag(c) for the Hankel lift of a length-N vector with window p.
    Counted entry by entry (plain definition)."""
    c = np.zeros(N, dtype=np.float64)
    for i in range(N - p + 1):
        for q in range(p):
            c[i + q] += 1.0
    return c
