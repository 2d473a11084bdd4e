"""Pins of oracle/transforms.py against definitions written independently.

* The centred unitary DFT is compared with the DFT matrix written entry by
  entry from its definition (phase exp(-2 pi i (k-N/2)(n-N/2)/N) / sqrt(N)).
* W: the DFT of an explicitly computed circular first difference equals
  w * DFT(x) (Sec. III-A, reading of the unnamed filter).
* Hankel multiplicity: closed form min(k+1, p, N-k, N-p+1).
"""
import numpy as np
import pytest

from oracle.transforms import fftc, ifftc, fft2c, ifft2c, filter_weights, hankel_multiplicity


def _dft_matrix(N):
    F = np.empty((N, N), dtype=np.complex128)
    for k in range(N):
        for n in range(N):
            F[k, n] = np.exp(-2j * np.pi * (k - N / 2) * (n - N / 2) / N) / np.sqrt(N)
    return F


@pytest.mark.parametrize("N", [4, 6, 8, 10, 12, 16])
def test_fftc_matches_definition(N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    F = _dft_matrix(N)
    np.testing.assert_allclose(fftc(x), F @ x, atol=1e-13)
    np.testing.assert_allclose(ifftc(x), F.conj().T @ x, atol=1e-13)


def test_fftc_centre_and_unitary():
    N = 16
    d = np.zeros(N, complex)
    d[N // 2] = 1.0                                   # image-centre impulse
    np.testing.assert_allclose(fftc(d), np.full(N, 1 / np.sqrt(N)), atol=1e-15)
    one = np.ones(N, complex)
    spec = fftc(one)
    assert abs(spec[N // 2] - np.sqrt(N)) < 1e-12       # DC sits at index N/2
    assert np.abs(np.delete(spec, N // 2)).max() < 1e-12
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3, 8, 12)) + 1j * rng.standard_normal((3, 8, 12))
    assert abs(np.linalg.norm(fft2c(X)) - np.linalg.norm(X)) < 1e-12
    np.testing.assert_allclose(ifft2c(fft2c(X)), X, atol=1e-13)


@pytest.mark.parametrize("N", [8, 16, 64])
def test_weights_are_dft_of_first_difference(N):
    rng = np.random.default_rng(N + 1)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    dx = np.empty_like(x)
    for n in range(N):
        dx[n] = x[n] - x[n - 1]                       # circular: x[-1] = x[N-1]
    np.testing.assert_allclose(fftc(dx), filter_weights(N, 1) * fftc(x), atol=1e-12)
    np.testing.assert_allclose(filter_weights(N, 0), np.ones(N))
    assert abs(filter_weights(N, 1)[N // 2]) < 1e-15   # the difference kills DC


@pytest.mark.parametrize("N,p", [(8, 3), (17, 5), (64, 8), (256, 16), (10, 10), (9, 1)])
def test_multiplicity_closed_form(N, p):
    c = hankel_multiplicity(N, p)
    k = np.arange(N)
    closed = np.minimum.reduce([k + 1, np.full(N, p), N - k, np.full(N, N - p + 1)])
    np.testing.assert_array_equal(c, closed)
    assert c.sum() == (N - p + 1) * p
