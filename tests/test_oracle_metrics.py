"""Pins of oracle/metrics.py (SSOS, RLNE, MSSIM, T2 fit; Sec. IV and S3).

* SSOS / RLNE against their definitions written out on tiny arrays.
* MSSIM: identical images give 1; constant images give the closed form
  (2ab + C1) / (a^2 + b^2 + C1); a brute-force loop over every window of a
  tiny image, with the Gaussian weights applied by hand, gives the same mean.
* T2 fit: noise-free mono-exponential decays are recovered exactly; on noisy
  data the gradient of the sum of squares is zero at the fit; a decay whose T2
  lies outside the range is excluded.
"""
import numpy as np
import pytest

from oracle import metrics as om


def test_ssos_and_rlne_definitions():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, 4, 5)) + 1j * rng.standard_normal((3, 4, 5))
    s = om.ssos(X)
    for i in range(4):
        for j in range(5):
            assert abs(s[i, j] - np.sqrt(sum(abs(X[c, i, j]) ** 2 for c in range(3)))) < 1e-14
    a, b = rng.standard_normal(20), rng.standard_normal(20)
    assert abs(om.rlne(a, b) - np.sqrt(((a - b) ** 2).sum() / (a ** 2).sum())) < 1e-14


def test_mssim_identical_and_constant_images():
    rng = np.random.default_rng(2)
    A = rng.random((24, 20))
    assert abs(om.mssim(A, A) - 1.0) < 1e-12
    a, b = 0.7, 0.3
    L = 1.0
    C1 = (0.01 * L) ** 2
    val = om.mssim(np.full((16, 16), a), np.full((16, 16), b), L=L)
    assert abs(val - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-10


def test_mssim_matches_brute_force_windows():
    rng = np.random.default_rng(3)
    A = rng.random((15, 14))
    B = A + 0.1 * rng.standard_normal((15, 14))
    w = om.gaussian_window()
    L = A.max()
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    for i in range(15 - 10):
        for j in range(14 - 10):
            a, b = A[i:i + 11, j:j + 11], B[i:i + 11, j:j + 11]
            ma, mb = (w * a).sum(), (w * b).sum()
            va, vb = (w * (a - ma) ** 2).sum(), (w * (b - mb) ** 2).sum()
            cab = (w * (a - ma) * (b - mb)).sum()
            vals.append((2 * ma * mb + C1) * (2 * cab + C2) / ((ma * ma + mb * mb + C1) * (va + vb + C2)))
    assert abs(om.mssim(A, B) - np.mean(vals)) < 1e-12


def test_t2_fit_exact_noiseless_and_stationary_noisy():
    te = 10.0 * np.arange(1, 9)
    t2 = np.array([[20.0, 55.0], [120.0, 200.0]])
    m0 = np.array([[1.0, 0.4], [2.5, 0.9]])
    S = m0[None] * np.exp(-te[:, None, None] / t2[None])
    T2, M0 = om.t2_fit(S, te)
    np.testing.assert_allclose(T2, t2, rtol=1e-9)
    np.testing.assert_allclose(M0, m0, rtol=1e-9)
    rng = np.random.default_rng(4)
    Sn = S * (1 + 0.02 * rng.standard_normal(S.shape))
    T2n, M0n = om.t2_fit(Sn, te)
    for i in range(2):
        for j in range(2):
            r2, mm = 1.0 / T2n[i, j], M0n[i, j]
            e = np.exp(-te * r2)
            res = mm * e - Sn[:, i, j]
            grad = np.array([np.dot(res, e), np.dot(res, -mm * te * e)])
            scale = np.abs(Sn[:, i, j]).max() ** 2 * np.array([1.0, te.max()])
            assert (np.abs(grad) / scale).max() < 1e-7


def test_t2_fit_excludes_out_of_range():
    te = 10.0 * np.arange(1, 9)
    S = np.exp(-te / 5000.0)[:, None]
    T2, _ = om.t2_fit(S, te, t2_range=(1.0, 1000.0))
    assert np.isnan(T2).all()
