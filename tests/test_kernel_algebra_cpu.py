"""Host-side checks of the reformulations the CUDA kernels rely on (CPU, FP64, no oracle).

* The tridiagonal reduction forms each Householder reflector from the column x below
  the diagonal as v = x - alpha e1, alpha = -e^{i arg x0} |x|, tau = 1 / (|x|^2 + |x| |x0|),
  so that (I - tau v v^H) x = alpha e1 with tau real (H Hermitian and unitary).
* The eigenvector kernel applies the reflectors in batches: for reflectors u_j in the
  order of application (real tau_j), applying them one after the other to y equals
      s_j = d_j - sum_{i<j} tau_i C_ji s_i,   d = U^H y,  C = U^H U,
      y <- y - U diag(tau) s.
* The reverse mode evaluates the Daleckii-Krein divided difference of
  h(lambda) = 1 - t / sqrt(lambda) between two eigenvalues above t^2 as
  t / (s_i s_j (s_i + s_j)), s = sqrt(lambda), which has no cancellation.
"""
import numpy as np
import pytest


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _reflector(x):
    x0 = x[0]
    ax0 = abs(x0)
    xn = np.linalg.norm(x)
    phs = x0 / ax0 if ax0 > 0 else 1.0
    v = x.copy()
    v[0] = phs * (ax0 + xn)
    return v, 1.0 / (xn * xn + xn * ax0), -phs * xn


@pytest.mark.parametrize("m", [2, 5, 31, 191])
def test_householder_form_maps_column_to_alpha_e1(m):
    rng = np.random.default_rng(m)
    x = _crandn(rng, m)
    v, tau, alpha = _reflector(x)
    hx = x - tau * v * np.vdot(v, x)
    e = np.zeros(m, complex)
    e[0] = alpha
    assert np.allclose(hx, e, atol=1e-12 * np.linalg.norm(x))
    assert np.isclose(2.0 / tau, np.vdot(v, v).real)        # I - tau v v^H is unitary
    assert np.isclose(abs(alpha), np.linalg.norm(x))


def test_householder_form_real_leading_entry_zero():
    # x0 = 0: the phase defaults to 1 (the kernel's choice), the map still holds
    x = np.array([0.0, 3.0 + 4.0j, -1.0j])
    v, tau, alpha = _reflector(x)
    assert np.allclose(x - tau * v * np.vdot(v, x), [alpha, 0, 0], atol=1e-12)


def _sequential(y, U, tau):
    y = y.copy()
    for j in range(U.shape[1]):
        y = y - tau[j] * np.outer(U[:, j], U[:, j].conj() @ y)
    return y


def _blocked(y, U, tau):
    d = U.conj().T @ y
    C = U.conj().T @ U
    s = np.zeros_like(d)
    for j in range(U.shape[1]):
        s[j] = d[j] - sum(tau[i] * C[j, i] * s[i] for i in range(j))
    return y - U @ (tau[:, None] * s)


@pytest.mark.parametrize("n,kb,nbat", [(192, 189, 8), (40, 6, 7), (9, 2, 3), (57, 0, 1)])
def test_blocked_reflectors_equal_sequential(n, kb, nbat):
    """Batch of reflectors v_{kb}, v_{kb-1}, ... (nested supports rows > k), as staged by
    the kernel; one of them with tau = 0 (a column that was already reduced); several
    right-hand sides (the eigenvectors of a chunk)."""
    rng = np.random.default_rng(n + kb)
    U = np.zeros((n, nbat), complex)
    tau = np.zeros(nbat)
    for j in range(nbat):
        k = kb - j
        v, t, _ = _reflector(_crandn(rng, n - k - 1))
        U[k + 1:, j] = v
        tau[j] = t
    if nbat > 2:
        U[:, 1] = 0.0
        tau[1] = 0.0
    y = _crandn(rng, n, 3)
    ref = _sequential(y, U, tau)
    assert np.allclose(_blocked(y, U, tau), ref, atol=1e-11 * np.linalg.norm(y))
    # the product of the reflectors is unitary: norms are kept
    assert np.allclose(np.linalg.norm(ref, axis=0), np.linalg.norm(y, axis=0))


def test_divided_difference_cancellation_free():
    rng = np.random.default_rng(7)
    t = 0.8
    s = t + rng.uniform(1e-3, 5.0, size=200)
    si, sj = s[:100], s[100:]
    h = lambda x: 1.0 - t / x                                  # noqa: E731
    direct = (h(si) - h(sj)) / (si * si - sj * sj)
    assert np.allclose(t / (si * sj * (si + sj)), direct, rtol=1e-9)
    # equal singular values: the form at s_i = s_j is the derivative h'(lambda), lambda = s^2
    hl = lambda lam: 1.0 - t / np.sqrt(lam)                   # noqa: E731
    for x in s[:5]:
        lam, dl = x * x, 1e-6 * x * x
        deriv = (hl(lam + dl) - hl(lam - dl)) / (2 * dl)
        assert np.isclose(t / (x * x * (x + x)), deriv, rtol=1e-6)
