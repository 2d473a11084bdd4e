"""Pins of oracle/svt.py (singular value thresholding, Eqs. 16-17).

* Textbook special cases: a diagonal matrix with complex entries is
  soft-thresholded entry by entry (magnitude shrunk, phase kept); a rank-one
  sigma*u*v^H maps to max(sigma - t, 0)*u*v^H.
* Invariants: S_t(P A Q) = P S_t(A) Q for unitary P, Q; S_0 = identity;
  S_t(A) = 0 for t >= sigma_max.
* Prox optimality: S_t(A) minimises t*||Z||_* + 0.5*||Z - A||_F^2, checked
  against random perturbations.
"""
import numpy as np
import pytest

from oracle.svt import svt, svt_rank, nuclear_norm


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _unitary(rng, n):
    q, r = np.linalg.qr(_crandn(rng, n, n))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_diagonal_soft_threshold():
    rng = np.random.default_rng(0)
    d = _crandn(rng, 6)
    t = 0.9 * np.median(np.abs(d))
    A = np.zeros((8, 6), complex)
    for i in range(6):
        A[i, i] = d[i]
    Z = svt(A, t)
    expect = np.zeros_like(A)
    for i in range(6):
        mag = abs(d[i])
        expect[i, i] = (mag - t) * d[i] / mag if mag > t else 0.0
    np.testing.assert_allclose(Z, expect, atol=1e-13)


def test_rank_one():
    rng = np.random.default_rng(1)
    u = _crandn(rng, 7)
    u /= np.linalg.norm(u)
    v = _crandn(rng, 5)
    v /= np.linalg.norm(v)
    A = 3.0 * np.outer(u, v.conj())
    np.testing.assert_allclose(svt(A, 1.25), 1.75 * np.outer(u, v.conj()), atol=1e-13)
    np.testing.assert_allclose(svt(A, 3.5), 0 * A, atol=1e-15)


def test_unitary_invariance_and_limits():
    rng = np.random.default_rng(2)
    A = _crandn(rng, 9, 6)
    P, Q = _unitary(rng, 9), _unitary(rng, 6)
    t = 1.3
    np.testing.assert_allclose(svt(P @ A @ Q, t), P @ svt(A, t) @ Q, atol=1e-12)
    np.testing.assert_allclose(svt(A, 0.0), A, atol=1e-12)
    smax = np.linalg.norm(A, 2)
    assert np.abs(svt(A, smax * 1.0000001)).max() < 1e-12
    assert svt_rank(A, 0.0) == 6


@pytest.mark.parametrize("shape", [(5, 5), (9, 4), (4, 9)])
def test_prox_optimality(shape):
    rng = np.random.default_rng(3 + shape[0])
    A = _crandn(rng, *shape)
    t = 0.6 * np.linalg.svd(A, compute_uv=False)[1]
    Z = svt(A, t)

    def f(W):
        return t * nuclear_norm(W) + 0.5 * np.linalg.norm(W - A) ** 2

    f0 = f(Z)
    for k in range(200):
        scale = 10.0 ** rng.uniform(-6, 0)
        assert f(Z + scale * _crandn(rng, *shape)) >= f0 - 1e-12
