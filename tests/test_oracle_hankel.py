"""Pins of oracle/hankel.py.

* H agrees with scipy.linalg.hankel (an independent library routine).
* Rank pins (the annihilating-filter property the paper relies on in
  Sec. I and Sec. III-B): a sum of R distinct complex exponentials gives a
  Hankel matrix of rank exactly R, also after coil concatenation; with
  |z_r| = 1 the conjugate-flipped (VC, Eq. 4) channels keep rank R; a
  piecewise-constant image row with R jumps gives rank R after W; a
  mono-exponential echo decay gives a rank-1 parameter lift (Eq. 7).
* Adjoints: Re<L x, E> = Re<x, L^T E> (real inner product, since the VC
  channels are antilinear) and H* H = diag(multiplicity).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle.transforms import fftc, filter_weights, hankel_multiplicity
from oracle import hankel as hk


def _rel_sv(A):
    s = np.linalg.svd(A, compute_uv=False)
    return s / s[0]


def test_hankel_matches_scipy():
    rng = np.random.default_rng(0)
    for N, p in [(9, 3), (17, 5), (32, 8)]:
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        l = N - p + 1
        ref = scipy.linalg.hankel(v[:l], v[l - 1:])
        np.testing.assert_array_equal(hk.hankel(v, p), ref)
        for i in range(l):
            for c in range(p):
                assert hk.hankel(v, p)[i, c] == v[i + c]


@pytest.mark.parametrize("R", [1, 2, 3, 5])
def test_rank_sum_of_exponentials_multicoil(R):
    rng = np.random.default_rng(R)
    N, p, J = 40, 8, 4
    z = rng.uniform(0.7, 1.0, R) * np.exp(1j * rng.uniform(-np.pi, np.pi, R))
    a = rng.standard_normal((J, R)) + 1j * rng.standard_normal((J, R))
    i = np.arange(N)
    V = a @ (z[:, None] ** i[None, :])                 # [J][N]
    A = hk.lift_vectors(V, None, p, False)
    s = _rel_sv(A)
    assert s[R - 1] > 1e-6 and (R == len(s) or s[R] < 1e-12)


@pytest.mark.parametrize("R", [1, 2, 4])
def test_rank_vc_unit_modulus(R):
    rng = np.random.default_rng(10 + R)
    N, p, J = 48, 8, 3
    z = np.exp(1j * rng.uniform(-np.pi, np.pi, R))      # |z| = 1
    a = rng.standard_normal((J, R)) + 1j * rng.standard_normal((J, R))
    V = a @ (z[:, None] ** np.arange(N)[None, :])
    A = hk.lift_vectors(V, None, p, True)               # [H x_j | H x_j^dagger]
    assert A.shape == (N - p + 1, 2 * J * p)
    s = _rel_sv(A)
    assert s[R - 1] > 1e-6 and s[R] < 1e-12
    # the dagger of a generic (non-unit-modulus) signal does raise the rank
    z2 = 0.8 * z
    V2 = a @ (z2[:, None] ** np.arange(N)[None, :])
    assert _rel_sv(hk.lift_vectors(V2, None, p, True))[R] > 1e-8


@pytest.mark.parametrize("R", [2, 3, 6])
def test_rank_weighted_piecewise_constant(R):
    rng = np.random.default_rng(20 + R)
    N, p = 64, 12
    # circularly piecewise-constant row with exactly R jumps: x = cumsum(d),
    # d has R nonzeros summing to zero, so the circular difference of x is d
    d = np.zeros(N, complex)
    pos = rng.choice(N, R, replace=False)
    d[pos] = rng.uniform(0.5, 2.0, R) * np.exp(1j * rng.uniform(0, 2 * np.pi, R))
    d[pos[-1]] -= d.sum()
    x = np.cumsum(d)
    v = fftc(x)
    A = hk.lift_vectors(v[None], filter_weights(N, 1), p, False)
    s = _rel_sv(A)
    assert s[R - 1] > 1e-6 and s[R] < 1e-12
    # without W the same row is not low rank
    assert _rel_sv(hk.lift_vectors(v[None], None, p, False))[R] > 1e-6


def test_rank_parameter_lift_monoexponential():
    rng = np.random.default_rng(5)
    L, J, M, N, pP = 8, 3, 2, 3, 4
    te = 10.0 * (np.arange(L) + 1)
    t2 = rng.uniform(20, 200, (M, N))
    coil = rng.standard_normal((J, M, N)) + 1j * rng.standard_normal((J, M, N))
    Xi = coil[None] * np.exp(-te[:, None, None, None] / t2[None, None])
    A = hk.lift_param(Xi, pP)                            # [M*N][L-pP+1][J*pP]
    assert A.shape == (M * N, L - pP + 1, J * pP)
    for a in A:
        s = _rel_sv(a)
        assert s[1] < 1e-12


def _rip(a, b):
    return float(np.real(np.vdot(b, a)))             # Re <a, b>


@pytest.mark.parametrize("vc", [False, True])
@pytest.mark.parametrize("weight", [0, 1])
def test_adjoint_identity_rows_cols(vc, weight):
    rng = np.random.default_rng(7 + vc + 2 * weight)
    J, M, N, p = 3, 10, 12, 4
    C = 2 * J if vc else J
    wN, wM = filter_weights(N, weight), filter_weights(M, weight)
    x = rng.standard_normal((J, M, N)) + 1j * rng.standard_normal((J, M, N))
    Er = rng.standard_normal((M, N - p + 1, C * p)) + 1j * rng.standard_normal((M, N - p + 1, C * p))
    Ec = rng.standard_normal((N, M - p + 1, C * p)) + 1j * rng.standard_normal((N, M - p + 1, C * p))
    lhs = _rip(hk.lift_rows(x, wN, p, vc), Er)
    rhs = _rip(x, hk.lift_rows_adjoint(Er, wN, p, vc, J, N))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    lhs = _rip(hk.lift_cols(x, wM, p, vc), Ec)
    rhs = _rip(x, hk.lift_cols_adjoint(Ec, wM, p, vc, J, M))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("vc", [False, True])
def test_adjoint_identity_parameter(vc):
    rng = np.random.default_rng(11 + vc)
    L, J, M, N, p, pP = 6, 2, 3, 10, 4, 3
    C = 2 * J if vc else J
    w = filter_weights(N, 1)
    x = rng.standard_normal((L, J, M, N)) + 1j * rng.standard_normal((L, J, M, N))
    Epe = rng.standard_normal((M * L, N - p + 1, C * p)) + 1j * rng.standard_normal((M * L, N - p + 1, C * p))
    Ep = rng.standard_normal((M * N, L - pP + 1, J * pP)) + 1j * rng.standard_normal((M * N, L - pP + 1, J * pP))
    lhs = _rip(hk.lift_pe(x, w, p, vc), Epe)
    rhs = _rip(x, hk.lift_pe_adjoint(Epe, w, p, vc, L, J, M, N))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    lhs = _rip(hk.lift_param(x, pP), Ep)
    rhs = _rip(x, hk.lift_param_adjoint(Ep, pP, L, J, M, N))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_hankel_normal_is_multiplicity():
    N, p = 13, 5
    for k in range(N):
        e = np.zeros(N, complex)
        e[k] = 1.0
        back = hk.hankel_adjoint(hk.hankel(e, p), N)
        expect = np.zeros(N)
        expect[k] = hankel_multiplicity(N, p)[k]
        np.testing.assert_array_equal(back.real, expect)


def test_dagger_involution_and_antilinearity():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    np.testing.assert_array_equal(hk.dagger(hk.dagger(v)), v)
    np.testing.assert_allclose(hk.dagger(1j * v), -1j * hk.dagger(v))
    assert hk.dagger(v)[0] == np.conj(v[-1])
