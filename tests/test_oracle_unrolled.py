"""Pins of the FP64 reverse-mode oracle (SVT derivative, unrolled Algorithm S1).

* ``svt_vjp`` against central finite differences of ``svt`` (FP64, step 1e-6:
  truncation O(h^2 ||S'''||) ~ 1e-12, rounding ~ u/h ~ 1e-10 relative) along
  random directions, in A and in t, for tall, wide and square matrices with
  the threshold inside the spectrum; plus the closed forms t = 0 (S_0 = id,
  so Abar = Zbar and tbar = -Re tr(Zbar^H sum_i u_i v_i^H)) and t > sigma_max
  (S_t = 0 in a neighbourhood: Abar = 0, tbar = 0).
* ``unrolled_2d`` with t_k = 1/beta, tau_k = tau is Algorithm S1 (``shlr``)
  exactly; with varying t_k / tau_k its gradient from ``unrolled_2d_vjp``
  agrees with central differences of the forward in every t_k, tau_k and in
  Y along a random direction (SHLR, SHLR-V, hard data consistency).  The
  last iteration's t, tau do not reach the output: their gradients are 0.
"""
import numpy as np
import pytest

from synth import make_inputs
from synth.configs import get_config
from oracle.svt import svt, svt_vjp
from oracle.admm import shlr
from oracle.unrolled import unrolled_2d, unrolled_2d_vjp


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("shape", [(7, 4), (4, 7), (5, 5), (9, 3)])
def test_svt_vjp_matches_finite_differences(shape):
    rng = np.random.default_rng(11 + shape[0] * 7 + shape[1])
    A = _crandn(rng, *shape)
    s = np.linalg.svd(A, compute_uv=False)
    t = 0.5 * (s[0] + s[1]) if len(s) < 3 else 0.5 * (s[1] + s[2])
    Zb = _crandn(rng, *shape)
    Ab, tb = svt_vjp(A, Zb, t)
    h = 1e-6

    def L(X, tt):
        return np.real(np.vdot(Zb, svt(X, tt)))

    for _ in range(3):
        d = _crandn(rng, *shape)
        fd = (L(A + h * d, t) - L(A - h * d, t)) / (2 * h)
        assert abs(np.real(np.vdot(Ab, d)) - fd) <= 1e-7 * max(1.0, abs(fd))
    fdt = (L(A, t + h) - L(A, t - h)) / (2 * h)
    assert abs(tb - fdt) <= 1e-7 * max(1.0, abs(fdt))


def test_svt_vjp_closed_forms():
    rng = np.random.default_rng(5)
    A = _crandn(rng, 6, 4)
    Zb = _crandn(rng, 6, 4)
    # t = 0: identity map
    Ab, tb = svt_vjp(A, Zb, 0.0)
    assert np.abs(Ab - Zb).max() <= 1e-12
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    assert abs(tb - (-np.real(np.vdot(Zb, U @ Vh)))) <= 1e-12
    # t above every singular value: zero map near A
    Ab, tb = svt_vjp(A, Zb, 1.5 * s[0])
    assert np.abs(Ab).max() == 0.0 and tb == 0.0


def _small_case(model, lam):
    cfg = get_config("shlr_4c_64").with_(model=model, window=4, lam=lam, mask="random1d", R=3.0, n_acs=4)
    inp = make_inputs(cfg, small=(2, 16, 12))
    return cfg, inp["Y"], inp["mask"]


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_unrolled_constant_parameters_is_algorithm_s1(model):
    cfg, Y, U = _small_case(model, 1e4)
    n = 4
    X0 = shlr(Y, U, cfg.with_(n_iter=n))[0]
    Xu = unrolled_2d(Y, U, cfg, np.full(n, 1.0 / cfg.beta), np.full(n, cfg.tau))
    assert np.array_equal(X0, Xu)


@pytest.mark.parametrize("model,lam", [("SHLR", 1e4), ("SHLR_V", 1e4), ("SHLR", -1.0)])
def test_unrolled_vjp_matches_finite_differences(model, lam):
    cfg, Y, U = _small_case(model, lam)
    n = 4
    ts = (1.0 / cfg.beta) * (1.0 + 0.1 * np.arange(n))
    taus = cfg.tau * (1.0 - 0.05 * np.arange(n))
    rng = np.random.default_rng(3)
    Xb = _crandn(rng, *Y.shape)
    tb, taub, Yb = unrolled_2d_vjp(Y, U, cfg, ts, taus, Xb)

    def L(ts_, taus_, Y_):
        return np.real(np.vdot(Xb, unrolled_2d(Y_, U, cfg, ts_, taus_)))

    h = 1e-6
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        fd_t = (L(ts + e, taus, Y) - L(ts - e, taus, Y)) / (2 * h)
        e[k] = h * taus[k]
        fd_tau = (L(ts, taus + e, Y) - L(ts, taus - e, Y)) / (2 * h * taus[k])
        assert abs(tb[k] - fd_t) <= 1e-6 * max(1.0, abs(fd_t)), (k, tb[k], fd_t)
        assert abs(taub[k] - fd_tau) <= 1e-6 * max(abs(fd_tau), 1e-3), (k, taub[k], fd_tau)
    assert tb[-1] == 0.0 and taub[-1] == 0.0
    d = _crandn(rng, *Y.shape)
    fd_y = (L(ts, taus, Y + h * d) - L(ts, taus, Y - h * d)) / (2 * h)
    assert abs(np.real(np.vdot(Yb, d)) - fd_y) <= 1e-6 * max(1.0, abs(fd_y))
