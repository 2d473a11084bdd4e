"""Pins of oracle/admm.py (Algorithms S1 and S2, Eq. 15 / S7).

* The pointwise k-space divide of Eq. 15 (no G) equals a dense
  normal-equation solve built from the literal image-domain operators
  (Eq. 2 / 4 / 5), for SHLR and SHLR-V, with and without W; same for Eq. S7
  (SHLR-P / SHLR-VP).
* Fixed point: fully sampled data with hard data consistency leaves X = F*Y
  at every iteration.
* Homogeneity: (Y, lambda, beta, tau) -> (cY, lambda/c, beta/c, tau/c) gives
  X -> cX (the threshold 1/beta scales with the data).
* Blockwise descent of the augmented Lagrangian (Eq. 9): the X-step and the
  Z-step are exact minimisers, so neither increases L_beta.  This is the
  exact form of "the objective is non-increasing" for ADMM.
* Sanity: reconstruction beats zero filling on the small workload.
"""
import numpy as np
import pytest

import synth
from oracle import admm
from oracle.transforms import ifft2c, fftc, ifftc
from oracle.metrics import ssos, rlne


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _tiny_cfg(model, weight, lam=50.0):
    return synth.Workload(name="tiny", model=model, J=2, M=6, N=6, window=3, weight=weight,
                          lam=lam, beta=3.0, tau=3.0)


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
@pytest.mark.parametrize("weight", [0, 1])
def test_x_update_pointwise_equals_dense(model, weight):
    rng = np.random.default_rng(4 + weight)
    cfg = _tiny_cfg(model, weight)
    J, M, N, p = cfg.J, cfg.M, cfg.N, cfg.window
    C = 2 * J if model == "SHLR_V" else J
    U = (rng.random((M, N)) < 0.5).astype(np.uint8)
    Y = _crandn(rng, J, M, N) * U[None]
    s = admm.Shlr2D(Y, U, cfg)
    Zr, Dr = _crandn(rng, M, N - p + 1, C * p), _crandn(rng, M, N - p + 1, C * p)
    Zc, Dc = _crandn(rng, N, M - p + 1, C * p), _crandn(rng, N, M - p + 1, C * p)
    K_fast = s.x_update(Zr, Zc, Dr, Dc)
    b = cfg.beta
    K_dense = admm.dense_x_update_2d(Y, U, Zr - Dr / b, Zc - Dc / b, cfg)
    np.testing.assert_allclose(K_fast, K_dense, atol=1e-10 * np.abs(K_dense).max())


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_x_update_param_pointwise_equals_dense(model):
    rng = np.random.default_rng(9)
    cfg = synth.Workload(name="tinyp", model=model, J=1, M=2, N=6, L=4, window=3, window_param=2,
                         weight=1, lam=40.0, lam2=2.0, beta=2.0, tau=2.0)
    L, J, M, N, p, pP = cfg.L, cfg.J, cfg.M, cfg.N, cfg.window, cfg.window_param
    C = 2 * J if model == "SHLR_VP" else J
    U = np.zeros((L, M, N), np.uint8)
    for l in range(L):
        U[l][:, rng.random(N) < 0.5] = 1
    Y = _crandn(rng, L, J, M, N) * U[:, None]
    s = admm.ShlrParam(Y, U, cfg)
    Zpe, Dpe = _crandn(rng, M * L, N - p + 1, C * p), _crandn(rng, M * L, N - p + 1, C * p)
    Zp, Dp = _crandn(rng, M * N, L - pP + 1, J * pP), _crandn(rng, M * N, L - pP + 1, J * pP)
    K_fast = s.x_update(Zpe, Zp, Dpe, Dp)
    b = cfg.beta
    K_dense = admm.dense_x_update_param(Y, U, Zpe - Dpe / b, Zp - Dp / b, cfg)
    np.testing.assert_allclose(K_fast, K_dense, atol=1e-10 * np.abs(K_dense).max())


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_full_sampling_hard_dc_fixed_point(model):
    cfg = synth.get_config("shlr_4c_64").with_(model=model, mask="full", lam=0.0, J=2, M=32, N=32)
    inp = synth.make_inputs(cfg)
    s = admm.Shlr2D(inp["Y"], inp["mask"], cfg)
    st = s.init_state()
    for _ in range(3):
        st, rel = s.step(st)
        np.testing.assert_array_equal(st["K"], inp["Y"])
        assert rel == 0.0


def test_parameter_full_sampling_hard_dc_fixed_point():
    cfg = synth.get_config("shlrvp_8c_192_8e").with_(mask="full", lam=0.0, J=2, M=4, N=24, L=6, window=5)
    inp = synth.make_inputs(cfg)
    s = admm.ShlrParam(inp["Y"], inp["mask"], cfg)
    st = s.init_state()
    act = np.ones(cfg.M, bool)
    for _ in range(2):
        st, rel = s.step(st, act)
        np.testing.assert_array_equal(st["K"], inp["Y"])


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_homogeneity(model):
    cfg = synth.get_config("shlr_4c_64").with_(model=model, J=2, M=24, N=24, window=5)
    inp = synth.make_inputs(cfg)
    c = 7.5
    _, K1, _ = admm.shlr(inp["Y"], inp["mask"], cfg, n_iter=4)
    cfg2 = cfg.with_(lam=cfg.lam / c, beta=cfg.beta / c, tau=cfg.tau / c)
    _, K2, _ = admm.shlr(c * inp["Y"], inp["mask"], cfg2, n_iter=4)
    np.testing.assert_allclose(K2, c * K1, atol=1e-10 * np.abs(c * K1).max())


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_augmented_lagrangian_blockwise_descent(model):
    cfg = synth.get_config("shlr_4c_64").with_(model=model, J=2, M=24, N=24, window=5, d_init=0.0)
    inp = synth.make_inputs(cfg)
    s = admm.Shlr2D(inp["Y"], inp["mask"], cfg)
    st = s.init_state()
    for _ in range(6):
        L0 = s.lagrangian(st["K"], st["Zr"], st["Zc"], st["Dr"], st["Dc"])
        K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"])
        L1 = s.lagrangian(K, st["Zr"], st["Zc"], st["Dr"], st["Dc"])
        LXr, LXc = s.lifts(K)
        Zr, Zc = s.z_update(LXr, LXc, st["Dr"], st["Dc"])
        L2 = s.lagrangian(K, Zr, Zc, st["Dr"], st["Dc"])
        assert L1 <= L0 + 1e-9 * abs(L0)
        assert L2 <= L1 + 1e-9 * abs(L1)
        Dr, Dc = s.d_update(LXr, LXc, Zr, Zc, st["Dr"], st["Dc"])
        st = dict(K=K, Zr=Zr, Zc=Zc, Dr=Dr, Dc=Dc)


def test_x_step_is_minimiser_against_perturbations():
    cfg = synth.get_config("shlr_4c_64").with_(model="SHLR_V", J=2, M=16, N=16, window=4)
    inp = synth.make_inputs(cfg)
    s = admm.Shlr2D(inp["Y"], inp["mask"], cfg)
    rng = np.random.default_rng(5)
    st = s.init_state()
    st, _ = s.step(st)
    K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"])
    f0 = s.lagrangian(K, st["Zr"], st["Zc"], st["Dr"], st["Dc"])
    for _ in range(20):
        dK = 1e-3 * _crandn(rng, *K.shape)
        assert s.lagrangian(K + dK, st["Zr"], st["Zc"], st["Dr"], st["Dc"]) >= f0 - 1e-9 * abs(f0)


def test_reconstruction_beats_zero_filling():
    cfg = synth.get_config("shlr_4c_64")
    inp = synth.make_inputs(cfg)
    X, K, rels = admm.shlr(inp["Y"], inp["mask"], cfg, n_iter=30)
    zf = rlne(ssos(inp["truth"]), ssos(ifft2c(inp["Y"])))
    rec = rlne(ssos(inp["truth"]), ssos(X))
    assert rec < 0.8 * zf
    assert len(rels) == 30


def test_stopping_rule_stops_early():
    cfg = synth.get_config("shlr_4c_64").with_(J=2, M=24, N=24, window=5)
    inp = synth.make_inputs(cfg)
    s = admm.Shlr2D(inp["Y"], inp["mask"], cfg)
    st, rels = s.run(50, tol=1e-6)
    assert rels[-1] < 1e-6 and all(r >= 1e-6 for r in rels[:-1])
    assert len(rels) < 50
