"""Pins of oracle/spirit.py and of the SHLR-S / SHLR-SV X-update (Eq. 3, 6, 15).

* Calibration recovers an exact linear relation between coils: with
  coil 2 = c * coil 1 (coil 1 random) the only exact kernel is g[0,1,0,0] =
  1/c, g[1,0,0,0] = c (offsets (0, 0)), and a tiny Tikhonov weight returns it.
* The circular k-space correlation G is pixelwise in the image domain, with
  the per-pixel J x J weights sqrt(M N) F2D(kernel placed at the k-space
  centre + offset) (the image-domain SPIRiT operator of Eq. 3).
* apply_gh is the adjoint of apply_g.
* The CG X-update equals the dense normal-equation solve built from the
  literal image-domain operators with the lambda_1 ||(G - I) X||^2 term
  (SHLR-S and SHLR-SV, W on and off).
* Blockwise descent of the augmented Lagrangian with the SPIRiT term.
"""
import numpy as np
import pytest

import synth
from oracle import admm, spirit
from oracle.transforms import fftc, ifftc


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_calibration_recovers_exact_coil_relation():
    rng = np.random.default_rng(1)
    M, N, c = 16, 20, 0.7 - 0.4j
    x1 = _crandn(rng, M, N)
    Y = np.stack([x1, c * x1])
    g = spirit.calibrate(Y, n_acs=10, ksize=3, reg=1e-8)
    ref = np.zeros_like(g)
    ref[0, 1, 1, 1] = 1.0 / c
    ref[1, 0, 1, 1] = c
    np.testing.assert_allclose(g, ref, atol=1e-6)


def test_correlation_is_pixelwise_in_image_domain():
    rng = np.random.default_rng(2)
    J, M, N, ks = 3, 12, 10, 5
    h = ks // 2
    g = _crandn(rng, J, J, ks, ks)
    K = _crandn(rng, J, M, N)
    ifft2 = lambda x: ifftc(ifftc(x, axis=-1), axis=-2)
    W = np.zeros((J, J, M, N), dtype=complex)
    for a in range(ks):
        for b in range(ks):
            W[:, :, M // 2 + a - h, N // 2 + b - h] = g[:, :, a, b]
    Gimg = np.sqrt(M * N) * fftc(fftc(W, axis=-1), axis=-2)
    out = np.einsum("jkmn,kmn->jmn", Gimg, ifft2(K))
    np.testing.assert_allclose(out, ifft2(spirit.apply_g(K, g)), atol=1e-12 * np.abs(out).max())


def test_gh_is_adjoint():
    rng = np.random.default_rng(3)
    g = _crandn(rng, 2, 2, 5, 5)
    x, y = _crandn(rng, 2, 8, 9), _crandn(rng, 2, 8, 9)
    lhs = np.vdot(spirit.apply_g(x, g), y)
    rhs = np.vdot(x, spirit.apply_gh(y, g))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _tiny(model, weight):
    return synth.Workload(name="tiny", model=model, J=2, M=6, N=6, window=3, weight=weight, lam=50.0, beta=3.0,
                          tau=3.0, lam1=7.0, spirit_k=3, spirit_reg=1e-3, n_acs=4)


@pytest.mark.parametrize("model", ["SHLR_S", "SHLR_SV"])
@pytest.mark.parametrize("weight", [0, 1])
def test_cg_x_update_equals_dense_solve(model, weight):
    rng = np.random.default_rng(4 + weight)
    cfg = _tiny(model, weight)
    J, M, N, p = cfg.J, cfg.M, cfg.N, cfg.window
    C = 2 * J if model == "SHLR_SV" else J
    U = (rng.random((M, N)) < 0.5).astype(np.uint8)
    U[1:5] = 1
    Y = _crandn(rng, J, M, N) * U[None]
    s = admm.Shlr2D(Y, U, cfg)
    Zr, Dr = _crandn(rng, M, N - p + 1, C * p), _crandn(rng, M, N - p + 1, C * p)
    Zc, Dc = _crandn(rng, N, M - p + 1, C * p), _crandn(rng, N, M - p + 1, C * p)
    K_cg = s.x_update(Zr, Zc, Dr, Dc, K0=_crandn(rng, J, M, N))
    b = cfg.beta
    K_dense = admm.dense_x_update_2d(Y, U, Zr - Dr / b, Zc - Dc / b, cfg, g=s.g)
    np.testing.assert_allclose(K_cg, K_dense, atol=1e-9 * np.abs(K_dense).max())


@pytest.mark.parametrize("model", ["SHLR_S", "SHLR_SV"])
def test_spirit_lagrangian_blockwise_descent(model):
    cfg = synth.get_config("shlr_4c_64").with_(model=model, J=2, M=24, N=24, window=5, d_init=0.0,
                                                mask="random1d", R=3.0, n_acs=8, lam1=20.0, spirit_k=3)
    inp = synth.make_inputs(cfg)
    s = admm.Shlr2D(inp["Y"], inp["mask"], cfg)
    st = s.init_state()
    for _ in range(4):
        L0 = s.lagrangian(st["K"], st["Zr"], st["Zc"], st["Dr"], st["Dc"])
        K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"], K0=st["K"])
        L1 = s.lagrangian(K, st["Zr"], st["Zc"], st["Dr"], st["Dc"])
        LXr, LXc = s.lifts(K)
        Zr, Zc = s.z_update(LXr, LXc, st["Dr"], st["Dc"])
        L2 = s.lagrangian(K, Zr, Zc, st["Dr"], st["Dc"])
        assert L1 <= L0 + 1e-9 * abs(L0)
        assert L2 <= L1 + 1e-9 * abs(L1)
        Dr, Dc = s.d_update(LXr, LXc, Zr, Zc, st["Dr"], st["Dc"])
        st = dict(K=K, Zr=Zr, Zc=Zc, Dr=Dr, Dc=Dc)
