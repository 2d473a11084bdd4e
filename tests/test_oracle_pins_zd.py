"""Pins of the Z-step, the multiplier step, the per-FE-position freeze and
the objective of oracle/admm.py, against what the paper fixes.

Each check is written from the problem the paper states, not from the
oracle's own update formula:

* Z-step (Eqs. 11 and 16-17 for the 2D models; Eqs. S3-S4 and S8-S9 for the
  parameter models): the Z returned by the oracle minimises the augmented
  Lagrangian over Z (Eq. 9 / Eq. S1) with X and D fixed, tested against
  perturbations along Z itself, along each matrix's leading singular
  direction and along random directions.  The Lagrangian is written here from
  Eq. 9 / S1 with its own nuclear norm.  A planted mistake in the oracle's
  threshold (c / beta with c != 1, or the parameter-model thresholds 1/beta
  and lambda2/beta swapped) must be caught by the same check.
* Multiplier step (Eqs. 13-14 / S5-S6) with tau = beta: Z minimises
  g(Z) + beta/2 ||LX - Z + D/beta||^2 exactly when
  D + beta (LX - Z) lies in the subdifferential of g at Z, so the updated
  multiplier of every matrix has spectral norm <= w and Re<D+, Z> = w ||Z||_*,
  with w = 1 for row / column / PE lifts and w = lambda2 for the
  parameter-dimension lifts.  This fixes the sign and the scale of the
  multiplier update and which family carries lambda2.
* Algorithm S2: blockwise descent of the augmented Lagrangian of Eq. S1 and
  homogeneity (Y, lambda, beta, tau) -> (cY, lambda/c, beta/c, tau/c) with
  lambda2 unchanged (both thresholds then scale with c, so X -> cX).
* Per-FE-position stopping (Algorithm S2 runs each m on its own): in the
  batched oracle a position stops changing at its own stopping iteration,
  and every position equals a run of that position alone.
* Objective of Eq. 2 / Eq. 5 at a point where every lifted matrix is rank one
  with a singular value known in closed form.
"""
import numpy as np
import pytest

import synth
from oracle import admm, svt as osvt
from oracle.transforms import fftc


def _nuc(A):
    return float(np.linalg.svd(A, compute_uv=False).sum())


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _z_objective(families):
    """sum_f w_f sum ||Z_f||_* + beta/2 ||T_f - Z_f||^2 over families (w, Z, T, beta)."""
    def f(Zs):
        val = 0.0
        for (w, _, T, b), Z in zip(families, Zs):
            val += w * _nuc(Z) + 0.5 * b * float(np.sum(np.abs(T - Z) ** 2))
        return val
    return f


def _descent_directions(Zs, rng, n_random=6):
    """Perturbations of the stacked Z: +-Z, +-(u1 v1^H per matrix), random."""
    dirs = []
    for sgn in (1.0, -1.0):
        dirs.append([sgn * Z for Z in Zs])
        lead = []
        for Z in Zs:
            U, s, Vh = np.linalg.svd(Z, full_matrices=False)
            lead.append(sgn * U[..., :, :1] @ Vh[..., :1, :] * np.maximum(s[..., :1, None], 1e-3))
        dirs.append(lead)
    for _ in range(n_random):
        dirs.append([_crandn(rng, *Z.shape) * (np.abs(Z).mean() + 1e-3) for Z in Zs])
    return dirs


def _violations(f, Zs, rng, eps=1e-4):
    """Number of directions along which f decreases at Zs (0 at a minimiser)."""
    f0 = f(Zs)
    bad = 0
    for d in _descent_directions(Zs, rng):
        if f([Z + eps * dz for Z, dz in zip(Zs, d)]) < f0 - 1e-11 * abs(f0):
            bad += 1
    return bad


def _state_2d(model, iters=2):
    cfg = synth.get_config("shlr_4c_64").with_(model=model, J=2, M=16, N=16, window=4, beta=3.0, tau=3.0)
    inp = synth.make_inputs(cfg)
    s = admm.Shlr2D(inp["Y"], inp["mask"], cfg)
    st = s.init_state()
    for _ in range(iters):
        st, _ = s.step(st)
    return cfg, s, st


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_2d_z_step_minimises_augmented_lagrangian(model):
    """Eq. 11 solved by Eqs. 16-17: the oracle's Z minimises Eq. 9 over Z."""
    cfg, s, st = _state_2d(model)
    b = cfg.beta
    K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"])
    LXr, LXc = s.lifts(K)
    Zr, Zc = s.z_update(LXr, LXc, st["Dr"], st["Dc"])
    fam = [(1.0, None, LXr + st["Dr"] / b, b), (1.0, None, LXc + st["Dc"] / b, b)]
    f = _z_objective(fam)
    rng = np.random.default_rng(3)
    assert _violations(f, [Zr, Zc], rng) == 0
    # planted mistakes in the oracle's threshold (c / beta) are caught
    for c in (0.8, 1.25):
        Wr, Wc = osvt.svt(LXr + st["Dr"] / b, c / b), osvt.svt(LXc + st["Dc"] / b, c / b)
        assert _violations(f, [Wr, Wc], rng) > 0, c


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_2d_multiplier_is_nuclear_norm_subgradient(model):
    """Eqs. 13-14 with tau = beta: D+ in the subdifferential of ||.||_* at Z."""
    cfg, s, st = _state_2d(model)
    assert cfg.tau == cfg.beta
    new, _ = s.step(st)
    for Z, D in ((new["Zr"], new["Dr"]), (new["Zc"], new["Dc"])):
        for m in range(Z.shape[0]):
            assert np.linalg.norm(D[m], 2) <= 1.0 + 1e-9
            assert abs(np.real(np.vdot(D[m], Z[m])) - _nuc(Z[m])) <= 1e-9 * max(1.0, _nuc(Z[m]))


def _param_setup(model="SHLR_VP", lam2=0.4, beta=2.5):
    cfg = synth.get_config("shlrvp_8c_192_8e").with_(model=model, J=2, M=3, N=24, L=6, window=5,
                                                      window_param=3, lam2=lam2, beta=beta, tau=beta)
    inp = synth.make_inputs(cfg)
    return cfg, inp, admm.ShlrParam(inp["Y"], inp["mask"], cfg)


def _param_lagrangian(s, cfg, K, Zpe, Zp, Dpe, Dp):
    """Eq. S1 (scaled form, up to the constant -||D||^2 / (2 beta)): the PE lifts
    carry weight 1 (Eq. 7/8, sum over l), the echo-vector lifts weight lambda2
    (sum over n)."""
    b = cfg.beta
    LXpe, LXp = s.lifts(K)
    val = 0.5 * cfg.lam * float(np.sum(np.abs(s.U[:, None] * (s.Y - K)) ** 2)) if cfg.lam > 0 else 0.0
    val += sum(_nuc(z) for z in Zpe) + cfg.lam2 * sum(_nuc(z) for z in Zp)
    val += 0.5 * b * float(np.sum(np.abs(LXpe - Zpe + Dpe / b) ** 2))
    val += 0.5 * b * float(np.sum(np.abs(LXp - Zp + Dp / b) ** 2))
    return val


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_param_z_step_minimises_augmented_lagrangian(model):
    """Eqs. S3-S4 solved by S8-S9: thresholds 1/beta (PE lifts) and lambda2/beta
    (echo-vector lifts); swapping them, or scaling either, is caught."""
    cfg, inp, s = _param_setup(model)
    b = cfg.beta
    st = s.init_state()
    act = np.ones(cfg.M, bool)
    st, _ = s.step(st, act)
    new, _ = s.step(st, act)
    LXpe, LXp = s.lifts(new["K"])
    Tpe, Tp = LXpe + st["Dpe"] / b, LXp + st["Dp"] / b
    f = _z_objective([(1.0, None, Tpe, b), (cfg.lam2, None, Tp, b)])
    rng = np.random.default_rng(8)
    assert _violations(f, [new["Zpe"], new["Zp"]], rng) == 0
    swapped = [osvt.svt(Tpe, cfg.lam2 / b), osvt.svt(Tp, 1.0 / b)]
    assert _violations(f, swapped, rng) > 0
    for c in (0.8, 1.25):
        assert _violations(f, [new["Zpe"], osvt.svt(Tp, c * cfg.lam2 / b)], rng) > 0
        assert _violations(f, [osvt.svt(Tpe, c / b), new["Zp"]], rng) > 0


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_param_multipliers_are_weighted_subgradients(model):
    """Eqs. S5-S6 with tau = beta: D+ in w * d||.||_*(Z) with w = 1 (PE lifts)
    and w = lambda2 (echo-vector lifts)."""
    cfg, inp, s = _param_setup(model)
    st = s.init_state()
    act = np.ones(cfg.M, bool)
    st, _ = s.step(st, act)
    for w, Z, D in ((1.0, st["Zpe"], st["Dpe"]), (cfg.lam2, st["Zp"], st["Dp"])):
        for k in range(Z.shape[0]):
            assert np.linalg.norm(D[k], 2) <= w * (1.0 + 1e-9)
            assert abs(np.real(np.vdot(D[k], Z[k])) - w * _nuc(Z[k])) <= 1e-9 * max(1.0, _nuc(Z[k]))


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_param_augmented_lagrangian_blockwise_descent(model):
    cfg, inp, s = _param_setup(model)
    st = s.init_state()
    st = dict(st, Dpe=0 * st["Dpe"], Dp=0 * st["Dp"])
    act = np.ones(cfg.M, bool)
    for _ in range(5):
        L0 = _param_lagrangian(s, cfg, st["K"], st["Zpe"], st["Zp"], st["Dpe"], st["Dp"])
        new, _ = s.step(st, act)
        L1 = _param_lagrangian(s, cfg, new["K"], st["Zpe"], st["Zp"], st["Dpe"], st["Dp"])
        L2 = _param_lagrangian(s, cfg, new["K"], new["Zpe"], new["Zp"], st["Dpe"], st["Dp"])
        assert L1 <= L0 + 1e-9 * abs(L0)
        assert L2 <= L1 + 1e-9 * abs(L1)
        st = new


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_param_homogeneity_with_lambda2_fixed(model):
    cfg, inp, _ = _param_setup(model)
    c = 6.0
    _, K1, _ = admm.shlr_p(inp["Y"], inp["mask"], cfg, n_iter=4)
    cfg2 = cfg.with_(lam=cfg.lam / c, beta=cfg.beta / c, tau=cfg.tau / c)
    _, K2, _ = admm.shlr_p(c * inp["Y"], inp["mask"], cfg2, n_iter=4)
    np.testing.assert_allclose(K2, c * K1, atol=1e-10 * np.abs(c * K1).max())


def test_param_per_position_freeze_matches_single_position_runs():
    """Algorithm S2 solves each FE position m on its own with its own stopping
    test.  In the batched oracle, (a) position m's K and its lifts' Z, D stop
    changing at its own stopping iteration, and (b) every position equals a
    run of the single-position problem."""
    cfg, inp, s = _param_setup("SHLR_VP", lam2=2.0, beta=20.0)
    cfg = cfg.with_(M=4)
    inp = synth.make_inputs(cfg)
    s = admm.ShlrParam(inp["Y"], inp["mask"], cfg)
    tol, n_iter = 1e-4, 60
    st = s.init_state()
    active = np.ones(cfg.M, bool)
    iters = np.zeros(cfg.M, int)
    snaps = []
    for _ in range(n_iter):
        if not active.any():
            break
        st, rel = s.step(st, active)
        iters += active
        active = active & ~(rel < tol)
        snaps.append({k: v.copy() for k, v in st.items()})
    assert len(set(iters.tolist())) > 1, iters          # positions stop at different iterations
    L, N = cfg.L, cfg.N
    for m in range(cfg.M):
        k_m = iters[m]
        last = snaps[k_m - 1]
        for later in snaps[k_m:]:
            np.testing.assert_array_equal(later["K"][:, :, m], last["K"][:, :, m])
            for name, per in (("Zpe", L), ("Dpe", L), ("Zp", N), ("Dp", N)):
                np.testing.assert_array_equal(later[name][m * per:(m + 1) * per], last[name][m * per:(m + 1) * per])
        one = admm.ShlrParam(inp["Y"][:, :, m:m + 1], inp["mask"][:, m:m + 1], cfg.with_(M=1))
        st1, it1 = one.run(n_iter, tol)
        assert it1[0] == k_m
        np.testing.assert_allclose(st1["K"][:, :, 0], st["K"][:, :, m], rtol=0, atol=1e-12 * np.abs(st["K"]).max())


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_objective_closed_form_rank_one_lifts(model):
    """Eq. 2 / Eq. 5 at K[j, m, n] = a_j exp(2 pi i (k1 m / M + k2 n / N)), W = I:
    every row lift of the hybrid R = F_m* K and every column lift of
    C = F_n* K is rank one (unit-modulus exponential times coil weights).
    F_m* of an on-grid exponential is one spike of height sqrt(M), so one row
    lift has sigma = sqrt(M) ||a|| sqrt(l_r p) (times sqrt(2) with the virtual
    coils, whose conjugate-flipped exponential shares the row vector) and the
    others are zero; likewise for the columns.  The data term is lambda/2
    ||U (Y - K)||^2."""
    J, M, N, p = 3, 12, 10, 4
    cfg = synth.Workload(name="obj", model=model, J=J, M=M, N=N, window=p, weight=0, lam=7.0, beta=2.0, tau=2.0)
    rng = np.random.default_rng(2)
    a = _crandn(rng, J)
    k1, k2 = 3, 7
    mm, nn = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
    K = a[:, None, None] * np.exp(2j * np.pi * (k1 * mm / M + k2 * nn / N))[None]
    U = (rng.random((M, N)) < 0.5).astype(np.uint8)
    Y = U[None] * _crandn(rng, J, M, N)
    s = admm.Shlr2D(Y, U, cfg)
    vc = 2.0 if model == "SHLR_V" else 1.0
    na = np.linalg.norm(a)
    rows_term = np.sqrt(M) * na * np.sqrt(vc * (N - p + 1) * p)
    cols_term = np.sqrt(N) * na * np.sqrt(vc * (M - p + 1) * p)
    data = 0.5 * cfg.lam * np.sum(np.abs(U[None] * (Y - K)) ** 2)
    assert abs(s.objective(K) - (rows_term + cols_term + data)) <= 1e-9 * (rows_term + cols_term + data)
