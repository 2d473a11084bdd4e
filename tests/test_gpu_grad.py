"""GPU reverse mode: SVT VJP, X-update VJP and the unrolled reconstruction.

The CUDA results are compared with the FP64 oracle's reverse pass
(``oracle.svt.svt_vjp``: Hermitian dilation + Daleckii-Krein;
``oracle.unrolled.unrolled_2d_vjp``), which is itself pinned to central
finite differences on the CPU, and in one case directly with central
differences of the FP64 oracle forward.

Tolerances.  The GPU SVT VJP takes its eigenpairs from FP32 one-sided Jacobi
on [B; I] (rotation tolerance 2e-6) plus one Newton-Schulz step, which leaves
the eigenvector matrix orthonormal to ~u sqrt(s) (5e-7 at s = 192; without
the step the O(u) non-unitarity of each of ~10 s rotations per column added
up to 4e-5 and the VJP error to 1.2e-4), then forms ~10 batched FP32 products
of length <= len + s, each adding ~u sqrt(len) relative error.  With the
threshold kept half a singular-value gap away from every sigma, the measured
relative errors are <= 5.2e-6 (Abar) and <= 1.1e-5 (tbar) on these cases:
the bounds 2e-5 / 5e-5 keep a factor 4 above them.
The unrolled gradients go through 4 iterations of FP32 lift / SVT / adjoint /
transforms; they are compared relative to the largest component of each
gradient vector (2e-3) because tau_k's cotangents span three decades.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from synth.configs import get_config
from oracle import svt as osvt
from oracle import unrolled as ounr
from oracle import admm as oadmm
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11650_gb300 import build
    build()


def _api():
    from paper_2107_11650_gb300 import api
    return api


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def _spectrum_matrix(rng, m, n, decay):
    """A = U diag(sigma) V^H with sigma_i = decay^i (well separated)."""
    k = min(m, n)
    U, _ = np.linalg.qr(_crandn(rng, m, k))
    V, _ = np.linalg.qr(_crandn(rng, n, k))
    s = decay ** np.arange(k)
    return (U * s) @ V.conj().T, s


SVT_CASES = [(3, 9, 6, 0.8), (2, 6, 9, 0.8), (4, 21, 8, 0.85), (2, 57, 32, 0.93), (1, 241, 192, 0.985),
             (2, 113, 128, 0.97)]


@pytest.mark.parametrize("svd", ["eig", "jacobi"])
@pytest.mark.parametrize("nmat,rows,cols,decay", SVT_CASES)
def test_svt_vjp_matches_oracle(nmat, rows, cols, decay, svd):
    api = _api()
    rng = np.random.default_rng(rows * 31 + cols)
    As, Zbs, ts = [], [], []
    for _ in range(nmat):
        A, s = _spectrum_matrix(rng, rows, cols, decay)
        As.append(A)
        Zbs.append(_crandn(rng, rows, cols))
    # one threshold for the batch, midway between two singular values of the first matrix
    s = np.linalg.svd(As[0], compute_uv=False)
    r = max(1, len(s) // 3)
    t = 0.5 * (s[r - 1] + s[r])
    A = np.stack(As)
    Zb = np.stack(Zbs)
    ref_Ab = np.empty_like(A)
    ref_tb = 0.0
    for i in range(nmat):
        ref_Ab[i], tb = osvt.svt_vjp(A[i], Zb[i], t)
        ref_tb += tb
    plan = api.Plan(api.Desc(model="SHLR", J=12, M=256, N=256, window=16, svd=svd))
    dA, dZb = _dev(A), _dev(Zb)
    dAb = torch.empty_like(dA)
    dZ = torch.empty_like(dA)
    dtb = torch.zeros(1, dtype=torch.float32, device="cuda")
    api.selr_svt_vjp(plan, dA, dZb, t, dAb, dtb, Z_out=dZ)
    assert api.selr_sync_status(plan) == 0
    err = rel_l2(_host(dAb), ref_Ab)
    assert err <= 2e-5, err
    assert rel_l2(_host(dZ), osvt.svt(A, t)) <= 1e-5
    tb = float(dtb.cpu())
    assert abs(tb - ref_tb) <= 5e-5 * max(1.0, abs(ref_tb)), (tb, ref_tb)
    plan.close()


def test_svt_vjp_rejects_bad_arguments():
    api = _api()
    plan = api.Plan(api.Desc(model="SHLR", J=2, M=16, N=16, window=4))
    A = torch.zeros((1, 13, 8), dtype=torch.complex64, device="cuda")
    tb = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(api._lib.SelrError):
        api.selr_svt_vjp(plan, A, A.clone(), -1.0, torch.empty_like(A), tb)
    big = torch.zeros((64, 13, 8), dtype=torch.complex64, device="cuda")   # above the plan's capacity
    with pytest.raises(api._lib.SelrError):
        api.selr_svt_vjp(plan, big, big.clone(), 0.1, torch.empty_like(big), tb)
    plan.close()


@pytest.mark.parametrize("lam", [1e4, -1.0])
def test_dc_vjp_is_adjoint_of_x_update(lam):
    """With Y = 0 the X-update is linear in (a, b) and in Y: check
    Re<K(a, b), Kbar> = Re<a, F_m* Sbar> + Re<b, F_n* Sbar> and
    Re<K(Y), Kbar> = Re<Y, Ybar>."""
    api = _api()
    J, M, N = 3, 24, 20
    desc = api.Desc(model="SHLR", J=J, M=M, N=N, window=5, lam=lam)
    plan = api.Plan(desc)
    rng = np.random.default_rng(9)
    mask = synth.mask_1d_random(M, N, 3.0, 4, np.random.default_rng(1))
    dmask = torch.from_numpy(mask).cuda()
    a, b, Kb, Y = (_crandn(rng, J, M, N) for _ in range(4))
    # K(a, b) with Y = 0
    da, db = _dev(a), _dev(b)
    K = torch.zeros((J, M, N), dtype=torch.complex64, device="cuda")
    api.selr_dc(plan, torch.zeros_like(K), dmask, da, db, K)
    Sb = torch.empty_like(K)
    Yb = torch.empty_like(K)
    api.selr_dc_vjp(plan, dmask, _dev(Kb), Sb, Yb)
    ar, ac = torch.empty_like(K), torch.empty_like(K)
    api.selr_transform(plan, 0, True, Sb, ar)
    api.selr_transform(plan, 1, True, Sb, ac)
    lhs = np.real(np.vdot(Kb, _host(K)))
    rhs = np.real(np.vdot(a, _host(ar))) + np.real(np.vdot(b, _host(ac)))
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(np.abs(Kb) ** 2) * np.sum(np.abs(a) ** 2 + np.abs(b) ** 2))
    # K(Y) with a = b = 0
    K2 = torch.zeros_like(K)
    api.selr_dc(plan, _dev(Y), dmask, torch.zeros_like(K), torch.zeros_like(K), K2)
    lhs = np.real(np.vdot(Kb, _host(K2)))
    rhs = np.real(np.vdot(Y, _host(Yb)))
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(np.abs(Kb) ** 2) * np.sum(np.abs(Y) ** 2))
    plan.close()


def _unrolled_case(model, lam):
    cfg = get_config("shlr_4c_64").with_(model=model, window=4, lam=lam, mask="random1d", R=3.0, n_acs=4)
    inp = synth.make_inputs(cfg, small=(2, 16, 12))
    return cfg, inp["Y"], inp["mask"]


def _engine(cfg, mask, n):
    from paper_2107_11650_gb300.unrolled import UnrolledSHLR
    api = _api()
    desc = api.Desc.from_workload(cfg.with_(J=2, M=mask.shape[0], N=mask.shape[1]))
    return UnrolledSHLR(desc, torch.from_numpy(mask).cuda(), n)


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_unrolled_forward_matches_solve_and_oracle(model):
    api = _api()
    cfg, Y, U = _unrolled_case(model, 1e4)
    n = 4
    net = _engine(cfg, U, n)
    dY = _dev(Y)
    with torch.no_grad():
        X = net(dY)
    # constant parameters: the plan's own solver
    desc = api.Desc.from_workload(cfg.with_(J=2, M=16, N=12), max_iter=n)
    plan = api.Plan(desc)
    Xs = torch.empty_like(dY)
    api.selr_solve(plan, dY, torch.from_numpy(U).cuda(), Xs)
    assert rel_l2(_host(X), _host(Xs)) <= 1e-5
    ref = oadmm.shlr(Y, U, cfg.with_(n_iter=n))[0]
    assert rel_l2(_host(X), ref) <= 1e-4
    # varying parameters against the oracle's unrolled forward
    ts = (1.0 / cfg.beta) * (1.0 + 0.1 * np.arange(n))
    taus = cfg.tau * (1.0 - 0.05 * np.arange(n))
    with torch.no_grad():
        net.ts.copy_(torch.tensor(ts))
        net.taus.copy_(torch.tensor(taus))
        X2 = net(dY)
    ref2 = ounr.unrolled_2d(Y, U, cfg, ts, taus)
    assert rel_l2(_host(X2), ref2) <= 1e-4
    plan.close()


@pytest.mark.parametrize("model,lam", [("SHLR", 1e4), ("SHLR_V", 1e4), ("SHLR", -1.0)])
def test_unrolled_gradient_matches_fp64_reference(model, lam):
    cfg, Y, U = _unrolled_case(model, lam)
    n = 4
    ts = (1.0 / cfg.beta) * (1.0 + 0.1 * np.arange(n))
    taus = cfg.tau * (1.0 - 0.05 * np.arange(n))
    rng = np.random.default_rng(3)
    Xb = _crandn(rng, *Y.shape)
    ref_t, ref_tau, ref_Y = ounr.unrolled_2d_vjp(Y, U, cfg, ts, taus, Xb)
    net = _engine(cfg, U, n)
    with torch.no_grad():
        net.ts.copy_(torch.tensor(ts))
        net.taus.copy_(torch.tensor(taus))
    dY = _dev(Y).requires_grad_(True)
    X = net(dY)
    loss = (_dev(Xb).conj() * X).real.sum()
    loss.backward()
    g_t = net.ts.grad.cpu().numpy().astype(np.float64)
    g_tau = net.taus.grad.cpu().numpy().astype(np.float64)
    assert np.abs(g_t - ref_t).max() <= 2e-3 * np.abs(ref_t).max(), (g_t, ref_t)
    assert np.abs(g_tau - ref_tau).max() <= 2e-3 * np.abs(ref_tau).max(), (g_tau, ref_tau)
    assert rel_l2(_host(dY.grad), ref_Y) <= 2e-3
    # and directly against central differences of the FP64 forward in t_0, tau_0
    h = 1e-6

    def L(ts_, taus_):
        return np.real(np.vdot(Xb, ounr.unrolled_2d(Y, U, cfg, ts_, taus_)))

    e = np.zeros(n)
    e[0] = h
    fd_t = (L(ts + e, taus) - L(ts - e, taus)) / (2 * h)
    assert abs(g_t[0] - fd_t) <= 2e-3 * np.abs(ref_t).max()
    e[0] = h * taus[0]
    fd_tau = (L(ts, taus + e) - L(ts, taus - e)) / (2 * h * taus[0])
    assert abs(g_tau[0] - fd_tau) <= 2e-3 * np.abs(ref_tau).max()


def test_unrolled_keeps_only_k_and_d_per_iteration():
    """Checkpoints hold (K_k, D_row, D_col) per iteration and nothing else."""
    cfg, Y, U = _unrolled_case("SHLR", 1e4)
    net = _engine(cfg, U, 3)
    X, ckpts = net.engine.forward(_dev(Y), net.ts, net.taus)
    assert len(ckpts) == 3
    for K, D in ckpts:
        assert K.shape == Y.shape and set(D) == {"row", "col"}


def test_unrolled_batch_sums_instance_gradients():
    """Two instances of different sizes sharing t_k, tau_k: the gradients are
    the sums of the instances' FP64 reference gradients.  The batched forward
    (one plan for both instances) rounds differently from the per-instance
    forward (states differ by ~1e-6 after two iterations), and on this case the
    threshold and step gradients of the first iteration move by 2.6e-3
    relative under such a state change (close singular values make the
    gradient's own derivative large; no singular value is within 1e-3 of a
    threshold), so an FP32 forward cannot place them closer to the FP64 values
    than that: bound 5e-3.  The batched gradients also equal, to rounding, the
    per-instance reverse passes run from the batched checkpoints."""
    from paper_2107_11650_gb300.unrolled import UnrolledBatch
    api = _api()
    n = 3
    base = get_config("shlr_4c_64").with_(window=4, mask="random1d", R=3.0, n_acs=4)
    cases = [(base, (2, 16, 12)), (base.with_(model="SHLR", seed=7), (3, 20, 24))]
    rng = np.random.default_rng(21)
    ref_t = np.zeros(n)
    ref_tau = np.zeros(n)
    descs, masks, Ys, Xbs = [], [], [], []
    ts = (1.0 / base.beta) * (1.0 + 0.05 * np.arange(n))
    taus = base.tau * np.ones(n)
    for cfg, small in cases:
        inp = synth.make_inputs(cfg, small=small)
        c = cfg.with_(J=small[0], M=small[1], N=small[2])
        Xb = _crandn(rng, *inp["Y"].shape)
        t_, tau_, _ = ounr.unrolled_2d_vjp(inp["Y"], inp["mask"], c, ts, taus, Xb)
        ref_t += t_
        ref_tau += tau_
        descs.append(api.Desc.from_workload(c))
        masks.append(torch.from_numpy(inp["mask"]).cuda())
        Ys.append(_dev(inp["Y"]))
        Xbs.append(_dev(Xb))
    net = UnrolledBatch(descs, masks, n)
    with torch.no_grad():
        net.ts.copy_(torch.tensor(ts))
        net.taus.copy_(torch.tensor(taus))
    Xs = net(Ys)
    loss = sum((xb.conj() * x).real.sum() for xb, x in zip(Xbs, Xs))
    loss.backward()
    g_t = net.ts.grad.cpu().numpy().astype(np.float64)
    g_tau = net.taus.grad.cpu().numpy().astype(np.float64)
    assert np.abs(g_t - ref_t).max() <= 5e-3 * np.abs(ref_t).max(), (g_t, ref_t)
    assert np.abs(g_tau - ref_tau).max() <= 5e-3 * np.abs(ref_tau).max(), (g_tau, ref_tau)
    # the same reverse pass, instance by instance, from the batched checkpoints
    from paper_2107_11650_gb300.unrolled import _BatchCheckpoints
    bp = net.bplan
    Yp = bp.pack(Ys, torch.complex64)
    Xp = torch.empty_like(Yp)
    ckK = torch.empty((n, bp.nK), dtype=torch.complex64, device="cuda")
    ckD = torch.empty((n, api.selr_lifted_elems(bp)), dtype=torch.complex64, device="cuda")
    api.selr_solve_unrolled(bp, Yp, net.mask_p, Xp, list(ts), list(taus), ckK, ckD)
    tsum = np.zeros(n)
    for i, e in enumerate(net.engines):
        _, tb, _ = e.backward(_BatchCheckpoints(bp, ckK, ckD, i, e), Ys[i], torch.tensor(ts), torch.tensor(taus),
                              Xbs[i])
        tsum += tb.cpu().numpy()
    assert np.abs(g_t - tsum).max() <= 1e-5 * np.abs(tsum).max(), (g_t, tsum)


def test_unrolled_forward_full_size_instance_matches_stored_oracle():
    """The differentiable forward (per-op calls of UnrolledSHLR, t_k = 1/beta,
    tau_k = tau, which is Algorithm S1) on the largest instance of the unrolled
    batch (24 coils, 320x320, window 16, 24 ACS lines: lifted 305 x 384, order
    305), 10 iterations, against FP64 oracle values stored by
    tests/golden/make_golden.py."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "unrolled_11_10it.npz")
    if not os.path.exists(path):
        pytest.skip("no stored oracle values for unrolled_11")
    from paper_2107_11650_gb300 import api
    from paper_2107_11650_gb300.unrolled import UnrolledSHLR
    g = np.load(path)
    wl = synth.unrolled_instance("unrolled_11")
    inp = synth.make_inputs(wl)
    net = UnrolledSHLR(api.Desc.from_workload(wl, gram="3xtf32"), torch.from_numpy(inp["mask"]).cuda(), wl.n_iter)
    with torch.no_grad():
        X = net(torch.from_numpy(inp["Y"].astype(np.complex64)).cuda())
    assert api.selr_sync_status(net.engine.plan) == 0
    xs = X.cpu().numpy().astype(np.complex128).ravel()[g["idx"]]
    assert np.linalg.norm(xs - g["values"]) / np.linalg.norm(g["values"]) < 1e-4


def test_unrolled_batch_forward_is_one_batched_graph():
    """The batched forward (selr_solve_unrolled on one batched plan, one CUDA
    graph per call) with varying t_k, tau_k equals each instance's per-op
    forward and the oracle's unrolled forward; a second call with other
    parameters updates the graph and is right too."""
    from paper_2107_11650_gb300.unrolled import UnrolledBatch, Unrolled2D
    api = _api()
    n = 4
    base = get_config("shlr_4c_64").with_(window=4, mask="random1d", R=3.0, n_acs=4)
    cases = [(base, (2, 16, 12)), (base.with_(seed=7), (3, 20, 24)), (base.with_(seed=9), (2, 24, 24))]
    descs, masks, Ys, inps = [], [], [], []
    for cfg, small in cases:
        inp = synth.make_inputs(cfg, small=small)
        c = cfg.with_(J=small[0], M=small[1], N=small[2])
        inps.append((c, inp))
        descs.append(api.Desc.from_workload(c))
        masks.append(torch.from_numpy(inp["mask"]).cuda())
        Ys.append(_dev(inp["Y"]))
    net = UnrolledBatch(descs, masks, n)
    for trial in range(2):
        ts = (1.0 / base.beta) * (1.0 + 0.1 * np.arange(n) + 0.05 * trial)
        taus = base.tau * (1.0 - 0.05 * np.arange(n) - 0.02 * trial)
        with torch.no_grad():
            net.ts.copy_(torch.tensor(ts))
            net.taus.copy_(torch.tensor(taus))
            Xs = net(Ys)
        for (c, inp), X, e in zip(inps, Xs, net.engines):
            Xe, _ = e.forward(_dev(inp["Y"]), torch.tensor(ts), torch.tensor(taus))
            assert rel_l2(_host(X), _host(Xe)) <= 1e-5
            ref = ounr.unrolled_2d(inp["Y"], inp["mask"], c, ts, taus)
            assert rel_l2(_host(X), ref) <= 1e-4
