"""Batched plans of uneven instances (selr_plan_create_batch).

Each instance of a batch must reconstruct exactly what a plan of its own
computes: the arithmetic per matrix is the same, only the launch that
carries it differs (instances of one SVT size class share the tridiagonal
template of the largest order in the class, which changes the rounding
order), so the comparison with the single-instance plans uses 1e-5 and the
comparison with the FP64 oracle the parity bound 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from synth.configs import get_config
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


def _instances(model):
    base = get_config("shlr_4c_64").with_(model=model, mask="random1d", R=3.0, n_acs=4)
    sizes = [(2, 24, 24, 4), (3, 32, 40, 5), (4, 48, 48, 8), (2, 20, 30, 3)]
    out = []
    for i, (J, M, N, p) in enumerate(sizes):
        cfg = base.with_(J=J, M=M, N=N, window=p, seed=11 + i, lam=1e4 if i % 2 == 0 else 5e3)
        inp = synth.make_inputs(cfg)
        out.append((cfg, inp["Y"], inp["mask"]))
    return out


@pytest.mark.parametrize("model,svd", [("SHLR", "eig"), ("SHLR_V", "eig"), ("SHLR", "jacobi")])
def test_batch_matches_single_plans_and_oracle(model, svd):
    api = _api()
    n_iter = 8
    inst = _instances(model)
    descs = [api.Desc.from_workload(c, max_iter=n_iter, svd=svd) for c, _, _ in inst]
    plan = api.BatchPlan(descs)
    Yp = plan.pack([torch.from_numpy(Y.astype(np.complex64)).cuda() for _, Y, _ in inst], torch.complex64)
    mp = plan.pack([torch.from_numpy(m).cuda() for _, _, m in inst], torch.uint8, mask=True)
    Xp = torch.empty_like(Yp)
    it, rel = api.selr_solve_batch(plan, Yp, mp, Xp)
    assert it == n_iter
    assert api.selr_sync_status(plan) == 0
    for i, (cfg, Y, m) in enumerate(inst):
        single = api.Plan(descs[i])
        Yd = torch.from_numpy(Y.astype(np.complex64)).cuda()
        Xs = torch.empty_like(Yd)
        api.selr_solve(single, Yd, torch.from_numpy(m).cuda(), Xs)
        xb = plan.unpack(Xp, i).cpu().numpy().astype(np.complex128)
        assert rel_l2(xb, Xs.cpu().numpy().astype(np.complex128)) <= 1e-5
        ref = oadmm.shlr(Y, m, cfg, n_iter=n_iter)[0]
        assert rel_l2(xb, ref) <= 1e-4
        single.close()
    plan.close()


def test_batch_stops_when_every_instance_converges():
    api = _api()
    inst = _instances("SHLR")
    tol = 1e-4
    descs = [api.Desc.from_workload(c, max_iter=60, tol=tol) for c, _, _ in inst]
    plan = api.BatchPlan(descs)
    Yp = plan.pack([torch.from_numpy(Y.astype(np.complex64)).cuda() for _, Y, _ in inst], torch.complex64)
    mp = plan.pack([torch.from_numpy(m).cuda() for _, _, m in inst], torch.uint8, mask=True)
    Xp = torch.empty_like(Yp)
    it, rel = api.selr_solve_batch(plan, Yp, mp, Xp)
    singles = []
    for i, (c, Y, m) in enumerate(inst):
        sp = api.Plan(descs[i])
        Yd = torch.from_numpy(Y.astype(np.complex64)).cuda()
        si, _ = api.selr_solve(sp, Yd, torch.from_numpy(m).cuda(), torch.empty_like(Yd))
        singles.append(si)
        sp.close()
    assert it == max(singles)
    assert rel < tol or it == 60
    plan.close()


def test_batch_rejects_single_operator_calls():
    api = _api()
    inst = _instances("SHLR")
    plan = api.BatchPlan([api.Desc.from_workload(c) for c, _, _ in inst[:2]])
    with pytest.raises(api._lib.SelrError):
        plan.lift_shape("row")
    plan.close()


def _param_instances(model):
    base = get_config("shlrvp_8c_192_8e").with_(model=model)
    sizes = [(2, 6, 48, 8, 8, 4), (1, 4, 40, 6, 6, 3), (3, 5, 36, 8, 7, 4)]     # J, M, N, L, p, p_P
    out = []
    for i, (J, M, N, L, p, pP) in enumerate(sizes):
        cfg = base.with_(J=J, M=M, N=N, L=L, window=p, window_param=pP, seed=61 + i,
                         lam2=2.0 if i != 1 else 1.5)
        d = synth.make_inputs(cfg)
        out.append((cfg, d["Y"], d["mask"]))
    return out


@pytest.mark.parametrize("model,gram", [("SHLR_VP", "fp32"), ("SHLR_P", "3xtf32")])
def test_parameter_model_batch_matches_single_plans_and_oracle(model, gram):
    """Uneven SHLR-P / SHLR-VP instances (different coils, FE positions, PE
    lengths, echo counts, windows and lambda2) in one batched plan: the PE lifts
    of all instances share the eigensolver launches and the echo-vector lifts
    the warp-per-matrix SVT; each instance equals its own plan and the oracle
    (Algorithm S2)."""
    api = _api()
    n_iter = 8
    inst = _param_instances(model)
    descs = [api.Desc.from_workload(c, max_iter=n_iter, gram=gram) for c, _, _ in inst]
    plan = api.BatchPlan(descs)
    Yp = plan.pack([torch.from_numpy(Y.astype(np.complex64)).cuda() for _, Y, _ in inst], torch.complex64)
    mp = plan.pack([torch.from_numpy(m).cuda() for _, _, m in inst], torch.uint8, mask=True)
    Xp = torch.empty_like(Yp)
    it, _ = api.selr_solve_batch(plan, Yp, mp, Xp)
    assert it == n_iter and api.selr_sync_status(plan) == 0
    for i, (cfg, Y, m) in enumerate(inst):
        single = api.Plan(descs[i])
        Yd = torch.from_numpy(Y.astype(np.complex64)).cuda()
        Xs = torch.empty_like(Yd)
        api.selr_solve(single, Yd, torch.from_numpy(m).cuda(), Xs)
        xb = plan.unpack(Xp, i).cpu().numpy().astype(np.complex128)
        assert rel_l2(xb, Xs.cpu().numpy().astype(np.complex128)) <= 1e-5, i
        ref = oadmm.shlr_p(Y, m, cfg, n_iter=n_iter)[0]
        assert rel_l2(xb, ref) <= 1e-4, i
        single.close()
    plan.close()


def test_parameter_model_batch_per_position_stopping():
    """tol >= 0: every FE position of every instance stops on its own criterion;
    the batch runs as long as the slowest position, and each instance equals the
    oracle run with the same stopping rule."""
    api = _api()
    tol = 1e-4
    inst = _param_instances("SHLR_VP")
    descs = [api.Desc.from_workload(c, max_iter=40, tol=tol) for c, _, _ in inst]
    plan = api.BatchPlan(descs)
    Yp = plan.pack([torch.from_numpy(Y.astype(np.complex64)).cuda() for _, Y, _ in inst], torch.complex64)
    mp = plan.pack([torch.from_numpy(m).cuda() for _, _, m in inst], torch.uint8, mask=True)
    Xp = torch.empty_like(Yp)
    it, _ = api.selr_solve_batch(plan, Yp, mp, Xp)
    assert api.selr_sync_status(plan) == 0
    longest = 0
    for i, (cfg, Y, m) in enumerate(inst):
        Xo, _, iters = oadmm.shlr_p(Y, m, cfg, n_iter=40, tol=tol)
        longest = max(longest, int(iters.max()))
        xb = plan.unpack(Xp, i).cpu().numpy().astype(np.complex128)
        assert rel_l2(xb, Xo) < 1e-3, i
    assert abs(it - longest) <= 1
    plan.close()
