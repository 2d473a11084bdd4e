"""Checkpoint / resume of selr_solve (state_inout) and the per-matrix rank sums.

* k1 iterations, a checkpoint (K, D, E = Z - D/beta, activity flags: the
  state between two passes of the loop body of Algorithm S1 / S2), then k2
  resumed iterations give bitwise the image of k1 + k2 iterations in one
  call: batched and plain, SHLR and SHLR-VP (with the per-position stopping
  rule, so the activity flags travel in the checkpoint), and a batched plan.
* After one iteration, the eigensolver's rank of every lifted matrix equals
  the number of singular values above t = 1/beta of the oracle's lifted
  matrices L(X) + D/beta (Eqs. 16-17), except at most a few matrices whose
  singular value lies within FP32 rounding of t.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from synth.configs import get_config
from oracle import admm as oadmm
from oracle.svt import svt_rank

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


def _run(api, plan, Y, m, n, state=None, resume=False):
    X = torch.empty_like(Y)
    s = torch.cuda.Stream()
    plan.set_iterations(n, plan.desc.tol)
    with torch.cuda.stream(s):
        it, _ = api.selr_solve(plan, Y, m, X, state=state, resume=resume, stream=s)
    assert api.selr_sync_status(plan, s) == 0
    return X.cpu(), it


@pytest.mark.parametrize("name,exec_mode,tol", [("shlr_4c_64", "batched", -1.0), ("shlr_4c_64", "plain", -1.0),
                                               ("shlrvp_8c_192_8e", "batched", 1e-4)])
def test_resume_is_bitwise_equal_to_one_run(name, exec_mode, tol):
    api = _api()
    wl = get_config(name)
    if wl.model == "SHLR_VP":
        wl = wl.with_(J=2, M=6, N=48, window=8)
    inp = synth.make_inputs(wl)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"]).cuda()
    k1, k2 = 5, 9
    plan = api.Plan(api.Desc.from_workload(wl, exec=exec_mode, tol=tol, gram="3xtf32"))
    X_full, it_full = _run(api, plan, Y, m, k1 + k2)
    state = api.new_state(plan)
    X1, it1 = _run(api, plan, Y, m, k1, state=state)
    X2, it2 = _run(api, plan, Y, m, k2, state=state, resume=True)
    assert torch.equal(X_full, X2)
    if tol < 0:
        assert (it1, it2, it_full) == (k1, k2, k1 + k2)
    # a different plan of the same description resumes from the same checkpoint
    plan2 = api.Plan(api.Desc.from_workload(wl, exec=exec_mode, tol=tol, gram="3xtf32"))
    state2 = api.new_state(plan2)
    _run(api, plan2, Y, m, k1, state=state2)
    X3, _ = _run(api, plan2, Y, m, k2, state=state2, resume=True)
    assert torch.equal(X_full, X3)


def test_resume_batched_plan():
    api = _api()
    base = get_config("shlr_4c_64").with_(mask="random1d", R=3.0, n_acs=4)
    cfgs = [base.with_(J=2, M=24, N=24, window=4, seed=41), base.with_(J=3, M=32, N=40, window=5, seed=42)]
    inps = [synth.make_inputs(c) for c in cfgs]
    plan = api.BatchPlan([api.Desc.from_workload(c, max_iter=10) for c in cfgs])
    Yp = plan.pack([torch.from_numpy(i["Y"].astype(np.complex64)).cuda() for i in inps], torch.complex64)
    mp = plan.pack([torch.from_numpy(i["mask"]).cuda() for i in inps], torch.uint8, mask=True)
    X_full = torch.empty_like(Yp)
    api.selr_solve_batch(plan, Yp, mp, X_full)
    state = api.new_state(plan)
    plan.set_iterations(4)
    X1 = torch.empty_like(Yp)
    api.selr_solve_batch(plan, Yp, mp, X1, state=state)
    plan.set_iterations(6)
    X2 = torch.empty_like(Yp)
    api.selr_solve_batch(plan, Yp, mp, X2, state=state, resume=True)
    assert api.selr_sync_status(plan) == 0
    assert torch.equal(X_full, X2)


def test_rank_sums_match_oracle_ranks_after_one_iteration():
    api = _api()
    wl = get_config("shlr_4c_64")
    inp = synth.make_inputs(wl)
    plan = api.Plan(api.Desc.from_workload(wl, max_iter=1))
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    _run(api, plan, Y, torch.from_numpy(inp["mask"]).cuda(), 1)
    sums, it = api.selr_plan_rank_sums(plan)
    assert it == 1
    s = oadmm.Shlr2D(inp["Y"], inp["mask"], wl)
    st = s.init_state()
    K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"])
    LXr, LXc = s.lifts(K)
    b = wl.beta
    ref = np.concatenate([svt_rank(LXr + st["Dr"] / b, 1.0 / b), svt_rank(LXc + st["Dc"] / b, 1.0 / b)])
    assert sums.shape == ref.shape
    assert np.count_nonzero(sums != ref) <= 2, (sums, ref)
    assert ref.sum() > 0


def test_fp32_peak_probe_is_plausible():
    api = _api()
    tf, ms = api.selr_probe_fp32_peak(False, 2048)
    tf2, _ = api.selr_probe_fp32_peak(True, 2048)
    assert 20.0 < tf < 400.0 and ms > 0
    assert 20.0 < tf2 < 800.0
