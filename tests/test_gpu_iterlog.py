"""Per-iteration JSONL log (paper_2107_11650_gb300.iterlog): the logged run,
one iteration at a time through the checkpoint path, ends bit for bit on the X
of one uninterrupted solve; each line carries the stopping quantity of
Algorithms S1 / S2 and the per-family histogram of singular values above the
threshold, whose counts equal the oracle's after the first iteration."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import admm as oadmm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11650_gb300 import build
    build()


def test_logged_run_matches_one_solve_and_oracle_ranks(tmp_path):
    from paper_2107_11650_gb300 import api, iterlog
    wl = synth.get_config("shlr_4c_64").with_(n_iter=4)
    inp = synth.make_inputs(wl)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"]).cuda()
    plan = api.Plan(api.Desc.from_workload(wl, gram="fp32"))
    X1 = torch.empty_like(Y)
    api.selr_solve(plan, Y, m, X1)
    assert api.selr_sync_status(plan) == 0
    path = str(tmp_path / "log.jsonl")
    X2 = torch.empty_like(Y)
    recs = iterlog.run_logged(plan, Y, m, X2, 4, path)
    assert torch.equal(X1, X2)
    lines = [json.loads(l) for l in open(path)]
    assert lines == json.loads(json.dumps(recs)) and [r["iteration"] for r in lines] == [1, 2, 3, 4]
    nrow = plan.lift_shape("row")[0]
    for r in lines:
        assert r["status"] == 0 and np.isfinite(r["rel_change"]) and r["rel_change"] > 0 and r["ms"] > 0
        assert sum(r["rank_hist"]["row"].values()) == nrow
    # first iteration: the counts of singular values above t = 1/beta equal those of the
    # oracle's first iteration (Algorithm S1: X-update, lifts, SVT of lift + D / beta), up to
    # two matrices with a singular value within FP32 rounding of t
    s = oadmm.Shlr2D(inp["Y"].astype(np.complex64).astype(np.complex128), inp["mask"], wl)
    st = s.init_state()
    K = s.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"])
    LXr, _ = s.lifts(K)
    b = wl.beta
    ranks = np.array([(np.linalg.svd(A, compute_uv=False) > 1.0 / b).sum() for A in LXr + st["Dr"] / b])
    ref = {int(v): int(c) for v, c in zip(*np.unique(ranks, return_counts=True))}
    got = lines[0]["rank_hist"]["row"]
    keys = set(ref) | set(int(k) for k in got)
    moved = sum(abs(ref.get(k, 0) - got.get(str(k), got.get(k, 0))) for k in keys)
    assert moved <= 4, (got, ref)
