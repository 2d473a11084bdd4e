"""Parity cases of the eigensolver SVT that depend on its launch chain and on
the tensor-core Gram, each checked per matrix (or per instance / FE position)
against the FP64 oracle, not only as one Frobenius ratio over the batch.

* Two calls of selr_svt on one 3xTF32 plan with different inputs and ranks:
  the k_eigvec -> apply hand-off flag of the first call must not be seen by
  the second call's apply (small batches, where every CTA of the chain is
  resident at once, are where a stale flag would be read).
* SHLR-P / SHLR-VP reconstructions with the 3xTF32 Gram (Algorithm S2 with
  both lift families and the warp-per-matrix parameter lifts in one plan).
* A batched plan of uneven 2D instances with the 3xTF32 Gram.
* Matrices with more than 64 singular values above t (k_apply_eig), FP32 and
  3xTF32 Gram, with the rank against numpy's SVD.
Bars: 1e-5 relative per SVT matrix (FP32-level Gram modes), 1e-4 per
reconstruction after a fixed iteration count.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from synth.configs import get_config
from oracle import svt as osvt
from oracle import admm as oadmm
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu
SVT_TOL = 1e-5
TOL = 1e-4


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


def _spectral(rng, nmat, rows, cols, decay):
    k = min(rows, cols)
    out = []
    for _ in range(nmat):
        U, _ = np.linalg.qr(_crandn(rng, rows, k))
        V, _ = np.linalg.qr(_crandn(rng, cols, k))
        out.append((U * decay ** np.arange(k)) @ V.conj().T)
    return np.stack(out)


def _worst(a, ref, axes):
    """Largest relative error over the slices that `axes` leaves."""
    num = np.sqrt(np.sum(np.abs(a - ref) ** 2, axis=axes))
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=axes))
    return float(np.max(num / den))


def _gpu_svt(plan, A, t):
    api = _api()
    dA = torch.from_numpy(A.astype(np.complex64)).cuda()
    rank = torch.full((A.shape[0],), -1, dtype=torch.int32, device="cuda")
    api.selr_svt(plan, dA, t, rank_out=rank)
    assert api.selr_sync_status(plan) == 0
    return dA.cpu().numpy().astype(np.complex128), rank.cpu().numpy()


@pytest.mark.parametrize("gram", ["3xtf32", "tf32"])
def test_svt_twice_on_one_tensor_core_plan(gram):
    api = _api()
    rng = np.random.default_rng(77)
    plan = api.Plan(api.Desc(model="SHLR", J=4, M=64, N=64, window=8, gram=gram))
    cases = [(_spectral(rng, 4, 57, 32, 0.80), 8), (_spectral(rng, 6, 57, 32, 0.93), 20),
             (_spectral(rng, 3, 57, 32, 0.70), 2)]
    bound = SVT_TOL if gram == "3xtf32" else 2e-3
    for A, r in cases:
        s = np.linalg.svd(A, compute_uv=False)
        t = float(0.5 * (s[0, r - 1] + s[0, r]))
        Z, rank = _gpu_svt(plan, A, t)
        ref = osvt.svt(A, t)
        assert _worst(Z, ref, (1, 2)) < bound
        assert (rank == (s > t).sum(axis=1)).all(), (rank, (s > t).sum(axis=1))
    plan.close()


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_parameter_models_with_3xtf32_gram(model):
    api = _api()
    wl = get_config("shlrvp_8c_192_8e").with_(model=model, J=2, M=8, N=48, window=8, n_iter=10)
    inp = synth.make_inputs(wl)
    plan = api.Plan(api.Desc.from_workload(wl, gram="3xtf32"))
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    X = torch.empty_like(Y)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        it, _ = api.selr_solve(plan, Y, torch.from_numpy(inp["mask"]).cuda(), X, stream=s)
    assert it == 10 and api.selr_sync_status(plan, s) == 0
    Xo, _, _ = oadmm.shlr_p(inp["Y"], inp["mask"], wl, n_iter=10)
    Xg = X.cpu().numpy().astype(np.complex128)
    assert rel_l2(Xg, Xo) < TOL
    assert _worst(Xg, Xo, (0, 1, 3)) < 2 * TOL          # worst FE position
    plan.close()


def test_batch_plan_with_3xtf32_gram():
    api = _api()
    base = get_config("shlr_4c_64").with_(mask="random1d", R=3.0, n_acs=4)
    sizes = [(2, 24, 24, 4), (3, 32, 40, 5), (4, 48, 48, 8), (2, 20, 30, 3)]
    inst = []
    for i, (J, M, N, p) in enumerate(sizes):
        cfg = base.with_(J=J, M=M, N=N, window=p, seed=31 + i)
        d = synth.make_inputs(cfg)
        inst.append((cfg, d["Y"], d["mask"]))
    n_iter = 8
    plan = api.BatchPlan([api.Desc.from_workload(c, max_iter=n_iter, gram="3xtf32") for c, _, _ in inst])
    Yp = plan.pack([torch.from_numpy(Y.astype(np.complex64)).cuda() for _, Y, _ in inst], torch.complex64)
    mp = plan.pack([torch.from_numpy(m).cuda() for _, _, m in inst], torch.uint8, mask=True)
    Xp = torch.empty_like(Yp)
    it, _ = api.selr_solve_batch(plan, Yp, mp, Xp)
    assert it == n_iter and api.selr_sync_status(plan) == 0
    for i, (cfg, Y, m) in enumerate(inst):
        Xo = oadmm.shlr(Y, m, cfg, n_iter=n_iter)[0]
        Xg = plan.unpack(Xp, i).cpu().numpy().astype(np.complex128)
        assert rel_l2(Xg, Xo) < TOL, i
    plan.close()


@pytest.mark.parametrize("gram", ["fp32", "3xtf32"])
@pytest.mark.parametrize("nmat,rows,cols,r", [(3, 241, 192, 100), (2, 300, 256, 90), (2, 130, 200, 70)])
def test_svt_more_than_64_pairs_above_threshold(gram, nmat, rows, cols, r):
    api = _api()
    rng = np.random.default_rng(rows + cols + r)
    A = _spectral(rng, nmat, rows, cols, 0.985)
    s = np.linalg.svd(A, compute_uv=False)
    t = float(0.5 * (s[0, r - 1] + s[0, r]))
    plan = api.Plan(api.Desc(model="SHLR", J=12, M=320, N=320, window=16, gram=gram))
    Z, rank = _gpu_svt(plan, A, t)
    assert (rank == r).all() and (rank > 64).all()
    assert _worst(Z, osvt.svt(A, t), (1, 2)) < SVT_TOL
    plan.close()
