"""Eigenvectors refined per inverse-iteration pass (8 or 16: k_eigvec with
256 or 512 threads) on matrices with many pairs above the threshold: the
SVT matches the oracle for every chunk, with exact ranks, and a reconstruction
gives the same result whatever the chunk; the tuning setter validates its
arguments."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import svt as osvt
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11650_gb300 import build
    build()


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("chunk", [8, 16])
@pytest.mark.parametrize("rows,cols,r", [(181, 192, 45), (241, 192, 20), (120, 90, 33)])
def test_high_rank_svt_matches_oracle(chunk, rows, cols, r):
    from paper_2107_11650_gb300 import api
    rng = np.random.default_rng(rows + cols + r)
    plan = api.Plan(api.Desc(model="SHLR_V", J=12, M=256, N=256, window=16))
    plan.set_tuning("fp32", chunk)
    assert plan.tuning()["ev_chunk"] == chunk
    nmat, k = 4, min(rows, cols)
    A = np.empty((nmat, rows, cols), dtype=np.complex128)
    for m in range(nmat):
        U, _ = np.linalg.qr(_crandn(rng, rows, k))
        V, _ = np.linalg.qr(_crandn(rng, cols, k))
        s = np.concatenate([np.geomspace(10.0, 1.2, r), np.geomspace(0.8, 1e-3, k - r)])
        A[m] = (U * s) @ V.conj().T
    At = torch.from_numpy(A.astype(np.complex64)).cuda()
    rank = torch.empty(nmat, dtype=torch.int32, device="cuda")
    api.selr_svt(plan, At, 1.0, rank)
    assert api.selr_sync_status(plan) == 0
    np.testing.assert_array_equal(rank.cpu().numpy(), osvt.svt_rank(A, 1.0))
    assert rel_l2(At.cpu().numpy().astype(np.complex128), osvt.svt(A, 1.0)) < 1e-4


def test_reconstruction_independent_of_chunk():
    from paper_2107_11650_gb300 import api
    wl = synth.get_config("shlrvp_8c_192_8e").with_(J=4, M=16, N=96, window=12, n_iter=6)
    inp = synth.make_inputs(wl)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"]).cuda()
    out = {}
    for chunk in (8, 16):
        plan = api.Plan(api.Desc.from_workload(wl))
        plan.set_tuning("fp32", chunk)
        X = torch.empty_like(Y)
        api.selr_solve(plan, Y, m, X)
        assert api.selr_sync_status(plan) == 0
        out[chunk] = X.cpu().numpy().astype(np.complex128)
    assert rel_l2(out[8], out[16]) < 1e-5


def test_set_tuning_validates():
    from paper_2107_11650_gb300 import api
    plan = api.Plan(api.Desc())
    with pytest.raises(api._lib.SelrError) as e:
        plan.set_tuning("fp32", 32)
    assert e.value.code == 1
