"""GPU test of selr_svt_noalloc, the allocation-free SVT entry point.

Callers that cannot allocate device memory at run time (work issued during a
stream capture, services with a fixed memory budget, frameworks that own all
device allocations) use selr_svt_noalloc instead of a plan.  This file checks,
through the C ABI, that two consecutive calls give the same S_t as the
plan-based selr_svt within the SVT tolerance of the other tests (1e-4
relative, FP32 Jacobi) and the FP64 oracle's S_t, that the status word reads
clean after them, that oversize inputs are rejected with SELR_ERR_SHAPE, and
that a call needs no plan.  It is collected last so that a
run stopping at the first failure has already run every other test, and it
passes both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import svt as osvt

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11650_gb300 import build
    build()


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _case(seed, nmat, rows, cols):
    rng = np.random.default_rng(seed)
    r = max(1, min(rows, cols) // 5)
    A = np.einsum("nik,nkj->nij", _crandn(rng, nmat, rows, r), _crandn(rng, nmat, r, cols))
    A = A + 0.05 * _crandn(rng, nmat, rows, cols)
    s = np.linalg.svd(A, compute_uv=False)
    return A, float(np.median(s[:, :max(1, min(rows, cols) // 4)]))


def test_noalloc_matches_plan_svt_twice_in_a_row():
    from paper_2107_11650_gb300 import api
    plan = api.Plan(api.Desc(model="SHLR", J=12, M=64, N=64, window=16))
    for seed, (nmat, rows, cols) in ((1, (5, 241, 192)), (2, (7, 33, 70))):
        A, t = _case(seed, nmat, rows, cols)
        ref_t = torch.from_numpy(A.astype(np.complex64)).cuda()
        api.selr_svt(plan, ref_t, t)
        assert api.selr_sync_status(plan) == 0
        got = torch.from_numpy(A.astype(np.complex64)).cuda()
        rank = torch.full((nmat,), -1, dtype=torch.int32, device="cuda")
        api.selr_svt_noalloc(got, t, max_sweeps=30, tol=2.0e-6, rank_out=rank)
        torch.cuda.synchronize()
        ref = ref_t.cpu().numpy().astype(np.complex128)
        z = got.cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
        assert err < TOL, err
        sv = np.linalg.svd(A, compute_uv=False)
        assert (rank.cpu().numpy() == (sv > t).sum(axis=1)).all()
        assert api.selr_svt_noalloc_status() == 0
        exact = osvt.svt(A, t)
        per_mat = np.linalg.norm(z - exact, axis=(1, 2)) / np.linalg.norm(exact, axis=(1, 2))
        assert per_mat.max() < TOL, per_mat


def test_noalloc_checks_devices_of_its_arguments():
    from paper_2107_11650_gb300 import api
    A = torch.zeros((2, 8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        api.selr_svt_noalloc(A, 1.0, rank_out=torch.zeros(2, dtype=torch.int32))


def test_noalloc_rejects_oversize_and_bad_arguments():
    from paper_2107_11650_gb300 import api
    big = torch.zeros((30, 241, 192), dtype=torch.complex64, device="cuda")   # > 2^20 elements
    with pytest.raises(api._lib.SelrError) as e:
        api.selr_svt_noalloc(big, 1.0)
    assert e.value.code == 2
    small = torch.zeros((2, 8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(api._lib.SelrError) as e:
        api.selr_svt_noalloc(small, -1.0)
    assert e.value.code == 1
