"""GPU parity of each C-ABI operator against the FP64 oracle.

Every comparison runs the CUDA path through the C ABI (ctypes binding) and
the oracle on the same seeded inputs.  Tolerances are FP32-level:
* linear operators (transform, lift, adjoint, X-update): relative Frobenius
  error <= 2e-6 / 5e-6 (one or two roundings per output, short sums);
* SVT: <= 1e-4 for both methods.  The Gram + eigensolver path reaches
  ~1e-6 (FP32 emulation of the same steps: 6.5e-7 on the 241x192 case).
  One-sided Jacobi in FP32 perturbs each column by O(u),
  u = 2^-24, per significant rotation; a column takes about sweeps * (s - 1)
  of them (15 * 383 here at most), so the backward error is about
  u * sqrt(5700) ~ 5e-6 of ||B||, and ||Z|| can be a third of ||B|| when the
  threshold sits inside the spectrum.  The bound keeps a factor ~6 above that.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import transforms as otr
from oracle import hankel as ohk
from oracle import svt as osvt
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


CASES_2D = [
    dict(model="SHLR", J=4, M=64, N=64, window=8, weight=1),
    dict(model="SHLR_V", J=3, M=30, N=40, window=7, weight=1),
    dict(model="SHLR", J=2, M=48, N=18, window=5, weight=0),
    dict(model="SHLR_V", J=12, M=64, N=64, window=16, weight=1),
]


@pytest.mark.parametrize("case", CASES_2D)
def test_transform(case):
    api = _api()
    rng = np.random.default_rng(1)
    plan = api.Plan(api.Desc(**case))
    x = _crandn(rng, case["J"], case["M"], case["N"])
    xd = _dev(x)
    out = torch.empty_like(xd)
    for dim, axis in ((0, 1), (1, 2)):
        for inv in (False, True):
            api.selr_transform(plan, dim, inv, xd, out)
            ref = otr.ifftc(x, axis=axis) if inv else otr.fftc(x, axis=axis)
            assert rel_l2(_host(out), ref) < 2e-6
    # in place
    y = xd.clone()
    api.selr_transform(plan, 1, False, y, y)
    assert rel_l2(_host(y), otr.fftc(x, axis=2)) < 2e-6


@pytest.mark.parametrize("case", CASES_2D)
def test_lift_rows_cols(case):
    api = _api()
    rng = np.random.default_rng(2)
    d = api.Desc(**case)
    plan = api.Plan(d)
    J, M, N, p = case["J"], case["M"], case["N"], case["window"]
    vc = case["model"] == "SHLR_V"
    x = _crandn(rng, J, M, N)
    for axis, fn, w in (("row", ohk.lift_rows, otr.filter_weights(N, case["weight"])),
                        ("col", ohk.lift_cols, otr.filter_weights(M, case["weight"]))):
        n, r, c = plan.lift_shape(axis)
        D = _crandn(rng, n, r, c)
        A = torch.empty((n, r, c), dtype=torch.complex64, device="cuda")
        api.selr_lift(plan, axis, _dev(x), _dev(D), A)
        ref = fn(x, w, p, vc) + D / d.beta
        assert ref.shape == (n, r, c)
        assert rel_l2(_host(A), ref) < 2e-6
        api.selr_lift(plan, axis, _dev(x), None, A)
        assert rel_l2(_host(A), fn(x, w, p, vc)) < 2e-6


@pytest.mark.parametrize("case", CASES_2D)
def test_adjoint_rows_cols(case):
    api = _api()
    rng = np.random.default_rng(3)
    plan = api.Plan(api.Desc(**case))
    J, M, N, p = case["J"], case["M"], case["N"], case["window"]
    vc = case["model"] == "SHLR_V"
    for axis in ("row", "col"):
        n, r, c = plan.lift_shape(axis)
        E = _crandn(rng, n, r, c)
        out = torch.empty((J, M, N), dtype=torch.complex64, device="cuda")
        api.selr_adjoint(plan, axis, _dev(E), out)
        if axis == "row":
            ref = ohk.lift_rows_adjoint(E, otr.filter_weights(N, case["weight"]), p, vc, J, N)
        else:
            ref = ohk.lift_cols_adjoint(E, otr.filter_weights(M, case["weight"]), p, vc, J, M)
        assert rel_l2(_host(out), ref) < 2e-6


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_lift_adjoint_parameter(model):
    api = _api()
    rng = np.random.default_rng(4)
    L, J, M, N, p, pP = 8, 3, 6, 48, 12, 4
    d = api.Desc(model=model, J=J, M=M, N=N, L=L, window=p, window_param=pP)
    plan = api.Plan(d)
    vc = model == "SHLR_VP"
    x = _crandn(rng, L, J, M, N)
    w = otr.filter_weights(N, 1)
    n, r, c = plan.lift_shape("pe")
    D = _crandn(rng, n, r, c)
    A = torch.empty((n, r, c), dtype=torch.complex64, device="cuda")
    api.selr_lift(plan, "pe", _dev(x), _dev(D), A)
    assert rel_l2(_host(A), ohk.lift_pe(x, w, p, vc) + D / d.beta) < 2e-6
    out = torch.empty_like(_dev(x))
    api.selr_adjoint(plan, "pe", _dev(D), out)
    assert rel_l2(_host(out), ohk.lift_pe_adjoint(D, w, p, vc, L, J, M, N)) < 2e-6
    n, r, c = plan.lift_shape("param")
    assert (n, r, c) == (M * N, L - pP + 1, J * pP)
    D = _crandn(rng, n, r, c)
    A = torch.empty((n, r, c), dtype=torch.complex64, device="cuda")
    api.selr_lift(plan, "param", _dev(x), _dev(D), A)
    assert rel_l2(_host(A), ohk.lift_param(x, pP) + D / d.beta) < 2e-6
    api.selr_adjoint(plan, "param", _dev(D), out)
    assert rel_l2(_host(out), ohk.lift_param_adjoint(D, pP, L, J, M, N)) < 2e-6


def _lowrank_plus_noise(rng, nmat, rows, cols, rank, noise):
    A = np.einsum("nik,nkj->nij", _crandn(rng, nmat, rows, rank), _crandn(rng, nmat, rank, cols))
    return A + noise * _crandn(rng, nmat, rows, cols)


@pytest.mark.parametrize("svd", ["eig", "jacobi"])
@pytest.mark.parametrize("shape", [(57, 32), (241, 192), (181, 192), (5, 32), (17, 9), (9, 17), (33, 33),
                                   (241, 384), (1, 7), (7, 1), (2, 2),
                                   # orders 193-208 (seven rows per lane), > 256 (global-memory
                                   # reduction) and the largest accepted order
                                   (205, 210), (300, 280), (480, 480)])
def test_svt_matches_oracle(shape, svd):
    api = _api()
    rng = np.random.default_rng(sum(shape))
    rows, cols = shape
    nmat = 6
    plan = api.Plan(api.Desc(model="SHLR_V", J=12, M=256, N=256, window=16, svd=svd))
    A = _lowrank_plus_noise(rng, nmat, rows, cols, max(1, min(rows, cols) // 6), 0.05)
    s = np.linalg.svd(A, compute_uv=False)
    t = float(np.median(s[:, : max(1, min(rows, cols) // 4)]))
    At = _dev(A)
    rank = torch.empty(nmat, dtype=torch.int32, device="cuda")
    api.selr_svt(plan, At, t, rank)
    assert api.selr_sync_status(plan) == 0
    Z = _host(At)
    ref = osvt.svt(A, t)
    assert rel_l2(Z, ref) < 1e-4, rel_l2(Z, ref)
    np.testing.assert_array_equal(rank.cpu().numpy(), osvt.svt_rank(A, t))


@pytest.mark.parametrize("svd", ["eig", "jacobi"])
def test_svt_special_cases(svd):
    api = _api()
    rng = np.random.default_rng(9)
    plan = api.Plan(api.Desc(svd=svd))
    A = _crandn(rng, 3, 20, 12)
    At = _dev(A)
    api.selr_svt(plan, At, 0.0)                       # S_0 = identity
    assert rel_l2(_host(At), A) < 2e-6
    At = _dev(A)
    api.selr_svt(plan, At, 1e6)                       # t >= sigma_max -> 0
    assert np.abs(_host(At)).max() == 0.0
    Z0 = torch.zeros((2, 20, 12), dtype=torch.complex64, device="cuda")
    api.selr_svt(plan, Z0, 0.5)                       # zero matrix stays zero
    assert np.abs(_host(Z0)).max() == 0.0
    assert api.selr_sync_status(plan) == 0


def test_svt_rejects_bad_shapes():
    api = _api()
    plan = api.Plan(api.Desc(J=1, M=16, N=16, window=4))
    big = torch.zeros((64, 200, 200), dtype=torch.complex64, device="cuda")
    with pytest.raises(api._lib.SelrError) as e:
        api.selr_svt(plan, big, 1.0)
    assert e.value.code == 2
    with pytest.raises(api._lib.SelrError) as e:
        api.selr_svt(plan, big[:1, :4, :4].contiguous(), -1.0)
    assert e.value.code == 1


@pytest.mark.parametrize("model,lam", [("SHLR", 1e4), ("SHLR_V", 50.0), ("SHLR", 0.0)])
def test_dc_matches_oracle(model, lam):
    api = _api()
    rng = np.random.default_rng(5)
    J, M, N, p = 3, 32, 48, 6
    wl = synth.Workload(name="t", model=model, J=J, M=M, N=N, window=p, lam=lam, beta=7.0, tau=7.0)
    plan = api.Plan(api.Desc.from_workload(wl))
    U = synth.mask_1d_random(M, N, 3.0, 6, rng)
    Y = _crandn(rng, J, M, N) * U[None]
    s = oadmm.Shlr2D(Y, U, wl)
    C = 2 * J if model == "SHLR_V" else J
    Zr, Dr = _crandn(rng, M, N - p + 1, C * p), _crandn(rng, M, N - p + 1, C * p)
    Zc, Dc = _crandn(rng, N, M - p + 1, C * p), _crandn(rng, N, M - p + 1, C * p)
    K0 = _crandn(rng, J, M, N)
    ref = s.x_update(Zr, Zc, Dr, Dc)
    b = wl.beta
    a_row = torch.empty((J, M, N), dtype=torch.complex64, device="cuda")
    a_col = torch.empty_like(a_row)
    api.selr_adjoint(plan, "row", _dev(Zr - Dr / b), a_row)
    api.selr_adjoint(plan, "col", _dev(Zc - Dc / b), a_col)
    K = _dev(K0)
    rel = torch.zeros(1, dtype=torch.float32, device="cuda")
    api.selr_dc(plan, _dev(Y), _dev(U, torch.uint8), a_row, a_col, K, rel)
    assert rel_l2(_host(K), ref) < 5e-6
    ref_rel = np.sum(np.abs(ref - K0) ** 2) / np.sum(np.abs(K0) ** 2)
    assert abs(rel.item() - ref_rel) < 1e-5 * ref_rel


@pytest.mark.parametrize("model", ["SHLR_P", "SHLR_VP"])
def test_dc_parameter_matches_oracle(model):
    api = _api()
    rng = np.random.default_rng(6)
    L, J, M, N, p, pP = 6, 2, 4, 30, 7, 3
    wl = synth.Workload(name="t", model=model, J=J, M=M, N=N, L=L, window=p, window_param=pP,
                        lam=300.0, lam2=2.0, beta=5.0, tau=5.0)
    plan = api.Plan(api.Desc.from_workload(wl))
    U = np.zeros((L, M, N), np.uint8)
    for l in range(L):
        U[l] = synth.mask_1d_random(M, N, 3.0, 4, np.random.default_rng(l), axis=1)
    Y = _crandn(rng, L, J, M, N) * U[:, None]
    s = oadmm.ShlrParam(Y, U, wl)
    C = 2 * J if model == "SHLR_VP" else J
    Zpe, Dpe = _crandn(rng, M * L, N - p + 1, C * p), _crandn(rng, M * L, N - p + 1, C * p)
    Zp, Dp = _crandn(rng, M * N, L - pP + 1, J * pP), _crandn(rng, M * N, L - pP + 1, J * pP)
    K0 = _crandn(rng, L, J, M, N)
    ref = s.x_update(Zpe, Zp, Dpe, Dp)
    b = wl.beta
    a_pe = torch.empty((L, J, M, N), dtype=torch.complex64, device="cuda")
    a_p = torch.empty_like(a_pe)
    api.selr_adjoint(plan, "pe", _dev(Zpe - Dpe / b), a_pe)
    api.selr_adjoint(plan, "param", _dev(Zp - Dp / b), a_p)
    K = _dev(K0)
    api.selr_dc(plan, _dev(Y), _dev(U, torch.uint8), a_pe, a_p, K)
    assert rel_l2(_host(K), ref) < 5e-6
