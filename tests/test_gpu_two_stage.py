"""Two-stage Householder reduction (Hermitian band of half-bandwidth 16, then bulge
chasing) against the oracle: SVT values and exact ranks at orders across its range
(48 .. 192, ragged and multiples of 32, both orientations of the lifted matrix, low and
high ranks), the full-size 12-coil 256x256 SHLR and 4-parameter SHLR-VP reconstructions
against the stored FP64 oracle values, agreement with the one-stage reduction on a
reduced solve, and canaries around every output at ragged orders."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import svt as osvt
from oracle.metrics import rel_l2

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


def _lowrank(rng, nmat, rows, cols, r, top=10.0):
    k = min(rows, cols)
    A = np.empty((nmat, rows, cols), dtype=np.complex128)
    for m in range(nmat):
        U, _ = np.linalg.qr(_crandn(rng, rows, k))
        V, _ = np.linalg.qr(_crandn(rng, cols, k))
        s = np.concatenate([np.geomspace(top, 1.2, r), np.geomspace(0.8, 1e-3, k - r)])
        A[m] = (U * s) @ V.conj().T
    return A


def _plan(mode):
    """A plan whose own lifts (512 of order 192) give the two-stage scratch for the calls."""
    from paper_2107_11650_gb300 import api
    plan = api.Plan(api.Desc.from_workload(synth.get_config("shlr_12c_256")))
    plan.set_reduction(mode)
    return plan


@pytest.mark.parametrize("rows,cols,r", [(60, 48, 5), (241, 192, 12), (241, 192, 60), (192, 241, 20),
                                         (200, 191, 9), (97, 150, 30), (120, 97, 3), (70, 50, 49), (64, 64, 1)])
def test_two_stage_svt_matches_oracle(rows, cols, r):
    from paper_2107_11650_gb300 import api
    rng = np.random.default_rng(rows * 7 + cols + r)
    nmat = 5
    A = _lowrank(rng, nmat, rows, cols, r)
    out = {}
    for mode in (2, 1):
        plan = _plan(mode)
        At = torch.from_numpy(A.astype(np.complex64)).cuda()
        rank = torch.empty(nmat, dtype=torch.int32, device="cuda")
        api.selr_svt(plan, At, 1.0, rank)
        assert api.selr_sync_status(plan) == 0
        np.testing.assert_array_equal(rank.cpu().numpy(), osvt.svt_rank(A, 1.0))
        out[mode] = At.cpu().numpy().astype(np.complex128)
        ref = osvt.svt(A, 1.0)
        assert rel_l2(out[mode], ref) < TOL
        # every matrix on its own (a wrong matrix cannot hide in the batch ratio)
        for i in range(nmat):
            assert rel_l2(out[mode][i], ref[i]) < TOL, (mode, i)
    assert not np.array_equal(out[1], out[2])          # the two reductions did run


def test_two_stage_dense_spectrum_and_zero_matrix():
    """A full-rank random matrix (every pair above a small threshold) and an all-zero matrix
    (every reflector skipped) in one call."""
    from paper_2107_11650_gb300 import api
    rng = np.random.default_rng(3)
    plan = _plan(2)
    A = np.stack([_crandn(rng, 150, 130) / 10.0, np.zeros((150, 130))])
    At = torch.from_numpy(A.astype(np.complex64)).cuda()
    rank = torch.empty(2, dtype=torch.int32, device="cuda")
    api.selr_svt(plan, At, 0.05, rank)
    assert api.selr_sync_status(plan) == 0
    np.testing.assert_array_equal(rank.cpu().numpy(), osvt.svt_rank(A, 0.05))
    out = At.cpu().numpy().astype(np.complex128)
    assert rel_l2(out[0], osvt.svt(A[:1], 0.05)[0]) < TOL
    assert np.abs(out[1]).max() == 0.0


def _golden(name):
    d = os.path.join(os.path.dirname(__file__), "golden")
    hits = sorted(f for f in os.listdir(d) if f.startswith(name + "_") and f.endswith("it.npz"))
    return os.path.join(d, hits[0]) if hits else None


@pytest.mark.parametrize("name,gram", [("shlr_12c_256", "bf16x6"), ("shlr_12c_256", "fp32"),
                                       ("shlrvp_8c_192_8e", "bf16x6")])
def test_two_stage_full_size_sampled_golden(name, gram):
    """The stored FP64 oracle values after 30 iterations (tests/golden/make_golden.py), with
    the two-stage reduction forced for every eligible order."""
    from paper_2107_11650_gb300 import api
    path = _golden(name)
    if path is None:
        pytest.skip(f"no stored oracle values for {name}")
    g = np.load(path)
    wl = synth.get_config(name)
    inp = synth.make_inputs(wl)
    d = api.Desc.from_workload(wl, exec="batched", tol=-1.0, gram=gram)
    d.max_iter = int(g["n_iter"])
    plan = api.Plan(d)
    plan.set_reduction(2)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"].astype(np.uint8)).cuda()
    X = torch.empty_like(Y)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        api.selr_solve(plan, Y, m, X, stream=s)
    assert api.selr_sync_status(plan, s) == 0
    Xh = X.cpu().numpy().astype(np.complex128)
    xs = Xh.ravel()[g["idx"]]
    err = np.linalg.norm(xs - g["values"]) / np.linalg.norm(g["values"])
    assert err < TOL, err


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_two_stage_agrees_with_one_stage(model):
    from paper_2107_11650_gb300 import api
    wl = synth.get_config("shlr_12c_256").with_(model=model, J=4, M=96, N=80, window=12, n_iter=8)
    inp = synth.make_inputs(wl)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"].astype(np.uint8)).cuda()
    out = {}
    for mode in (1, 2):
        plan = api.Plan(api.Desc.from_workload(wl, gram="fp32"))
        plan.set_reduction(mode)
        X = torch.empty_like(Y)
        api.selr_solve(plan, Y, m, X)
        assert api.selr_sync_status(plan) == 0
        out[mode] = X.cpu().numpy().astype(np.complex128)
    assert rel_l2(out[2], out[1]) < 1e-5
    assert not np.array_equal(out[1], out[2])


GUARD = 4096
CANARY = 0x7FC0DEAD


@pytest.mark.parametrize("rows,cols", [(61, 49), (200, 97), (250, 191), (181, 192)])
def test_two_stage_outputs_stay_in_bounds(rows, cols):
    from paper_2107_11650_gb300 import api
    plan = _plan(2)
    nm = 3
    n = nm * rows * cols
    raw = torch.full(((n + 2 * GUARD) * 2,), CANARY, dtype=torch.int32, device="cuda")
    A = torch.view_as_complex(raw[2 * GUARD:2 * (GUARD + n)].view(torch.float32).view(n, 2))
    g = torch.Generator(device="cuda").manual_seed(rows + cols)
    A.copy_(torch.randn(n, dtype=torch.complex64, device="cuda", generator=g))
    rawr = torch.full((nm + 2 * GUARD,), CANARY, dtype=torch.int32, device="cuda")
    R = rawr[GUARD:GUARD + nm]
    api.selr_svt(plan, A.view(nm, rows, cols), 0.5, rank_out=R)
    assert api.selr_sync_status(plan) == 0
    torch.cuda.synchronize()
    for buf, gw in ((raw, 2 * GUARD), (rawr, GUARD)):
        assert bool((buf[:gw] == CANARY).all() and (buf[-gw:] == CANARY).all())


def test_autotune_tries_two_stage_and_keeps_a_set_mode():
    """The autotuner times the two-stage reduction on a plan left at mode 0 (order 48 here) and
    reports the mode in force; a plan set to one-stage stays one-stage.  The two tuned plans
    (possibly different Gram modes and reductions) agree within the metric's tolerance."""
    from paper_2107_11650_gb300 import api
    wl = synth.get_config("shlr_12c_256").with_(J=4, M=96, N=80, window=12, n_iter=4)
    inp = synth.make_inputs(wl)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"].astype(np.uint8)).cuda()
    plan = api.Plan(api.Desc.from_workload(wl))
    assert plan.autotune(Y, m)["reduction"] in (0, 2)
    fixed = api.Plan(api.Desc.from_workload(wl))
    fixed.set_reduction(1)
    assert fixed.autotune(Y, m)["reduction"] == 1
    out = []
    for p in (plan, fixed):
        X = torch.empty_like(Y)
        api.selr_solve(p, Y, m, X)
        assert api.selr_sync_status(p) == 0
        out.append(X.cpu().numpy().astype(np.complex128))
    assert rel_l2(out[0], out[1]) < TOL
