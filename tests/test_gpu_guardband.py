"""Guard bands: every output the library writes is given as the middle of a larger
buffer whose head and tail hold a canary bit pattern; after the call (and a
synchronisation) the canaries must be intact, i.e. no kernel wrote outside the
array it was given.  Ragged sizes (3 coils, 20 x 18, window 5: lifts of 14 x 15
and 16 x 15; SVT orders that are not multiples of 32; batched and plain
execution; every Gram mode on the tensor cores) so that partial tiles, tails
and the bound checks of every kernel are exercised.  The canaries are compared
bit for bit on the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth

pytestmark = pytest.mark.gpu

GUARD = 4096                      # elements on each side
CANARY = 0x7FC0DEAD               # a NaN payload no kernel produces


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11650_gb300 import build
    build()


def _guarded(n, dtype):
    """((raw buffer, guard length in raw elements), middle view of n elements of dtype), the
    guards set to the canary; the raw buffer is int32 words (uint8 bytes for dtype uint8)."""
    if dtype == torch.uint8:
        raw = torch.full((n + 2 * GUARD,), 0xA5, dtype=torch.uint8, device="cuda")
        return (raw, GUARD), raw[GUARD:GUARD + n]
    words = 2 if dtype == torch.complex64 else 1
    raw = torch.full(((n + 2 * GUARD) * words,), CANARY, dtype=torch.int32, device="cuda")
    mid = raw[GUARD * words:(GUARD + n) * words]
    if dtype == torch.complex64:
        mid = torch.view_as_complex(mid.view(torch.float32).view(n, 2))
    elif dtype == torch.float32:
        mid = mid.view(torch.float32)
    return (raw, GUARD * words), mid


def _intact(guarded):
    raw, gw = guarded
    torch.cuda.synchronize()
    want = 0xA5 if raw.dtype == torch.uint8 else CANARY
    return bool((raw[:gw] == want).all() and (raw[-gw:] == want).all())


def _case(model="SHLR", exec_mode="batched", gram="fp32"):
    from paper_2107_11650_gb300 import api
    wl = synth.get_config("shlr_4c_64").with_(model=model, J=3, M=20, N=18, window=5, n_acs=6, n_iter=3,
                                              mask="random1d", R=3.0)
    inp = synth.make_inputs(wl)
    plan = api.Plan(api.Desc.from_workload(wl, exec=exec_mode, gram=gram))
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"].astype(np.uint8)).cuda()
    return api, plan, Y, m


@pytest.mark.parametrize("model,exec_mode,gram", [("SHLR", "batched", "fp32"), ("SHLR_V", "plain", "fp32"),
                                                  ("SHLR", "batched", "3xtf32"), ("SHLR_V", "batched", "bf16x6"),
                                                  ("SHLR_S", "batched", "fp32")])
def test_solve_outputs_stay_in_bounds(model, exec_mode, gram):
    api, plan, Y, m = _case(model, exec_mode, gram)
    fullX, X = _guarded(Y.numel(), torch.complex64)
    X = X.view(Y.shape)
    nb = api.selr_state_bytes(plan)
    fullS, S = _guarded(nb, torch.uint8)
    api.selr_solve(plan, Y, m, X, state=S)
    assert api.selr_sync_status(plan) == 0
    assert _intact(fullX) and _intact(fullS)
    api.selr_solve(plan, Y, m, X, state=S, resume=True)
    assert api.selr_sync_status(plan) == 0
    assert _intact(fullX) and _intact(fullS)


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_operator_outputs_stay_in_bounds(model):
    api, plan, Y, m = _case(model)
    n = Y.numel()
    fullT, T = _guarded(n, torch.complex64)
    api.selr_transform(plan, 0, True, Y, T.view(Y.shape))
    assert _intact(fullT)
    for axis in ("row", "col"):
        nm, r, c = plan.lift_shape(axis)
        fullA, A = _guarded(nm * r * c, torch.complex64)
        api.selr_lift(plan, axis, T.view(Y.shape), None, A.view(nm, r, c))
        assert _intact(fullA)
        fullR, R = _guarded(nm, torch.int32)
        api.selr_svt(plan, A.view(nm, r, c), 0.05, rank_out=R)
        assert _intact(fullA) and _intact(fullR)
        fullX, Xa = _guarded(n, torch.complex64)
        api.selr_adjoint(plan, axis, A.view(nm, r, c), Xa.view(Y.shape))
        assert _intact(fullX)
        fullB, Ab = _guarded(nm * r * c, torch.complex64)
        fullZ, Z = _guarded(nm * r * c, torch.complex64)
        fullt, tb = _guarded(1, torch.float32)
        Zb = torch.randn(nm, r, c, dtype=torch.complex64, device="cuda")
        api.selr_svt_vjp(plan, A.view(nm, r, c), Zb, 0.05, Ab.view(nm, r, c), tb, Z_out=Z.view(nm, r, c))
        assert _intact(fullB) and _intact(fullZ) and _intact(fullt)
    fullK, K = _guarded(n, torch.complex64)
    K.copy_(Y.reshape(-1))
    fullr, rel = _guarded(1, torch.float32)
    api.selr_dc(plan, Y, m, torch.zeros_like(Y), torch.zeros_like(Y), K.view(Y.shape), rel_out=rel)
    assert _intact(fullK) and _intact(fullr)
    assert api.selr_sync_status(plan) == 0


@pytest.mark.parametrize("rows,cols", [(37, 29), (61, 33), (200, 97), (250, 230), (305, 261)])
def test_svt_orders_not_multiple_of_32_stay_in_bounds(rows, cols):
    """Orders 29, 33 and 97 take the shared-memory reduction, 230 the hybrid one (first columns in
    global memory) and 261 the global-memory one, with partial warps and ragged tiles of every
    kernel of the chain."""
    from paper_2107_11650_gb300 import api
    plan = api.Plan(api.Desc(model="SHLR_V", J=12, M=256, N=256, window=16))   # scratch for orders <= 480
    g = torch.Generator(device="cuda").manual_seed(rows * cols)
    nm = 3
    fullA, A = _guarded(nm * rows * cols, torch.complex64)
    A.copy_(torch.randn(nm * rows * cols, dtype=torch.complex64, device="cuda", generator=g))
    fullR, R = _guarded(nm, torch.int32)
    api.selr_svt(plan, A.view(nm, rows, cols), 0.5, rank_out=R)
    assert api.selr_sync_status(plan) == 0
    assert _intact(fullA) and _intact(fullR)
