"""SHLR-S / SHLR-SV (Eq. 3 / Eq. 6, Eq. 15 with the SPIRiT term) on the GPU
against the FP64 oracle.

* The SPIRiT kernel calibrated on the GPU (FP64 normal equations, Cholesky per
  target coil) equals the oracle's calibration of the same complex64 data.
* Reconstructions (SHLR-S and SHLR-SV, 10 iterations, batched and plain) match
  the oracle, whose X-update is an exact CG solve (relative residual 1e-12),
  while the GPU runs 30 Jacobi-preconditioned CG iterations.
* The checkpoint of a SPIRiT plan resumes bitwise.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import admm as oadmm, spirit as ospirit
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu
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


def _case(model, J=4, M=64, N=64, window=8, n_acs=12, n_iter=10, ks=5):
    wl = synth.get_config("shlr_12c_256").with_(model=model, J=J, M=M, N=N, window=window, n_acs=n_acs,
                                                 n_iter=n_iter, spirit_k=ks)
    inp = synth.make_inputs(wl)
    inp["Y"] = inp["Y"].astype(np.complex64).astype(np.complex128)
    return wl, inp


@pytest.mark.parametrize("J,ks", [(4, 5), (8, 3), (3, 7)])
def test_calibration_matches_oracle(J, ks):
    api = _api()
    wl, inp = _case("SHLR_S", J=J, ks=ks, n_acs=16)
    plan = api.Plan(api.Desc.from_workload(wl))
    api.selr_spirit_calibrate(plan, torch.from_numpy(inp["Y"].astype(np.complex64)).cuda())
    g = api.selr_spirit_kernel(plan).cpu().numpy().astype(np.complex128)
    assert api.selr_sync_status(plan) == 0
    ref = ospirit.calibrate(inp["Y"], wl.n_acs, ks, wl.spirit_reg)
    assert rel_l2(g, ref) < 1e-5


@pytest.mark.parametrize("model,exec_mode", [("SHLR_S", "batched"), ("SHLR_SV", "batched"), ("SHLR_SV", "plain")])
def test_spirit_reconstruction_matches_oracle(model, exec_mode):
    api = _api()
    wl, inp = _case(model)
    plan = api.Plan(api.Desc.from_workload(wl, exec=exec_mode, gram="3xtf32"))
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    X = torch.empty_like(Y)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        it, _ = api.selr_solve(plan, Y, torch.from_numpy(inp["mask"]).cuda(), X, stream=s)
    assert it == wl.n_iter and api.selr_sync_status(plan, s) == 0
    Xo = oadmm.shlr(inp["Y"], inp["mask"], wl, n_iter=wl.n_iter)[0]
    Xg = X.cpu().numpy().astype(np.complex128)
    assert rel_l2(Xg, Xo) < TOL
    # it is a different reconstruction from plain SHLR on the same data
    Xp = oadmm.shlr(inp["Y"], inp["mask"], wl.with_(model="SHLR_V" if model == "SHLR_SV" else "SHLR"),
                    n_iter=wl.n_iter)[0]
    assert rel_l2(Xg, Xp) > 10 * TOL


def test_spirit_checkpoint_resume_bitwise():
    api = _api()
    wl, inp = _case("SHLR_SV", n_iter=8)
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    m = torch.from_numpy(inp["mask"]).cuda()
    plan = api.Plan(api.Desc.from_workload(wl))
    X1 = torch.empty_like(Y)
    api.selr_solve(plan, Y, m, X1)
    state = api.new_state(plan)
    plan.set_iterations(3)
    X2 = torch.empty_like(Y)
    api.selr_solve(plan, Y, m, X2, state=state)
    plan.set_iterations(5)
    api.selr_solve(plan, Y, m, X2, state=state, resume=True)
    assert api.selr_sync_status(plan) == 0
    assert torch.equal(X1, X2)
