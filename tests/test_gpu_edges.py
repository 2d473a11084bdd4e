"""Edge cases of the CUDA path against the oracle.

* Transform lengths on both FFT kernels: the compile-time lengths (64 ... 512,
  512 with lifts of 509, the longest a plan takes) and the generic kernel
  (100 = 2^2 5^2, 250 = 2 5^3), along both dims.
* Degenerate data: a solve on all-zero k-space (the multipliers start at 1, so
  the iterates are not zero; the oracle fixes what they are).
* A single coil (J = 1), the smallest channel count, rectangular and ragged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import admm as oadmm
from oracle import transforms as otr
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


@pytest.mark.parametrize("n", [64, 160, 256, 320, 512, 100, 250])
def test_transform_lengths_both_kernels(n):
    api = _api()
    rng = np.random.default_rng(n)
    plan = api.Plan(api.Desc(model="SHLR", J=2, M=n, N=n if n <= 320 else 16, window=4))
    d = plan.desc
    x = _crandn(rng, d.J, d.M, d.N)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    out = torch.empty_like(xd)
    for dim, axis in ((0, 1), (1, 2)):
        for inv in (False, True):
            api.selr_transform(plan, dim, inv, xd, out)
            ref = otr.ifftc(x, axis=axis) if inv else otr.fftc(x, axis=axis)
            assert rel_l2(out.cpu().numpy().astype(np.complex128), ref) < 3e-6, (n, dim, inv)
    assert api.selr_sync_status(plan) == 0


def _solve(wl, Y, mask, n_iter):
    api = _api()
    plan = api.Plan(api.Desc.from_workload(wl, max_iter=n_iter, gram="fp32"))
    Yd = torch.from_numpy(np.ascontiguousarray(Y).astype(np.complex64)).cuda()
    md = torch.from_numpy(np.ascontiguousarray(mask).astype(np.uint8)).cuda()
    X = torch.empty_like(Yd)
    api.selr_solve(plan, Yd, md, X)
    return X.cpu().numpy().astype(np.complex128), api.selr_sync_status(plan)


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_zero_data_solve_matches_oracle(model):
    wl = synth.get_config("shlr_4c_64").with_(model=model, J=3, M=32, N=24, window=6, n_iter=8)
    inp = synth.make_inputs(wl)
    Y = np.zeros_like(inp["Y"])
    X, st = _solve(wl, Y, inp["mask"], 8)
    assert st == 0 and np.isfinite(X).all()
    ref, _, _ = oadmm.shlr(Y, inp["mask"], wl, n_iter=8)
    assert np.linalg.norm(ref) > 0
    assert rel_l2(X, ref) < 1e-4


@pytest.mark.parametrize("model", ["SHLR", "SHLR_V"])
def test_single_coil_matches_oracle(model):
    wl = synth.Workload(name="one", model=model, J=1, M=36, N=40, window=5, mask="random1d", R=2.5, n_acs=6,
                        sigma_n=1e-3, seed=13, beta=20.0, tau=20.0, n_iter=10)
    inp = synth.make_inputs(wl)
    X, st = _solve(wl, inp["Y"], inp["mask"], 10)
    assert st == 0
    ref, _, _ = oadmm.shlr(inp["Y"].astype(np.complex64).astype(np.complex128), inp["mask"], wl, n_iter=10)
    assert rel_l2(X, ref) < 1e-4
