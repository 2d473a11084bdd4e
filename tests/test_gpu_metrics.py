"""GPU evaluation kernels (Sec. IV, Supplement S3) against the FP64 oracle.

SSOS element by element; RLNE; MSSIM (11 x 11 Gaussian window, C1, C2 from
the dynamic range) on 256 x 256 and ragged images; the pixelwise T2 fit on
noisy synthetic decays and on the per-echo SSOS of a GPU SHLR-VP
reconstruction (identical inputs on both sides).  Bars: 1e-6 relative (SSOS,
RLNE), 1e-5 absolute (MSSIM, FP32 window sums), 1e-4 relative on every pixel
the oracle keeps (T2, M0).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from synth.configs import get_config
from oracle import metrics as om

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


def _f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_ssos_and_rlne():
    api = _api()
    rng = np.random.default_rng(1)
    X = (rng.standard_normal((8, 37, 29)) + 1j * rng.standard_normal((8, 37, 29))).astype(np.complex64)
    s = api.selr_ssos(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = om.ssos(X.astype(np.complex128))
    assert np.abs(s - ref).max() <= 1e-6 * ref.max()
    P = (rng.standard_normal((4, 3, 16, 12)) + 1j * rng.standard_normal((4, 3, 16, 12))).astype(np.complex64)
    sp = api.selr_ssos(torch.from_numpy(P).cuda()).cpu().numpy()
    refp = om.ssos(P.astype(np.complex128), coil_axis=1)
    assert np.abs(sp - refp).max() <= 1e-6 * refp.max()
    a, b = rng.random(5000).astype(np.float32), rng.random(5000).astype(np.float32)
    r = float(api.selr_rlne(_f32(a), _f32(b)).item())
    assert abs(r - om.rlne(a.astype(np.float64), b.astype(np.float64))) <= 1e-6 * r


@pytest.mark.parametrize("M,N", [(256, 256), (37, 29), (11, 11)])
def test_mssim(M, N):
    api = _api()
    wl = get_config("shlr_4c_64")
    inp = synth.make_inputs(wl, small=(4, M, N))
    A = om.ssos(inp["truth"])
    rng = np.random.default_rng(M + N)
    B = A + 0.05 * A.max() * rng.standard_normal(A.shape)
    g, smap = api.selr_mssim(_f32(A), _f32(B))
    ref = om.mssim(A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64))
    assert abs(float(g.item()) - ref) < 1e-5, (float(g.item()), ref)
    assert smap.shape == (M - 10, N - 10)
    g1, _ = api.selr_mssim(_f32(A), _f32(A))
    assert abs(float(g1.item()) - 1.0) < 1e-5


def test_t2_fit_noisy_decays():
    api = _api()
    rng = np.random.default_rng(5)
    te = 10.0 * np.arange(1, 9)
    t2 = rng.uniform(20, 200, size=(24, 24))
    m0 = rng.uniform(0.2, 1.0, size=(24, 24))
    S = m0[None] * np.exp(-te[:, None, None] / t2[None])
    S = (S * (1 + 0.01 * rng.standard_normal(S.shape))).astype(np.float32)
    T2g, M0g = api.selr_t2_fit(_f32(S), te)
    T2o, M0o = om.t2_fit(S.astype(np.float64), te)
    keep = ~np.isnan(T2o)
    assert keep.mean() > 0.95
    np.testing.assert_array_equal(np.isnan(T2g.cpu().numpy()), ~keep)
    assert np.nanmax(np.abs(T2g.cpu().numpy()[keep] - T2o[keep]) / T2o[keep]) < 1e-4
    assert np.nanmax(np.abs(M0g.cpu().numpy()[keep] - M0o[keep]) / M0o[keep]) < 1e-4


def test_t2_map_of_a_reconstruction():
    api = _api()
    wl = get_config("shlrvp_8c_192_8e").with_(J=2, M=16, N=48, window=8, n_iter=10)
    inp = synth.make_inputs(wl)
    plan = api.Plan(api.Desc.from_workload(wl, gram="3xtf32"))
    Y = torch.from_numpy(inp["Y"].astype(np.complex64)).cuda()
    X = torch.empty_like(Y)
    api.selr_solve(plan, Y, torch.from_numpy(inp["mask"]).cuda(), X)
    assert api.selr_sync_status(plan) == 0
    # the reconstruction is hybrid (m, n image): per-echo SSOS over coils
    S = api.selr_ssos(X)
    te = [wl.te_ms * (l + 1) for l in range(wl.L)]
    T2g, _ = api.selr_t2_fit(S, te)
    T2o, _ = om.t2_fit(S.cpu().numpy().astype(np.float64), te)
    keep = ~np.isnan(T2o) & ~np.isnan(T2g.cpu().numpy())
    assert keep.mean() > 0.3
    assert np.max(np.abs(T2g.cpu().numpy()[keep] - T2o[keep]) / T2o[keep]) < 1e-4
