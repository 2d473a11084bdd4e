"""C-ABI checks that need no GPU.

* libselr.so builds (nvcc cross-compiles for sm_103a) and loads.
* It exports every function declared in include/selr.h.
* Descriptor validation rejects bad arguments before any CUDA call.
"""
import ctypes
import os
import re

import pytest

from paper_2107_11650_gb300 import build
from paper_2107_11650_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "selr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(selr_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def test_status_strings(lib):
    for code, name in _lib.STATUS_NAMES.items():
        assert lib.selr_status_string(code).decode() == name


def _desc(lib, **kw):
    d = _lib.SelrDesc()
    lib.selr_desc_default(ctypes.byref(d))
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw,code", [
    (dict(model=7), 1), (dict(J=0), 1), (dict(beta=0.0), 1), (dict(tau=-1.0), 1), (dict(max_iter=0), 1),
    (dict(weight=3), 1), (dict(exec_=5), 1), (dict(jacobi_tol=0.0), 1), (dict(lambda2=-1.0), 1),
    (dict(svd_method=2), 1), (dict(gram_precision=2), 1), (dict(gram_precision=-1), 1),
    (dict(fp64_fallback=2), 1), (dict(gram_precision=5), 1),
    (dict(model=6), 1), (dict(model=4, lambda_=0.0), 1), (dict(model=4, spirit_ksize=4), 1),
    (dict(model=5, cg_iters=0), 1), (dict(model=4, spirit_acs=2), 2), (dict(model=4, J=33), 1),
    (dict(M=63), 2), (dict(N=14 * 7), 2), (dict(window=65), 2), (dict(L=2), 2),
    (dict(model=3, L=8, window_param=9, N=64), 2), (dict(model=2, L=8, window_param=4, N=66 * 7), 2),
])
def test_descriptor_validation(lib, kw, code):
    d = _desc(lib, **kw)
    h = ctypes.c_void_p()
    assert lib.selr_plan_create(ctypes.byref(d), ctypes.byref(h)) == code
    assert not h.value


def test_descriptor_defaults(lib):
    d = _desc(lib)
    assert (d.model, d.J, d.M, d.N, d.L, d.window) == (0, 4, 64, 64, 1, 8)
    assert (d.svd_method, d.gram_precision, d.exec_) == (0, 0, 0)
    assert d.fp64_fallback == 1
    assert (d.spirit_ksize, d.spirit_acs, d.cg_iters) == (5, 24, 30) and abs(d.lambda1 - 1e3) < 1e-3
    assert ctypes.sizeof(_lib.SelrDesc) == 26 * 4


def test_batch_descriptor_validation(lib):
    """Batched plans: sizes and lambda may differ; everything else must agree; 2D models only."""
    def create(descs):
        arr = (_lib.SelrDesc * len(descs))(*descs)
        h = ctypes.c_void_p()
        code = lib.selr_plan_create_batch(arr, len(descs), ctypes.byref(h))
        assert not h.value
        return code
    a = _desc(lib, J=2, M=64, N=64, window=70)          # shape error reported per description
    assert create([_desc(lib), a]) == 2
    assert create([_desc(lib), _desc(lib, beta=10.0)]) == 1
    assert create([_desc(lib), _desc(lib, svd_method=1)]) == 1
    # parameter-model batches pass validation (no GPU here: creation then fails at the first CUDA call)
    assert create([_desc(lib, model=2, L=8, window_param=4), _desc(lib, model=2, L=6, window_param=3)]) not in (1, 2, 7)
    assert create([_desc(lib, model=2, L=8, window_param=4), _desc(lib, model=3, L=8, window_param=4)]) == 1
    h = ctypes.c_void_p()
    assert lib.selr_plan_create_batch(None, 2, ctypes.byref(h)) == 1
    arr = (_lib.SelrDesc * 1)(_desc(lib))
    assert lib.selr_plan_create_batch(arr, 0, ctypes.byref(h)) == 1
    assert lib.selr_plan_create_batch(arr, 33, ctypes.byref(h)) == 1
    assert lib.selr_plan_instance_layout(None, 0, None, None) == 1


def test_null_arguments(lib):
    assert lib.selr_plan_create(None, None) == 1
    assert lib.selr_plan_destroy(None) == 0
    assert lib.selr_sync_status(None, None) == 1
    assert lib.selr_solve(None, None, None, None, None, 0, None, None, None) == 1
    assert lib.selr_plan_workspace_bytes(None) == 0
    # the wait self-test validates its arguments before any CUDA call
    assert lib.selr_selftest_wait(0, 0) == 1
    assert lib.selr_selftest_wait(2, 100) == 1
    assert lib.selr_selftest_wait(1, 2000001) == 1
    # state, rank and probe entry points validate their arguments before any CUDA call
    n = ctypes.c_size_t()
    assert lib.selr_state_bytes(None, ctypes.byref(n)) == 1
    assert lib.selr_plan_rank_sums(None, None, 0, None, None) == 1
    tf = ctypes.c_float()
    assert lib.selr_probe_fp32_peak(2, 16, ctypes.byref(tf), None) == 1
    assert lib.selr_probe_fp32_peak(0, 0, ctypes.byref(tf), None) == 1
    assert lib.selr_probe_fp32_peak(0, 16, None, None) == 1
    # evaluation entry points
    assert lib.selr_ssos(None, 1, 1, 1, None, None) == 1
    assert lib.selr_rlne(None, None, 1, None, None) == 1
    assert lib.selr_spirit_calibrate(None, None, None) == 1
    assert lib.selr_solve_unrolled(None, None, None, None, None, None, 1, None, None, None) == 1
    assert lib.selr_lifted_unpack(None, None, 0, 0, None, None) == 1
    assert lib.selr_lifted_elems(None, None) == 1
    assert lib.selr_spirit_kernel(None, None, None) == 1
    assert lib.selr_mssim(None, None, 16, 16, 1.0, None, None, None) == 1
    assert lib.selr_max(None, 1, None, None) == 1
    te = (ctypes.c_float * 1)(1.0)
    assert lib.selr_t2_fit(None, te, 1, 1, 1.0, 10.0, None, None, None) == 1
    assert lib.selr_plan_set_tuning(None, 0, 16) == 1
    assert lib.selr_plan_set_reduction(None, 2) == 1
    assert lib.selr_plan_get_reduction(None, None) == 1
