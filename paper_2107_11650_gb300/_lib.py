"""ctypes loader for libselr.so (the C ABI declared in include/selr.h).

Argument marshalling only: no arithmetic of the method happens in Python.
Importing this module never builds anything; a missing or unloadable library
raises immediately (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libselr.so")

SELR_OK = 0
STATUS_NAMES = {0: "SELR_OK", 1: "SELR_ERR_INVALID_ARG", 2: "SELR_ERR_SHAPE", 3: "SELR_ERR_CUDA",
                4: "SELR_ERR_NO_CONVERGENCE", 5: "SELR_ERR_NONFINITE", 6: "SELR_ERR_TIMEOUT",
                7: "SELR_ERR_UNSUPPORTED", 8: "SELR_ERR_ALLOC"}
MODELS = {"SHLR": 0, "SHLR_V": 1, "SHLR_P": 2, "SHLR_VP": 3, "SHLR_S": 4, "SHLR_SV": 5}
AXES = {"row": 0, "col": 1, "pe": 2, "param": 3}
EXEC = {"batched": 0, "plain": 1}
SVD = {"eig": 0, "jacobi": 1}
GRAM = {"fp32": 0, "tf32": 1, "3xtf32": 3, "bf16x3": 4, "bf16x6": 6}

# Every function declared in include/selr.h, with its ctypes signature.
c_void_p, c_int32, c_float, c_size_t = ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, ctypes.c_size_t


class SelrDesc(ctypes.Structure):
    _fields_ = [("model", c_int32), ("J", c_int32), ("M", c_int32), ("N", c_int32), ("L", c_int32),
                ("window", c_int32), ("window_param", c_int32), ("weight", c_int32),
                ("lambda_", c_float), ("lambda2", c_float), ("beta", c_float), ("tau", c_float),
                ("d_init", c_float), ("max_iter", c_int32), ("tol", c_float),
                ("jacobi_max_sweeps", c_int32), ("jacobi_tol", c_float), ("exec_", c_int32),
                ("svd_method", c_int32), ("gram_precision", c_int32), ("lambda1", c_float),
                ("spirit_ksize", c_int32), ("spirit_acs", c_int32), ("spirit_reg", c_float), ("cg_iters", c_int32),
                ("fp64_fallback", c_int32)]


SIGNATURES = {
    "selr_desc_default": (None, [ctypes.POINTER(SelrDesc)]),
    "selr_plan_create": (c_int32, [ctypes.POINTER(SelrDesc), ctypes.POINTER(c_void_p)]),
    "selr_plan_destroy": (c_int32, [c_void_p]),
    "selr_plan_workspace_bytes": (c_size_t, [c_void_p]),
    "selr_lift_shape": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                  ctypes.POINTER(c_int32)]),
    "selr_transform": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "selr_lift": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "selr_svt": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_void_p, c_void_p]),
    "selr_svt_noalloc": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_float, c_int32, c_float, c_void_p,
                                   c_void_p]),
    "selr_svt_noalloc_status": (c_int32, [c_void_p]),
    "selr_adjoint": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "selr_spirit_calibrate": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "selr_spirit_kernel": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "selr_dc": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "selr_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                             ctypes.POINTER(c_int32), ctypes.POINTER(c_float), c_void_p]),
    "selr_state_bytes": (c_int32, [c_void_p, ctypes.POINTER(c_size_t)]),
    "selr_solve_unrolled": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_float),
                                      ctypes.POINTER(c_float), c_int32, c_void_p, c_void_p, c_void_p]),
    "selr_lifted_elems": (c_int32, [c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "selr_lifted_unpack": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "selr_plan_rank_sums": (c_int32, [c_void_p, ctypes.POINTER(ctypes.c_int64), c_int32, ctypes.POINTER(c_int32),
                                      c_void_p]),
    "selr_probe_fp32_peak": (c_int32, [c_int32, c_int32, ctypes.POINTER(c_float), ctypes.POINTER(c_float)]),
    "selr_ssos": (c_int32, [c_void_p, c_int32, c_int32, ctypes.c_int64, c_void_p, c_void_p]),
    "selr_rlne": (c_int32, [c_void_p, c_void_p, ctypes.c_int64, c_void_p, c_void_p]),
    "selr_mssim": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_float, c_void_p, c_void_p, c_void_p]),
    "selr_max": (c_int32, [c_void_p, ctypes.c_int64, c_void_p, c_void_p]),
    "selr_t2_fit": (c_int32, [c_void_p, ctypes.POINTER(c_float), c_int32, ctypes.c_int64, c_float, c_float, c_void_p,
                              c_void_p, c_void_p]),
    "selr_sync_status": (c_int32, [c_void_p, c_void_p]),
    "selr_selftest_wait": (c_int32, [c_int32, c_int32]),
    "selr_set_iterations": (c_int32, [c_void_p, c_int32, c_float]),
    "selr_profile_enable": (c_int32, [c_void_p, c_int32]),
    "selr_profile_read": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_float), ctypes.POINTER(c_int32)]),
    "selr_status_string": (ctypes.c_char_p, [c_int32]),
    "selr_last_error_string": (ctypes.c_char_p, []),
    "selr_plan_create_batch": (c_int32, [ctypes.POINTER(SelrDesc), c_int32, ctypes.POINTER(c_void_p)]),
    "selr_plan_instance_layout": (c_int32, [c_void_p, c_int32, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]),
    "selr_plan_autotune": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "selr_plan_set_tuning": (c_int32, [c_void_p, c_int32, c_int32]),
    "selr_plan_set_reduction": (c_int32, [c_void_p, c_int32]),
    "selr_plan_get_reduction": (c_int32, [c_void_p, ctypes.POINTER(c_int32)]),
    "selr_plan_tuning": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                   ctypes.POINTER(c_int32)]),
    "selr_svt_vjp": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_void_p,
                               c_void_p, c_void_p, c_void_p]),
    "selr_dc_vjp": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "selr_axpby": (c_int32, [ctypes.c_int64, c_float, c_void_p, c_float, c_void_p, c_float, c_void_p, c_void_p,
                             c_void_p]),
    "selr_dot_re": (c_int32, [c_void_p, ctypes.c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
}

_lib = None


def load(path: str | None = None):
    """Load libselr.so (cached).  Raises RuntimeError if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libselr.so not found at {p}; build it with "
                           "`python -m paper_2107_11650_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class SelrError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")


def check(code, where):
    if code != SELR_OK:
        if code == 3 and _lib is not None:
            where = f"{where} ({_lib.selr_last_error_string().decode()})"
        raise SelrError(code, where)
