"""Python binding of libselr with the C entry-point names.

Argument marshalling only: each function checks that its torch tensors are
contiguous CUDA tensors of the expected dtype and shape, then calls the C ABI
with their device pointers and the current CUDA stream.  Every step of the
reconstruction runs in libselr's kernels; if the library is missing the call
raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import AXES, EXEC, GRAM, MODELS, SVD, SelrDesc, check


@dataclass
class Desc:
    """Mirror of ``selr_desc`` (include/selr.h)."""
    model: str = "SHLR"
    J: int = 4
    M: int = 64
    N: int = 64
    L: int = 1
    window: int = 8
    window_param: int = 4
    weight: int = 1
    lam: float = 1.0e4
    lam2: float = 2.0
    beta: float = 20.0
    tau: float = 20.0
    d_init: float = 1.0
    max_iter: int = 30
    tol: float = -1.0
    jacobi_max_sweeps: int = 30
    jacobi_tol: float = 2.0e-6
    exec: str = "batched"
    svd: str = "eig"
    gram: str = "fp32"
    lam1: float = 1.0e3
    spirit_k: int = 5
    spirit_acs: int = 24
    spirit_reg: float = 1.0e-3
    cg_iters: int = 30
    fp64_fallback: int = 1

    @classmethod
    def from_workload(cls, w, **over):
        kw = dict(model=w.model, J=w.J, M=w.M, N=w.N, L=w.L, window=w.window, window_param=w.window_param,
                  weight=w.weight, lam=w.lam, lam2=w.lam2, beta=w.beta, tau=w.tau, d_init=w.d_init,
                  max_iter=w.n_iter, lam1=w.lam1, spirit_k=w.spirit_k, spirit_acs=w.n_acs,
                  spirit_reg=w.spirit_reg, cg_iters=w.cg_iters)
        kw.update(over)
        return cls(**kw)

    def to_c(self) -> SelrDesc:
        d = SelrDesc()
        d.model = MODELS[self.model]
        d.J, d.M, d.N, d.L = self.J, self.M, self.N, self.L
        d.window, d.window_param, d.weight = self.window, self.window_param, self.weight
        d.lambda_, d.lambda2, d.beta, d.tau = self.lam, self.lam2, self.beta, self.tau
        d.d_init, d.max_iter, d.tol = self.d_init, self.max_iter, self.tol
        d.jacobi_max_sweeps, d.jacobi_tol = self.jacobi_max_sweeps, self.jacobi_tol
        d.exec_ = EXEC[self.exec]
        d.svd_method = SVD[self.svd]
        d.gram_precision = GRAM[self.gram]
        d.lambda1, d.spirit_ksize, d.spirit_acs = self.lam1, self.spirit_k, self.spirit_acs
        d.spirit_reg, d.cg_iters = self.spirit_reg, self.cg_iters
        d.fp64_fallback = int(self.fp64_fallback)
        return d


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype, name, numel=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owns a ``selr_plan`` (device workspace on the current device)."""

    def __init__(self, desc: Desc):
        self.lib = _lib.load()
        self.desc = desc
        h = ctypes.c_void_p()
        cd = desc.to_c()
        check(self.lib.selr_plan_create(ctypes.byref(cd), ctypes.byref(h)), "selr_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.selr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nK(self):
        d = self.desc
        return d.L * d.J * d.M * d.N

    def workspace_bytes(self):
        return int(self.lib.selr_plan_workspace_bytes(self.handle))

    def set_iterations(self, max_iter, tol=-1.0):
        check(self.lib.selr_set_iterations(self.handle, int(max_iter), float(tol)), "selr_set_iterations")
        self.desc.max_iter, self.desc.tol = int(max_iter), float(tol)

    def autotune(self, Y, mask, allow_tf32=False, stream=None):
        """selr_plan_autotune on (Y, mask); returns the settings in force."""
        X = torch.empty_like(Y)
        nm = mask.numel()
        check(self.lib.selr_plan_autotune(self.handle, _ptr(Y, torch.complex64, "Y", self.nK),
                                          _ptr(mask, torch.uint8, "mask", nm),
                                          _ptr(X, torch.complex64, "X", self.nK), 1 if allow_tf32 else 0,
                                          _stream(stream)), "selr_plan_autotune")
        return self.tuning()

    def tuning(self):
        g, c, w = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(self.lib.selr_plan_tuning(self.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(w)),
              "selr_plan_tuning")
        names = {v: k for k, v in GRAM.items()}
        red = ctypes.c_int32()
        check(self.lib.selr_plan_get_reduction(self.handle, ctypes.byref(red)), "selr_plan_get_reduction")
        return {"gram": names.get(g.value, g.value), "ev_chunk": c.value, "jacobi_max_sweeps": w.value,
                "reduction": red.value}

    def set_tuning(self, gram, ev_chunk=0):
        """selr_plan_set_tuning: Gram mode (name as in Desc) and eigenvectors per pass (0, 8, 16)."""
        check(self.lib.selr_plan_set_tuning(self.handle, GRAM[gram], int(ev_chunk)), "selr_plan_set_tuning")
        self.desc.gram = gram

    def set_reduction(self, mode):
        """selr_plan_set_reduction: 0 by order, 1 one-stage, 2 two-stage (orders 48 .. 192)."""
        check(self.lib.selr_plan_set_reduction(self.handle, int(mode)), "selr_plan_set_reduction")

    STAGES = ("adjoint", "dc", "hybrid_fft", "lift", "gram", "svd", "apply")

    def profile(self, on=True):
        check(self.lib.selr_profile_enable(self.handle, 1 if on else 0), "selr_profile_enable")

    def profile_read(self):
        """{stage: (total_ms, iterations)} of the last profiled solve."""
        out = {}
        for k, name in enumerate(self.STAGES):
            ms, n = ctypes.c_float(), ctypes.c_int32()
            check(self.lib.selr_profile_read(self.handle, k, ctypes.byref(ms), ctypes.byref(n)), "selr_profile_read")
            out[name] = (ms.value, n.value)
        return out

    def lift_shape(self, axis):
        n, r, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(self.lib.selr_lift_shape(self.handle, AXES[axis], ctypes.byref(n), ctypes.byref(r), ctypes.byref(c)),
              "selr_lift_shape")
        return n.value, r.value, c.value


class BatchPlan(Plan):
    """A ``selr_plan`` for several 2D instances of uneven size (selr_plan_create_batch)."""

    def __init__(self, descs):
        self.lib = _lib.load()
        self.descs = list(descs)
        self.desc = self.descs[0]
        arr = (SelrDesc * len(self.descs))(*[d.to_c() for d in self.descs])
        h = ctypes.c_void_p()
        check(self.lib.selr_plan_create_batch(arr, len(self.descs), ctypes.byref(h)), "selr_plan_create_batch")
        self.handle = h

    @property
    def nK(self):
        return sum(d.L * d.J * d.M * d.N for d in self.descs)

    @property
    def n_mask(self):
        return sum(d.L * d.M * d.N for d in self.descs)

    def layout(self, i):
        """(k_offset, mask_offset) of instance i in the packed arrays."""
        k, m = ctypes.c_int64(), ctypes.c_int64()
        check(self.lib.selr_plan_instance_layout(self.handle, int(i), ctypes.byref(k), ctypes.byref(m)),
              "selr_plan_instance_layout")
        return k.value, m.value

    def pack(self, arrays, dtype, mask=False):
        """Concatenate per-instance tensors in the plan's packed order."""
        n = self.n_mask if mask else self.nK
        out = torch.empty(n, dtype=dtype, device=arrays[0].device)
        for i, a in enumerate(arrays):
            off = self.layout(i)[1 if mask else 0]
            out[off:off + a.numel()].copy_(a.reshape(-1))
        return out

    def unpack(self, packed, i):
        """View of instance i in a packed k-space / image array."""
        d = self.descs[i]
        off = self.layout(i)[0]
        return packed[off:off + d.L * d.J * d.M * d.N].view(d.J, d.M, d.N) if d.L == 1 else \
            packed[off:off + d.L * d.J * d.M * d.N].view(d.L, d.J, d.M, d.N)


def selr_solve_batch(plan: BatchPlan, Y, mask, X_out, state=None, resume=False, stream=None):
    """selr_solve on packed arrays of a batch plan; returns (iterations, largest relative change)."""
    it, rel = ctypes.c_int32(), ctypes.c_float()
    check(plan.lib.selr_solve(plan.handle, _ptr(Y, torch.complex64, "Y", plan.nK),
                              _ptr(mask, torch.uint8, "mask", plan.n_mask),
                              _ptr(X_out, torch.complex64, "X_out", plan.nK), _state_ptr(plan, state, resume),
                              1 if resume else 0, ctypes.byref(it), ctypes.byref(rel), _stream(stream)), "selr_solve")
    return it.value, rel.value


def selr_transform(plan: Plan, dim: int, inverse: bool, x, out, stream=None):
    check(plan.lib.selr_transform(plan.handle, dim, 1 if inverse else 0,
                                  _ptr(x, torch.complex64, "x", plan.nK), _ptr(out, torch.complex64, "out", plan.nK),
                                  _stream(stream)), "selr_transform")


def selr_lift(plan: Plan, axis: str, x, D, A_out, stream=None):
    n, r, c = plan.lift_shape(axis)
    check(plan.lib.selr_lift(plan.handle, AXES[axis], _ptr(x, torch.complex64, "x", plan.nK),
                             _ptr(D, torch.complex64, "D", n * r * c, allow_none=True),
                             _ptr(A_out, torch.complex64, "A_out", n * r * c), _stream(stream)), "selr_lift")


def selr_svt(plan: Plan, A, thresh: float, rank_out=None, stream=None):
    if A.dim() != 3:
        raise ValueError("A must be [nmat][rows][cols]")
    nmat, rows, cols = A.shape
    check(plan.lib.selr_svt(plan.handle, _ptr(A, torch.complex64, "A"), nmat, rows, cols, float(thresh),
                            _ptr(rank_out, torch.int32, "rank_out", nmat, allow_none=True), _stream(stream)),
          "selr_svt")


def _same_device(t, dev, name):
    if t is not None and isinstance(t, torch.Tensor) and t.device != dev:
        raise ValueError(f"{name} is on {t.device}, expected {dev}")


def selr_svt_noalloc(A, thresh: float, max_sweeps: int = 30, tol: float = 2.0e-6, rank_out=None, stream=None):
    """Allocation-free S_t of A [nmat][rows][cols] in place (no plan; fixed library scratch).

    The library resolves its scratch on the CURRENT device, so the call is made
    with A's device current and, by default, on that device's current stream."""
    lib = _lib.load()
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError("A must be a CUDA tensor")
    if A.dim() != 3:
        raise ValueError("A must be [nmat][rows][cols]")
    _same_device(rank_out, A.device, "rank_out")
    if stream is not None and stream.device != A.device:
        raise ValueError(f"stream is on {stream.device}, expected {A.device}")
    nmat, rows, cols = A.shape
    with torch.cuda.device(A.device):
        s = torch.cuda.current_stream(A.device) if stream is None else stream
        check(lib.selr_svt_noalloc(_ptr(A, torch.complex64, "A"), nmat, rows, cols, float(thresh),
                                   int(max_sweeps), float(tol),
                                   _ptr(rank_out, torch.int32, "rank_out", nmat, allow_none=True),
                                   ctypes.c_void_p(s.cuda_stream)), "selr_svt_noalloc")


def selr_svt_noalloc_status(device=None, stream=None) -> int:
    """Synchronise and return the condition of the last selr_svt_noalloc call on
    `device` (0 = SELR_OK, 4 = sweep cap reached, 5 = non-finite values)."""
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        s = torch.cuda.current_stream(dev) if stream is None else stream
        return int(lib.selr_svt_noalloc_status(ctypes.c_void_p(s.cuda_stream)))


def selr_adjoint(plan: Plan, axis: str, E, x_out, stream=None):
    n, r, c = plan.lift_shape(axis)
    check(plan.lib.selr_adjoint(plan.handle, AXES[axis], _ptr(E, torch.complex64, "E", n * r * c),
                                _ptr(x_out, torch.complex64, "x_out", plan.nK), _stream(stream)), "selr_adjoint")


def selr_dc(plan: Plan, Y, mask, adj_a, adj_b, K, rel_out=None, stream=None):
    d = plan.desc
    check(plan.lib.selr_dc(plan.handle, _ptr(Y, torch.complex64, "Y", plan.nK),
                           _ptr(mask, torch.uint8, "mask", d.L * d.M * d.N),
                           _ptr(adj_a, torch.complex64, "adj_a", plan.nK), _ptr(adj_b, torch.complex64, "adj_b", plan.nK),
                           _ptr(K, torch.complex64, "K", plan.nK),
                           _ptr(rel_out, torch.float32, "rel_out", 1, allow_none=True), _stream(stream)), "selr_dc")


def selr_state_bytes(plan: Plan) -> int:
    n = ctypes.c_size_t()
    check(plan.lib.selr_state_bytes(plan.handle, ctypes.byref(n)), "selr_state_bytes")
    return int(n.value)


def new_state(plan: Plan, device=None):
    """A device buffer for selr_solve's checkpoint (uint8, selr_state_bytes long)."""
    return torch.empty(selr_state_bytes(plan), dtype=torch.uint8, device=device or "cuda")


def _state_ptr(plan, state, resume):
    if state is None:
        if resume:
            raise ValueError("resume needs a state buffer")
        return None
    return _ptr(state, torch.uint8, "state", selr_state_bytes(plan))


def selr_solve(plan: Plan, Y, mask, X_out, state=None, resume=False, stream=None):
    """Run the reconstruction; returns (iterations, last relative change).

    state: optional uint8 device buffer (new_state) that receives the final
    checkpoint; resume=True starts from the checkpoint it holds."""
    d = plan.desc
    it, rel = ctypes.c_int32(), ctypes.c_float()
    check(plan.lib.selr_solve(plan.handle, _ptr(Y, torch.complex64, "Y", plan.nK),
                              _ptr(mask, torch.uint8, "mask", d.L * d.M * d.N),
                              _ptr(X_out, torch.complex64, "X_out", plan.nK), _state_ptr(plan, state, resume),
                              1 if resume else 0, ctypes.byref(it), ctypes.byref(rel), _stream(stream)), "selr_solve")
    return it.value, rel.value


def selr_plan_rank_sums(plan: Plan, stream=None):
    """(per-matrix rank sums over the last solve as a numpy int64 array, iterations)."""
    import numpy as np
    fams = ("row", "col") if plan.desc.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV") else ("pe", "param")
    n = sum(plan.lift_shape(a)[0] for a in fams) if not isinstance(plan, BatchPlan) else None
    if n is None:
        raise ValueError("rank sums of a batch plan: use the instance plans")
    out = np.zeros(n, dtype=np.int64)
    it = ctypes.c_int32()
    check(plan.lib.selr_plan_rank_sums(plan.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n,
                                       ctypes.byref(it), _stream(stream)), "selr_plan_rank_sums")
    return out, it.value


def selr_probe_fp32_peak(packed=False, iters=4096):
    """Measured FP32 FMA rate of the current device: (TFLOP/s, ms of the timed launch)."""
    lib = _lib.load()
    tf, ms = ctypes.c_float(), ctypes.c_float()
    check(lib.selr_probe_fp32_peak(1 if packed else 0, int(iters), ctypes.byref(tf), ctypes.byref(ms)),
          "selr_probe_fp32_peak")
    return tf.value, ms.value


def selr_sync_status(plan: Plan, stream=None) -> int:
    """Synchronise and return the device-side status code (0 = SELR_OK)."""
    return int(plan.lib.selr_sync_status(plan.handle, _stream(stream)))


def selr_selftest_wait(set_flag: bool, limit_us: int) -> int:
    """Run the eigensolver's bounded hand-off wait on a flag the host set (or did
    not set); returns the status code (0 = consumed, 6 = SELR_ERR_TIMEOUT)."""
    return int(_lib.load().selr_selftest_wait(1 if set_flag else 0, int(limit_us)))


# ------------------------------------------------------------- reverse mode
def selr_svt_vjp(plan: Plan, A, Zbar, thresh: float, Abar, tbar, Z_out=None, stream=None):
    """Abar <- VJP of S_t at A for cotangent Zbar; tbar (device float32[1]) <- dL/dt;
    Z_out (optional) <- S_t(A)."""
    if A.dim() != 3:
        raise ValueError("A must be [nmat][rows][cols]")
    nmat, rows, cols = A.shape
    n = A.numel()
    check(plan.lib.selr_svt_vjp(plan.handle, _ptr(A, torch.complex64, "A"), _ptr(Zbar, torch.complex64, "Zbar", n),
                                nmat, rows, cols, float(thresh), _ptr(Abar, torch.complex64, "Abar", n),
                                _ptr(tbar, torch.float32, "tbar", 1),
                                _ptr(Z_out, torch.complex64, "Z_out", n, allow_none=True), _stream(stream)),
          "selr_svt_vjp")


def selr_dc_vjp(plan: Plan, mask, Kbar, adj_out, Ybar=None, stream=None):
    d = plan.desc
    check(plan.lib.selr_dc_vjp(plan.handle, _ptr(mask, torch.uint8, "mask", d.L * d.M * d.N),
                               _ptr(Kbar, torch.complex64, "Kbar", plan.nK),
                               _ptr(adj_out, torch.complex64, "adj_out", plan.nK),
                               _ptr(Ybar, torch.complex64, "Ybar", plan.nK, allow_none=True), _stream(stream)),
          "selr_dc_vjp")


def selr_axpby(out, a, x, b=0.0, y=None, c=0.0, z=None, stream=None):
    """out = a x + b y + c z (complex64 device arrays of equal size)."""
    lib = _lib.load()
    n = x.numel()
    check(lib.selr_axpby(n, float(a), _ptr(x, torch.complex64, "x"), float(b),
                         _ptr(y, torch.complex64, "y", n, allow_none=True), float(c),
                         _ptr(z, torch.complex64, "z", n, allow_none=True), _ptr(out, torch.complex64, "out", n),
                         _stream(stream)), "selr_axpby")


def selr_dot_re(plan: Plan, x, y, out, stream=None):
    """out (device float32[1]) <- Re sum conj(x) y."""
    n = x.numel()
    check(plan.lib.selr_dot_re(plan.handle, n, _ptr(x, torch.complex64, "x"), _ptr(y, torch.complex64, "y", n),
                               _ptr(out, torch.float32, "out", 1), _stream(stream)), "selr_dot_re")


# ------------------------------------------------------------- evaluation
def selr_ssos(X, stream=None):
    """SSOS over coils of X [J][M][N] or [L][J][M][N] complex64 -> float32 [M][N] or [L][M][N]."""
    lib = _lib.load()
    if X.dim() not in (3, 4):
        raise ValueError("X must be [J][M][N] or [L][J][M][N]")
    nb, J = (1, X.shape[0]) if X.dim() == 3 else (X.shape[0], X.shape[1])
    npix = X.shape[-1] * X.shape[-2]
    out = torch.empty((nb,) + tuple(X.shape[-2:]), dtype=torch.float32, device=X.device)
    check(lib.selr_ssos(_ptr(X, torch.complex64, "X"), nb, J, npix, _ptr(out, torch.float32, "out"), _stream(stream)),
          "selr_ssos")
    return out[0] if X.dim() == 3 else out


def selr_rlne(x, xhat, stream=None):
    """RLNE of xhat against x (float32 device tensors of equal size) -> device float32[1]."""
    lib = _lib.load()
    out = torch.empty(1, dtype=torch.float32, device=x.device)
    check(lib.selr_rlne(_ptr(x, torch.float32, "x"), _ptr(xhat, torch.float32, "xhat", x.numel()), x.numel(),
                        _ptr(out, torch.float32, "out"), _stream(stream)), "selr_rlne")
    return out


def selr_max(v, stream=None):
    lib = _lib.load()
    out = torch.empty(1, dtype=torch.float32, device=v.device)
    check(lib.selr_max(_ptr(v, torch.float32, "v"), v.numel(), _ptr(out, torch.float32, "out"), _stream(stream)),
          "selr_max")
    return out


def selr_mssim(A, B, L=None, stream=None):
    """MSSIM of reference A and image B (float32 [M][N] device tensors) -> (device float32[1], SSIM map)."""
    lib = _lib.load()
    M, N = A.shape
    if L is None:
        L = float(selr_max(A, stream).item())
    smap = torch.empty((M - 10, N - 10), dtype=torch.float32, device=A.device)
    out = torch.empty(1, dtype=torch.float32, device=A.device)
    check(lib.selr_mssim(_ptr(A, torch.float32, "A"), _ptr(B, torch.float32, "B", A.numel()), M, N, float(L),
                         _ptr(smap, torch.float32, "ssim_map"), _ptr(out, torch.float32, "out"), _stream(stream)),
          "selr_mssim")
    return out, smap


def selr_t2_fit(S, te_ms, t2_min=1.0, t2_max=1000.0, stream=None):
    """Pixelwise T2 fit of magnitudes S [L][...] (float32 device) at echo times te_ms -> (T2, M0)."""
    lib = _lib.load()
    L = S.shape[0]
    npix = S.numel() // L
    te = (ctypes.c_float * L)(*[float(t) for t in te_ms])
    T2 = torch.empty(S.shape[1:], dtype=torch.float32, device=S.device)
    M0 = torch.empty_like(T2)
    check(lib.selr_t2_fit(_ptr(S, torch.float32, "S"), te, L, npix, float(t2_min), float(t2_max),
                          _ptr(T2, torch.float32, "T2"), _ptr(M0, torch.float32, "M0"), _stream(stream)),
          "selr_t2_fit")
    return T2, M0


def selr_spirit_calibrate(plan: Plan, Y, stream=None):
    """Calibrate the plan's SPIRiT kernel from the ACS rows of Y [J][M][N] (SHLR-S / SHLR-SV plans)."""
    check(plan.lib.selr_spirit_calibrate(plan.handle, _ptr(Y, torch.complex64, "Y", plan.nK), _stream(stream)),
          "selr_spirit_calibrate")


def selr_spirit_kernel(plan: Plan, stream=None):
    """The calibrated SPIRiT kernel [J][J][ks][ks] complex64."""
    d = plan.desc
    g = torch.empty((d.J, d.J, d.spirit_k, d.spirit_k), dtype=torch.complex64, device="cuda")
    check(plan.lib.selr_spirit_kernel(plan.handle, _ptr(g, torch.complex64, "g"), _stream(stream)),
          "selr_spirit_kernel")
    return g


# ------------------------------------------------------- unrolled forward
def selr_lifted_elems(plan: Plan) -> int:
    n = ctypes.c_int64()
    check(plan.lib.selr_lifted_elems(plan.handle, ctypes.byref(n)), "selr_lifted_elems")
    return int(n.value)


def selr_solve_unrolled(plan: Plan, Y, mask, X_out, ts, taus, ckpt_K=None, ckpt_D=None, stream=None):
    """Unrolled forward with per-iteration thresholds ts and steps taus (host sequences)."""
    n = len(ts)
    if len(taus) != n:
        raise ValueError("ts and taus must have the same length")
    nm = plan.n_mask if isinstance(plan, BatchPlan) else plan.desc.L * plan.desc.M * plan.desc.N
    tsa = (ctypes.c_float * n)(*[float(t) for t in ts])
    taa = (ctypes.c_float * n)(*[float(t) for t in taus])
    le = selr_lifted_elems(plan)
    check(plan.lib.selr_solve_unrolled(plan.handle, _ptr(Y, torch.complex64, "Y", plan.nK),
                                       _ptr(mask, torch.uint8, "mask", nm), _ptr(X_out, torch.complex64, "X", plan.nK),
                                       tsa, taa, n, _ptr(ckpt_K, torch.complex64, "ckpt_K", n * plan.nK, True),
                                       _ptr(ckpt_D, torch.complex64, "ckpt_D", n * le, True), _stream(stream)),
          "selr_solve_unrolled")


def selr_lifted_unpack(plan: Plan, packed, inst: int, axis: str, out, stream=None):
    """Family `axis` of instance `inst` out of a packed multiplier array into out [nmat][rows][cols]."""
    check(plan.lib.selr_lifted_unpack(plan.handle, _ptr(packed, torch.complex64, "packed"), int(inst), AXES[axis],
                                      _ptr(out, torch.complex64, "out"), _stream(stream)), "selr_lifted_unpack")
