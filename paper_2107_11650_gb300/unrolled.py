"""Unrolled SHLR / SHLR-V reconstruction with learnable per-iteration SVT
thresholds t_k and multiplier steps tau_k, differentiable by a hand-written
reverse pass (wrapped in ``torch.autograd.Function``).

Forward: n iterations of Algorithm S1 in the paper's order (X-update of
Eq. 15, Z = S_{t_k} of Eqs. 16-17, D-update of Eqs. 13-14 with step tau_k),
each step a call into libselr: the lift adjoints (selr_adjoint), the
k-space divide (selr_dc), the hybrid transforms (selr_transform), the lifts
(selr_lift), the SVT (selr_svt) and the multiplier arithmetic (selr_axpby).
With t_k = 1/beta and tau_k = tau the result is that of selr_solve.  The
output is the image X = F2D* K of the last X-update.

Memory: per iteration only (K_k, D_row, D_col) are kept (the multipliers
entering iteration k and the k-space iterate it produced); the lifted
matrices are recomputed in the reverse pass from them, and the SVT result Z
comes out of the SVT derivative call itself (selr_svt_vjp), so the reverse
pass runs one eigensolve per lifted matrix, like the forward.

Reverse, per iteration k from the last (cotangents Dbar_k, Ebar_k of the
multiplier and of E_k = Z_k - D_k / beta):
    Dp = Dbar_k - Ebar_k / beta,       Zbar = Ebar_k - tau_k Dp,
    taubar_k = Re <Dp, A - D / beta - Z>,
    Abar = SVT-VJP(A, Zbar) + tau_k Dp (selr_svt_vjp, also giving tbar_k),
    Dbar_{k-1} = (1 - tau_k / beta) Dp + Abar / beta,
    Kbar_k = F_m L_row^T Abar_row + F_n L_col^T Abar_col,
    Ebar_{k-1} = L (F* (beta Kbar_k / den)),   Ybar += lambda U Kbar_k / den
(selr_dc_vjp gives the last line's k-space factors; the last iteration only
contributes through K).
"""
from __future__ import annotations

import torch

from . import api
from .api import Desc, Plan

_C64 = torch.complex64


class Unrolled2D:
    """Forward / reverse engine for one SHLR or SHLR-V problem size."""

    def __init__(self, desc: Desc, mask, n_iter: int):
        if desc.model not in ("SHLR", "SHLR_V"):
            raise ValueError("unrolled reconstruction is defined for the 2D models SHLR and SHLR_V")
        if n_iter < 1:
            raise ValueError("n_iter must be >= 1")
        self.desc = desc
        self.plan = Plan(desc)
        self.n_iter = int(n_iter)
        self.mask = mask.reshape(desc.M, desc.N).contiguous()
        if self.mask.dtype != torch.uint8 or not self.mask.is_cuda:
            raise TypeError("mask must be a CUDA uint8 tensor [M][N]")
        self.dev = self.mask.device
        self.shape = (desc.J, desc.M, desc.N)
        self.lift = {ax: self.plan.lift_shape(ax) for ax in ("row", "col")}
        # hybrid transform dimension feeding each family (row: along M, col: along N)
        self.dim = {"row": 0, "col": 1}

    def _empty(self, shape):
        return torch.empty(shape, dtype=_C64, device=self.dev)

    def _zeros(self, shape):
        return torch.zeros(shape, dtype=_C64, device=self.dev)

    @staticmethod
    def _scalars(v, n, name):
        vals = [float(x) for x in v.detach().reshape(-1).cpu().tolist()]
        if len(vals) != n:
            raise ValueError(f"{name} must have {n} entries")
        return vals

    # ---------------------------------------------------------------- forward
    def _lifts(self, K, D):
        """A = lift(F* K) + D / beta for both families."""
        out = {}
        for ax in ("row", "col"):
            x = self._empty(self.shape)
            api.selr_transform(self.plan, self.dim[ax], True, K, x)
            A = self._empty(self.lift[ax])
            api.selr_lift(self.plan, ax, x, D[ax], A)
            out[ax] = A
        return out

    def _z_and_d(self, K, D, t, tau):
        """A = lift(F* K) + D / beta and Z = S_t(A) for both families."""
        A = self._lifts(K, D)
        out = {}
        for ax in ("row", "col"):
            Z = self._empty(self.lift[ax])
            api.selr_axpby(Z, 1.0, A[ax])
            api.selr_svt(self.plan, Z, t)
            out[ax] = (A[ax], Z)
        return out

    def _x_update(self, Y, E):
        adj = {}
        for ax in ("row", "col"):
            adj[ax] = self._empty(self.shape)
            api.selr_adjoint(self.plan, ax, E[ax], adj[ax])
        K = self._zeros(self.shape)
        api.selr_dc(self.plan, Y, self.mask, adj["row"], adj["col"], K)
        return K

    def forward(self, Y, ts, taus):
        """Returns (X, checkpoints); checkpoints[k] = (K_k, {axis: D entering iteration k})."""
        n, beta, d0 = self.n_iter, self.desc.beta, self.desc.d_init
        tv, tauv = self._scalars(ts, n, "ts"), self._scalars(taus, n, "taus")
        if min(tv) < 0.0:
            raise ValueError("thresholds must be >= 0")
        D = {ax: torch.full(self.lift[ax], d0, dtype=_C64, device=self.dev) for ax in ("row", "col")}
        E = {ax: torch.full(self.lift[ax], -d0 / beta, dtype=_C64, device=self.dev) for ax in ("row", "col")}
        ckpts = []
        K = None
        for k in range(n):
            K = self._x_update(Y, E)
            ckpts.append((K, D))
            if k == n - 1:
                break
            zs = self._z_and_d(K, D, tv[k], tauv[k])
            Dn, En = {}, {}
            for ax in ("row", "col"):
                A, Z = zs[ax]
                Dn[ax] = self._empty(self.lift[ax])
                api.selr_axpby(Dn[ax], 1.0 - tauv[k] / beta, D[ax], tauv[k], A, -tauv[k], Z)
                En[ax] = self._empty(self.lift[ax])
                api.selr_axpby(En[ax], 1.0, Z, -1.0 / beta, Dn[ax])
            D, E = Dn, En
        tmp = self._empty(self.shape)
        X = self._empty(self.shape)
        api.selr_transform(self.plan, 0, True, K, tmp)
        api.selr_transform(self.plan, 1, True, tmp, X)
        return X, ckpts

    # ---------------------------------------------------------------- reverse
    def backward(self, ckpts, Y, ts, taus, Xbar):
        """Returns (Ybar, tbar, taubar) for the cotangent Xbar of X."""
        n, beta = self.n_iter, self.desc.beta
        tv, tauv = self._scalars(ts, n, "ts"), self._scalars(taus, n, "taus")
        g_t = torch.zeros((n, 2), dtype=torch.float32, device=self.dev)
        g_tau = torch.zeros((n, 2), dtype=torch.float32, device=self.dev)
        Xbar = Xbar.to(_C64).contiguous()
        tmp = self._empty(self.shape)
        Kbar = self._empty(self.shape)
        api.selr_transform(self.plan, 0, False, Xbar, tmp)     # adjoint of F2D* is F2D
        api.selr_transform(self.plan, 1, False, tmp, Kbar)
        Ybar = self._zeros(self.shape)
        Dbar = Ebar = None
        for k in range(n - 1, -1, -1):
            K, D = ckpts[k]
            if k < n - 1:
                A = self._lifts(K, D)
                Kbar = self._zeros(self.shape)
                Dprev = {}
                for f, ax in enumerate(("row", "col")):
                    shp = self.lift[ax]
                    Dp = self._empty(shp)
                    api.selr_axpby(Dp, 1.0, Dbar[ax], -1.0 / beta, Ebar[ax])
                    Zb = self._empty(shp)
                    api.selr_axpby(Zb, 1.0, Ebar[ax], -tauv[k], Dp)
                    Ab = self._empty(shp)
                    Z = self._empty(shp)
                    api.selr_svt_vjp(self.plan, A[ax], Zb, tv[k], Ab, g_t[k, f:f + 1], Z_out=Z)
                    R = self._empty(shp)
                    api.selr_axpby(R, 1.0, A[ax], -1.0 / beta, D[ax], -1.0, Z)
                    api.selr_dot_re(self.plan, Dp, R, g_tau[k, f:f + 1])
                    api.selr_axpby(Ab, 1.0, Ab, tauv[k], Dp)
                    Dprev[ax] = self._empty(shp)
                    api.selr_axpby(Dprev[ax], 1.0 - tauv[k] / beta, Dp, 1.0 / beta, Ab)
                    xb = self._empty(self.shape)
                    api.selr_adjoint(self.plan, ax, Ab, xb)
                    api.selr_transform(self.plan, self.dim[ax], False, xb, xb)
                    api.selr_axpby(Kbar, 1.0, Kbar, 1.0, xb)
                Dbar = Dprev
            else:
                Dbar = {ax: self._zeros(self.lift[ax]) for ax in ("row", "col")}
            # X-update of iteration k
            Sb = self._empty(self.shape)
            Yb = self._empty(self.shape)
            api.selr_dc_vjp(self.plan, self.mask, Kbar, Sb, Yb)
            api.selr_axpby(Ybar, 1.0, Ybar, 1.0, Yb)
            Ebar = {}
            for ax in ("row", "col"):
                a = self._empty(self.shape)
                api.selr_transform(self.plan, self.dim[ax], True, Sb, a)
                Ebar[ax] = self._empty(self.lift[ax])
                api.selr_lift(self.plan, ax, a, None, Ebar[ax])
        return Ybar, g_t.sum(dim=1), g_tau.sum(dim=1)


class UnrolledFunction(torch.autograd.Function):
    """X = unrolled reconstruction(Y; t_1..t_n, tau_1..tau_n)."""

    @staticmethod
    def forward(ctx, Y, ts, taus, engine):
        Yc = Y.detach().to(_C64).contiguous()
        X, ckpts = engine.forward(Yc, ts, taus)
        ctx.engine = engine
        ctx.ckpts = ckpts
        ctx.save_for_backward(Yc, ts.detach(), taus.detach())
        return X

    @staticmethod
    def backward(ctx, Xbar):
        Yc, ts, taus = ctx.saved_tensors
        Ybar, tbar, taubar = ctx.engine.backward(ctx.ckpts, Yc, ts, taus, Xbar)
        ctx.ckpts = None
        return (Ybar if ctx.needs_input_grad[0] else None,
                tbar.to(ts.dtype).to(ts.device) if ctx.needs_input_grad[1] else None,
                taubar.to(taus.dtype).to(taus.device) if ctx.needs_input_grad[2] else None,
                None)


class UnrolledSHLR(torch.nn.Module):
    """Unrolled SHLR / SHLR-V with learnable t_k (init 1/beta) and tau_k (init tau)."""

    def __init__(self, desc: Desc, mask, n_iter: int):
        super().__init__()
        self.engine = Unrolled2D(desc, mask, n_iter)
        dev = self.engine.dev
        self.ts = torch.nn.Parameter(torch.full((n_iter,), 1.0 / desc.beta, dtype=torch.float32, device=dev))
        self.taus = torch.nn.Parameter(torch.full((n_iter,), desc.tau, dtype=torch.float32, device=dev))

    def forward(self, Y):
        return UnrolledFunction.apply(Y, self.ts, self.taus, self.engine)


class _BatchCheckpoints:
    """Checkpoints of one instance of a batched unrolled forward: (K_k, {axis: D_k}),
    the multipliers unpacked from the batch plan's layout when an iteration is
    reached in the reverse pass."""

    def __init__(self, bplan, ckK, ckD, inst, engine):
        self.bplan, self.ckK, self.ckD, self.inst, self.engine = bplan, ckK, ckD, inst, engine

    def __len__(self):
        return self.ckK.shape[0]

    def __getitem__(self, k):
        K = self.bplan.unpack(self.ckK[k], self.inst)
        D = {}
        for ax in ("row", "col"):
            D[ax] = torch.empty(self.engine.lift[ax], dtype=_C64, device=self.engine.dev)
            api.selr_lifted_unpack(self.bplan, self.ckD[k], self.inst, ax, D[ax])
        return K, D


class UnrolledBatchFunction(torch.autograd.Function):
    """(X_1, ..., X_B) = unrolled reconstruction of B instances (shared t_k, tau_k)
    in one batched plan; reverse pass per instance."""

    @staticmethod
    def forward(ctx, ts, taus, module, *Ys):
        bp = module.bplan
        n = module.n_iter
        Yp = bp.pack([y.detach().to(_C64).contiguous() for y in Ys], _C64)
        Xp = torch.empty_like(Yp)
        ckK = torch.empty((n, bp.nK), dtype=_C64, device=Yp.device)
        ckD = torch.empty((n, api.selr_lifted_elems(bp)), dtype=_C64, device=Yp.device)
        tv = [float(x) for x in ts.detach().cpu().tolist()]
        tauv = [float(x) for x in taus.detach().cpu().tolist()]
        if min(tv) < 0.0:
            raise ValueError("thresholds must be >= 0")
        api.selr_solve_unrolled(bp, Yp, module.mask_p, Xp, tv, tauv, ckK, ckD, stream=module.stream)
        torch.cuda.current_stream().wait_stream(module.stream)
        ctx.module = module
        ctx.ck = (ckK, ckD)
        ctx.Ys = [y.detach().to(_C64).contiguous() for y in Ys]
        ctx.save_for_backward(ts.detach(), taus.detach())
        return tuple(bp.unpack(Xp, i).clone() for i in range(len(Ys)))

    @staticmethod
    def backward(ctx, *Xbars):
        ts, taus = ctx.saved_tensors
        m = ctx.module
        ckK, ckD = ctx.ck
        tbar = torch.zeros_like(ts)
        taubar = torch.zeros_like(taus)
        Ybars = []
        for i, (e, Xb) in enumerate(zip(m.engines, Xbars)):
            if Xb is None:
                Ybars.append(None)
                continue
            ck = _BatchCheckpoints(m.bplan, ckK, ckD, i, e)
            Yb, tb, taub = e.backward(ck, ctx.Ys[i], ts, taus, Xb)
            tbar += tb.to(ts.dtype)
            taubar += taub.to(taus.dtype)
            Ybars.append(Yb)
        ctx.ck = None
        return (tbar, taubar, None, *Ybars)


class UnrolledBatch(torch.nn.Module):
    """A batch of unrolled reconstructions of uneven sizes sharing t_k and tau_k.

    The forward runs every instance in one batched plan (selr_plan_create_batch:
    the lifted matrices of all instances share the SVT launches) as one
    CUDA graph (selr_solve_unrolled) and keeps (K_k, D_k) per iteration; the
    reverse pass runs per instance on its own plan from those checkpoints."""

    def __init__(self, descs, masks, n_iter: int):
        super().__init__()
        if not descs or len(descs) != len(masks):
            raise ValueError("one mask per description is required")
        if len({(d.beta, d.tau) for d in descs}) != 1:
            raise ValueError("instances sharing t_k, tau_k must share beta and tau")
        self.n_iter = int(n_iter)
        self.engines = [Unrolled2D(d, m, n_iter) for d, m in zip(descs, masks)]
        self.bplan = api.BatchPlan(list(descs))
        self.mask_p = self.bplan.pack([e.mask for e in self.engines], torch.uint8, mask=True)
        dev = self.engines[0].dev
        self.stream = torch.cuda.Stream(device=dev)
        self.ts = torch.nn.Parameter(torch.full((n_iter,), 1.0 / descs[0].beta, dtype=torch.float32, device=dev))
        self.taus = torch.nn.Parameter(torch.full((n_iter,), descs[0].tau, dtype=torch.float32, device=dev))

    def forward(self, Ys):
        if len(Ys) != len(self.engines):
            raise ValueError("one k-space array per instance is required")
        self.stream.wait_stream(torch.cuda.current_stream())
        return list(UnrolledBatchFunction.apply(self.ts, self.taus, self, *Ys))
