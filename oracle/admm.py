"""ADMM for SHLR / SHLR-V (Algorithm S1) and SHLR-P / SHLR-VP (Algorithm S2).

Test infrastructure only (see ``oracle/__init__.py``).

Scaled-form ADMM exactly as the paper orders it: X-update (Eq. 15, or S7 for
the parameter models), Z-update by SVT (Eqs. 16-17 / S8-S9), multiplier
update (Eqs. 13-14 / S5-S6).  Initialisation Z = 0, D = d_init (the paper
writes D = 1, taken literally as every entry 1 + 0i).  X^(1) is taken as the
zero-filled reconstruction F* Y, which only enters the first value of the
stopping ratio ||X^(k+1) - X^(k)||^2 / ||X^(k)||^2.

Readings (the paper is silent or garbled at these points):
* SHLR-S / SHLR-SV (Eq. 3 / Eq. 6) add lambda_1/2 ||X - G X||^2 with the
  SPIRiT operator G of oracle/spirit.py; their X-update is solved by CG
  (see there).  The other models have no G term.
* Eq. 15 without the G term is diagonal in 2D k-space: the row-lift normal
  operator is diag(d_r(k_n)), the column-lift one diag(d_c(k_m)), with
  d(k) = c(k)|w(k)|^2 [+ c(N-1-k)|w(N-1-k)|^2 for the VC channels], and the
  data term is lambda*U.  The pointwise divide is cross-checked against a
  dense normal-equation solve built from the image-domain operators of
  Eq. 2 / Eq. 4 (:func:`dense_x_update_2d`).
* lambda <= 0 means hard data consistency (lambda -> infinity).
* Eq. S6 omits "vc" and Eq. S7 writes R_n*: read as H~_vc (as in Eq. 8) and P_n*.
* Sub-problems written as "min" (Eqs. 10-12, S2-S4) are read as argmin over
  the variable being updated.
"""
from __future__ import annotations

import numpy as np

from .transforms import fftc, ifftc, ifft2c, filter_weights, hankel_multiplicity
from .hankel import (lift_rows, lift_rows_adjoint, lift_cols, lift_cols_adjoint,
                     lift_pe, lift_pe_adjoint, lift_param, lift_param_adjoint,
                     lift_vectors)
from .svt import svt, nuclear_norm
from . import spirit


def normal_weights(N, p, w, vc):
    """Diagonal of sum_lifts (H W)^T (H W) in the lift's Fourier domain.

    Plain channel: c(k)|w(k)|^2.  VC channel (real-linear, see hankel.py):
    c(N-1-k)|w(N-1-k)|^2.  c = Hankel multiplicities."""
    c = hankel_multiplicity(N, p)
    d = c * np.abs(w) ** 2
    if vc:
        d = d + (c * np.abs(w) ** 2)[::-1]
    return d


def _dc_divide(lam, U, Y, rhs_b, den_b):
    """Pointwise solve (lam*U + den_b) K = lam*U*Y + rhs_b.  lam <= 0: hard data
    consistency (K = Y where sampled).  A point with a zero left-hand side
    (unsampled and unseen by every lift, e.g. k-space DC when W kills it) is
    unconstrained; the minimum-norm reading sets it to 0."""
    if lam > 0:
        num = lam * U * Y + rhs_b
        den = lam * U + den_b
    else:
        num, den = rhs_b, den_b
    safe = np.where(den != 0, den, 1.0)
    K = np.where(den != 0, num / safe, 0.0)
    if lam <= 0:
        K = np.where(U > 0, Y, K)
    return K


def _params(cfg):
    return dict(model=cfg.model, p=cfg.window, pP=cfg.window_param, weight=cfg.weight,
                lam=float(cfg.lam), lam2=float(cfg.lam2), beta=float(cfg.beta),
                tau=float(cfg.tau), d0=float(cfg.d_init), lam1=float(getattr(cfg, "lam1", 0.0)),
                ks=int(getattr(cfg, "spirit_k", 5)), reg=float(getattr(cfg, "spirit_reg", 1e-3)),
                n_acs=int(getattr(cfg, "n_acs", 0)))


# =========================================================== Algorithm S1
class Shlr2D:
    """SHLR (Eq. 2) / SHLR-V (Eq. 5) / SHLR-S (Eq. 3) / SHLR-SV (Eq. 6) solved
    by Algorithm S1."""

    def __init__(self, Y, U, cfg):
        self.Y = np.asarray(Y, dtype=np.complex128)
        self.U = np.asarray(U).astype(np.float64)
        P = _params(cfg)
        self.P = P
        self.vc = P["model"] in ("SHLR_V", "SHLR_SV")
        self.spirit = P["model"] in ("SHLR_S", "SHLR_SV")
        if self.spirit:
            if not P["lam"] > 0:
                raise ValueError("SHLR-S / SHLR-SV need a finite lambda")
            self.g = spirit.calibrate(self.Y, P["n_acs"], P["ks"], P["reg"])
        J, M, N = self.Y.shape
        self.J, self.M, self.N = J, M, N
        p = P["p"]
        self.C = 2 * J if self.vc else J
        self.wN = filter_weights(N, P["weight"])
        self.wM = filter_weights(M, P["weight"])
        self.d_r = normal_weights(N, p, self.wN, self.vc)
        self.d_c = normal_weights(M, p, self.wM, self.vc)

    # -- state ------------------------------------------------------------
    def init_state(self):
        J, M, N, C, p = self.J, self.M, self.N, self.C, self.P["p"]
        d0 = self.P["d0"]
        Dr = np.full((M, N - p + 1, C * p), d0, dtype=np.complex128)
        Dc = np.full((N, M - p + 1, C * p), d0, dtype=np.complex128)
        return dict(K=self.Y.copy(), Zr=np.zeros_like(Dr), Zc=np.zeros_like(Dc), Dr=Dr, Dc=Dc)

    # -- operators --------------------------------------------------------
    def lifts(self, K):
        """Row and column lifts of X = F2D* K (Eq. 2 / Eq. 4)."""
        p = self.P["p"]
        R = ifftc(K, axis=1)          # F^1D along n of each image row
        Cc = ifftc(K, axis=2)         # F^1D along m of each image column
        return lift_rows(R, self.wN, p, self.vc), lift_cols(Cc, self.wM, p, self.vc)

    def x_update(self, Zr, Zc, Dr, Dc, K0=None):
        """Eq. 15: without G a pointwise divide in 2D k-space; with G (SHLR-S /
        SHLR-SV) conjugate gradients on the normal equations from K0."""
        P = self.P
        b, lam, p = P["beta"], P["lam"], P["p"]
        a_row = lift_rows_adjoint(Zr - Dr / b, self.wN, p, self.vc, self.J, self.N)
        a_col = lift_cols_adjoint(Zc - Dc / b, self.wM, p, self.vc, self.J, self.M)
        rhs_b = b * (fftc(a_row, axis=1) + fftc(a_col, axis=2))
        den_b = b * (self.d_r[None, None, :] + self.d_c[None, :, None])
        U = self.U[None]
        if not self.spirit:
            return _dc_divide(lam, U, self.Y, rhs_b, den_b)
        diag = lam * U + den_b
        rhs = lam * U * self.Y + rhs_b
        x0 = self.Y.copy() if K0 is None else K0
        K, _ = spirit.cg(lambda x: spirit.normal_op(x, diag, P["lam1"], self.g), rhs, x0)
        return K

    def z_update(self, LXr, LXc, Dr, Dc):
        t = 1.0 / self.P["beta"]
        return svt(LXr + Dr / self.P["beta"], t), svt(LXc + Dc / self.P["beta"], t)

    def d_update(self, LXr, LXc, Zr, Zc, Dr, Dc):
        tau = self.P["tau"]
        return Dr + tau * (LXr - Zr), Dc + tau * (LXc - Zc)

    def lagrangian(self, K, Zr, Zc, Dr, Dc):
        """Scaled augmented Lagrangian of Eq. 9 without G, up to the constant
        -sum ||D||^2 / (2 beta)."""
        P = self.P
        b, lam = P["beta"], P["lam"]
        LXr, LXc = self.lifts(K)
        val = 0.5 * lam * np.sum(np.abs(self.U[None] * (self.Y - K)) ** 2) if lam > 0 else 0.0
        if self.spirit:
            val += 0.5 * P["lam1"] * np.sum(np.abs(spirit.apply_g(K, self.g) - K) ** 2)
        val += nuclear_norm(Zr).sum() + nuclear_norm(Zc).sum()
        val += 0.5 * b * np.sum(np.abs(LXr - Zr + Dr / b) ** 2)
        val += 0.5 * b * np.sum(np.abs(LXc - Zc + Dc / b) ** 2)
        return float(val)

    def objective(self, K):
        """Eq. 2 / Eq. 5 objective (nuclear norms + lambda/2 data term)."""
        LXr, LXc = self.lifts(K)
        val = nuclear_norm(LXr).sum() + nuclear_norm(LXc).sum()
        if self.P["lam"] > 0:
            val += 0.5 * self.P["lam"] * np.sum(np.abs(self.U[None] * (self.Y - K)) ** 2)
        if self.spirit:
            val += 0.5 * self.P["lam1"] * np.sum(np.abs(spirit.apply_g(K, self.g) - K) ** 2)
        return float(val)

    # -- Algorithm S1 -----------------------------------------------------
    def step(self, st):
        """One pass of the while-loop body: X, then Z, then D."""
        K = self.x_update(st["Zr"], st["Zc"], st["Dr"], st["Dc"], K0=st["K"])
        rel = np.sum(np.abs(K - st["K"]) ** 2) / np.sum(np.abs(st["K"]) ** 2)
        LXr, LXc = self.lifts(K)
        Zr, Zc = self.z_update(LXr, LXc, st["Dr"], st["Dc"])
        Dr, Dc = self.d_update(LXr, LXc, Zr, Zc, st["Dr"], st["Dc"])
        return dict(K=K, Zr=Zr, Zc=Zc, Dr=Dr, Dc=Dc), float(rel)

    def run(self, n_iter, tol=-1.0, state=None):
        st = self.init_state() if state is None else state
        rels = []
        for _ in range(n_iter):
            st, rel = self.step(st)
            rels.append(rel)
            if tol > 0 and rel < tol:
                break
        return st, rels


def shlr(Y, U, cfg, n_iter=None, tol=-1.0):
    """Run Algorithm S1; returns (X image [J][M][N], K, relative changes)."""
    s = Shlr2D(Y, U, cfg)
    st, rels = s.run(cfg.n_iter if n_iter is None else n_iter, tol)
    return ifft2c(st["K"]), st["K"], rels


# =========================================================== Algorithm S2
class ShlrParam:
    """SHLR-P (Eq. 7) / SHLR-VP (Eq. 8) solved by Algorithm S2, all FE positions
    m batched (each m is an independent problem; per-m stopping freezes m)."""

    def __init__(self, Yp, U, cfg):
        self.Y = np.asarray(Yp, dtype=np.complex128)      # [L][J][M][N], (m, k_n) hybrid
        self.U = np.asarray(U).astype(np.float64)         # [L][M][N]
        P = _params(cfg)
        self.P = P
        self.vc = P["model"] == "SHLR_VP"
        L, J, M, N = self.Y.shape
        self.L, self.J, self.M, self.N = L, J, M, N
        self.C = 2 * J if self.vc else J
        self.w = filter_weights(N, P["weight"])
        self.d_pe = normal_weights(N, P["p"], self.w, self.vc)
        self.c_p = hankel_multiplicity(L, P["pP"])

    def init_state(self):
        L, J, M, N, C = self.L, self.J, self.M, self.N, self.C
        p, pP, d0 = self.P["p"], self.P["pP"], self.P["d0"]
        Dpe = np.full((M * L, N - p + 1, C * p), d0, dtype=np.complex128)
        Dp = np.full((M * N, L - pP + 1, J * pP), d0, dtype=np.complex128)
        return dict(K=self.Y.copy(), Zpe=np.zeros_like(Dpe), Zp=np.zeros_like(Dp), Dpe=Dpe, Dp=Dp)

    def lifts(self, K):
        P = self.P
        Xi = ifftc(K, axis=3)                              # image along PE
        return lift_pe(K, self.w, P["p"], self.vc), lift_param(Xi, P["pP"])

    def x_update(self, Zpe, Zp, Dpe, Dp):
        """Eq. S7 as a pointwise divide in the (l, j, m, k_n) domain."""
        P = self.P
        b, lam = P["beta"], P["lam"]
        L, J, M, N = self.L, self.J, self.M, self.N
        a_pe = lift_pe_adjoint(Zpe - Dpe / b, self.w, P["p"], self.vc, L, J, M, N)
        a_p = lift_param_adjoint(Zp - Dp / b, P["pP"], L, J, M, N)
        rhs_b = b * (a_pe + fftc(a_p, axis=3))
        den_b = b * (self.d_pe[None, None, None, :] + self.c_p[:, None, None, None])
        U = self.U[:, None]
        return _dc_divide(lam, U, self.Y, rhs_b, den_b)

    def step(self, st, active):
        P = self.P
        b, tau = P["beta"], P["tau"]
        M, L, N = self.M, self.L, self.N
        Knew = self.x_update(st["Zpe"], st["Zp"], st["Dpe"], st["Dp"])
        num = np.sum(np.abs(Knew - st["K"]) ** 2, axis=(0, 1, 3))
        den = np.sum(np.abs(st["K"]) ** 2, axis=(0, 1, 3))
        rel = num / np.where(den > 0, den, 1.0)
        K = np.where(active[None, None, :, None], Knew, st["K"])
        LXpe, LXp = self.lifts(K)
        Zpe = svt(LXpe + st["Dpe"] / b, 1.0 / b)
        Zp = svt(LXp + st["Dp"] / b, P["lam2"] / b)
        Dpe = st["Dpe"] + tau * (LXpe - Zpe)
        Dp = st["Dp"] + tau * (LXp - Zp)
        a_pe = np.repeat(active, L)                        # matrices ordered (m, l)
        a_p = np.repeat(active, N)                         # matrices ordered (m, n)
        out = dict(K=K,
                   Zpe=np.where(a_pe[:, None, None], Zpe, st["Zpe"]),
                   Zp=np.where(a_p[:, None, None], Zp, st["Zp"]),
                   Dpe=np.where(a_pe[:, None, None], Dpe, st["Dpe"]),
                   Dp=np.where(a_p[:, None, None], Dp, st["Dp"]))
        return out, rel

    def run(self, n_iter, tol=-1.0, state=None):
        st = self.init_state() if state is None else state
        active = np.ones(self.M, dtype=bool)
        iters = np.zeros(self.M, dtype=np.int64)
        for _ in range(n_iter):
            if not active.any():
                break
            st, rel = self.step(st, active)
            iters += active
            if tol > 0:
                active = active & ~(rel < tol)
        return st, iters


def shlr_p(Yp, U, cfg, n_iter=None, tol=-1.0):
    """Run Algorithm S2; returns (X image [L][J][M][N], K, iterations per m)."""
    s = ShlrParam(Yp, U, cfg)
    st, iters = s.run(cfg.n_iter if n_iter is None else n_iter, tol)
    return ifftc(st["K"], axis=3), st["K"], iters


# ============================================ dense cross-check (tiny sizes)
def dense_x_update_2d(Y, U, Er, Ec, cfg, g=None):
    """Solve the X-subproblem of Eq. 10 (no G) by dense normal equations.

    Built from the literal image-domain operators: for every row m,
    X -> H~(_vc) W~ F~ P_m X (F^1D applied to the image row), likewise for
    columns, and X -> U F2D X.  The VC channels are only real-linear, so
    every operator is materialised as a real matrix acting on [Re x; Im x].
    Er, Ec are the targets Z - D/beta ([M][l][Cp], [N][l][Cp]).  Returns the
    k-space of the minimiser.  Intended for J*M*N <= ~200.
    """
    P = _params(cfg)
    vc = P["model"] in ("SHLR_V", "SHLR_SV")
    lam, b, p = P["lam"], P["beta"], P["p"]
    Y = np.asarray(Y, dtype=np.complex128)
    J, M, N = Y.shape
    wN = filter_weights(N, P["weight"])
    wM = filter_weights(M, P["weight"])
    n = J * M * N

    def lift_all(X):
        outs = []
        for m in range(M):
            v = np.stack([fftc(X[j, m, :]) for j in range(J)])
            outs.append(lift_vectors(v, wN, p, vc).ravel())
        for q in range(N):
            v = np.stack([fftc(X[j, :, q]) for j in range(J)])
            outs.append(lift_vectors(v, wM, p, vc).ravel())
        return np.concatenate(outs)

    def data(X):
        K = np.stack([fftc(fftc(X[j], axis=1), axis=0) for j in range(J)])
        return (U[None] * K).ravel()

    def realify(z):
        return np.concatenate([z.real, z.imag])

    def spirit_res(X):
        # (G - I) X with G applied in the image domain as F2D* G_k F2D (the k-space correlation)
        K = np.stack([fftc(fftc(X[j], axis=1), axis=0) for j in range(J)])
        R = spirit.apply_g(K, g) - K
        return np.stack([ifftc(ifftc(R[j], axis=1), axis=0) for j in range(J)]).ravel()

    cols_L, cols_A, cols_G = [], [], []
    for k in range(2 * n):
        e = np.zeros(n, dtype=np.complex128)
        e[k % n] = 1.0 if k < n else 1.0j
        X = e.reshape(J, M, N)
        cols_L.append(realify(lift_all(X)))
        cols_A.append(realify(data(X)))
        if g is not None:
            cols_G.append(realify(spirit_res(X)))
    Lm = np.stack(cols_L, axis=1)
    Am = np.stack(cols_A, axis=1)
    tgt = realify(np.concatenate([Er.ravel(), Ec.ravel()]))
    y = realify((U[None] * Y).ravel())
    H = b * Lm.T @ Lm
    rhs = b * Lm.T @ tgt
    if lam > 0:
        H = H + lam * Am.T @ Am
        rhs = rhs + lam * Am.T @ y
    if g is not None:
        Gm = np.stack(cols_G, axis=1)
        H = H + P["lam1"] * Gm.T @ Gm
    x = np.linalg.solve(H, rhs)
    X = (x[:n] + 1j * x[n:]).reshape(J, M, N)
    return np.stack([fftc(fftc(X[j], axis=1), axis=0) for j in range(J)])


def dense_x_update_param(Yp, U, Epe, Ep, cfg):
    """Dense normal-equation solve of the X-subproblem Eq. S2 (tiny sizes).

    Built from the literal operators of Eq. 7 / 8 on the image X_m^{PE-P}
    (every m at once): X -> H~(_vc) W~ F~ Q_l X (F^1D along PE of the echo-l
    column), X -> H~ P_n X (echo vectors, no F, no W), and X -> U F^PE X.
    Epe, Ep are the targets Z - D/beta.  Returns the minimiser in the
    (l, j, m, k_n) domain.
    """
    P = _params(cfg)
    vc = P["model"] == "SHLR_VP"
    lam, b, p, pP = P["lam"], P["beta"], P["p"], P["pP"]
    Yp = np.asarray(Yp, dtype=np.complex128)
    L, J, M, N = Yp.shape
    w = filter_weights(N, P["weight"])
    n = L * J * M * N

    def lift_all(X):
        outs = []
        for m in range(M):
            for l in range(L):
                v = np.stack([fftc(X[l, j, m, :]) for j in range(J)])
                outs.append(lift_vectors(v, w, p, vc).ravel())
        for m in range(M):
            for q in range(N):
                v = np.stack([X[:, j, m, q] for j in range(J)])
                outs.append(lift_vectors(v, None, pP, False).ravel())
        return np.concatenate(outs)

    def data(X):
        return (U[:, None] * fftc(X, axis=3)).ravel()

    def realify(z):
        return np.concatenate([z.real, z.imag])

    cols_L, cols_A = [], []
    for k in range(2 * n):
        e = np.zeros(n, dtype=np.complex128)
        e[k % n] = 1.0 if k < n else 1.0j
        X = e.reshape(L, J, M, N)
        cols_L.append(realify(lift_all(X)))
        cols_A.append(realify(data(X)))
    Lm = np.stack(cols_L, axis=1)
    Am = np.stack(cols_A, axis=1)
    tgt = realify(np.concatenate([Epe.ravel(), Ep.ravel()]))
    y = realify((U[:, None] * Yp).ravel())
    H = b * Lm.T @ Lm
    g = b * Lm.T @ tgt
    if lam > 0:
        H = H + lam * Am.T @ Am
        g = g + lam * Am.T @ y
    x = np.linalg.solve(H, g)
    X = (x[:n] + 1j * x[n:]).reshape(L, J, M, N)
    return fftc(X, axis=3)
