"""Unrolled Algorithm S1 with per-iteration thresholds and multiplier steps,
and its reverse-mode derivative, in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Forward: Algorithm S1 for SHLR / SHLR-V exactly as :class:`admm.Shlr2D` runs
it, except that iteration k uses its own SVT threshold t_k (Eqs. 16-17; the
paper fixes t = 1/beta) and multiplier step tau_k (Eqs. 13-14; the paper
fixes tau).  With t_k = 1/beta and tau_k = tau it is Algorithm S1 itself.
The output is the image X = F2D* K of the last X-update.

Reverse: the chain rule taken step by step backwards through the same
operations, for a real loss with cotangent Xbar of X (real inner product
Re tr(X^H Y)):
* X = F2D* K, the hybrid transforms and the X-update (Eq. 15) are linear in
  their array inputs: their derivatives are their adjoints (F* for F, the
  Hankel lift for the real adjoint of the lift, and the pointwise divide
  scaled by beta / den for Eq. 15);
* the SVT uses :func:`svt.svt_vjp` (Hermitian dilation + Daleckii-Krein);
* D_k = D + tau_k (A - D / beta - Z) with A = lift(K) + D / beta and
  E = Z - D_k / beta (the input of the next X-update).
Returns the gradients with respect to the thresholds, the steps and Y.
"""
from __future__ import annotations

import numpy as np

from .admm import Shlr2D
from .hankel import lift_rows, lift_rows_adjoint, lift_cols, lift_cols_adjoint
from .svt import svt, svt_vjp
from .transforms import fftc, ifftc, ifft2c, fft2c


def _svt_vjp_batch(A, Zbar, t):
    Abar = np.empty_like(A)
    tbar = 0.0
    for i in range(A.shape[0]):
        Abar[i], tb = svt_vjp(A[i], Zbar[i], t)
        tbar += tb
    return Abar, tbar


def unrolled_2d(Y, U, cfg, ts, taus, return_states=False):
    """n = len(ts) iterations of Algorithm S1 with per-iteration t_k, tau_k."""
    s = Shlr2D(Y, U, cfg)
    beta = s.P["beta"]
    st = s.init_state()
    Dr, Dc, Zr, Zc = st["Dr"], st["Dc"], st["Zr"], st["Zc"]
    states = []
    K = None
    for k in range(len(ts)):
        states.append((Dr.copy(), Dc.copy()))
        K = s.x_update(Zr, Zc, Dr, Dc)
        LXr, LXc = s.lifts(K)
        Zr = svt(LXr + Dr / beta, ts[k])
        Zc = svt(LXc + Dc / beta, ts[k])
        Dr = Dr + taus[k] * (LXr - Zr)
        Dc = Dc + taus[k] * (LXc - Zc)
        states[-1] = states[-1] + (K.copy(),)
    X = ifft2c(K)
    return (X, states) if return_states else X


def unrolled_2d_vjp(Y, U, cfg, ts, taus, Xbar):
    """Gradient of Re tr(Xbar^H X) with respect to (ts, taus, Y)."""
    s = Shlr2D(Y, U, cfg)
    P = s.P
    beta, lam, p, vc = P["beta"], P["lam"], P["p"], s.vc
    J, M, N = s.J, s.M, s.N
    n = len(ts)
    _, states = unrolled_2d(Y, U, cfg, ts, taus, return_states=True)
    Uf = s.U[None]
    den_b = beta * (s.d_r[None, None, :] + s.d_c[None, :, None])
    tbar = np.zeros(n)
    taubar = np.zeros(n)
    Ybar = np.zeros_like(s.Y)
    Kbar = fft2c(np.asarray(Xbar, dtype=np.complex128))     # adjoint of F2D*
    Dbar_r = Dbar_c = None
    for k in range(n - 1, -1, -1):
        Dr, Dc, K = states[k]
        if k < n - 1:
            # Z- and D-updates of iteration k (their outputs feed iteration k + 1)
            LXr, LXc = s.lifts(K)
            Ar, Ac = LXr + Dr / beta, LXc + Dc / beta
            Zr, Zc = svt(Ar, ts[k]), svt(Ac, ts[k])
            Kbar = np.zeros_like(K)
            for (A, D, Z, Db, Eb, lift_adj, w, ax) in (
                    (Ar, Dr, Zr, Dbar_r, Ebar_r, lift_rows_adjoint, s.wN, 1),
                    (Ac, Dc, Zc, Dbar_c, Ebar_c, lift_cols_adjoint, s.wM, 2)):
                Dp = Db - Eb / beta                     # cotangent of D_k through D_k and E_k
                Zb = Eb - taus[k] * Dp
                taubar[k] += np.real(np.vdot(Dp, A - D / beta - Z))
                Ab, tb = _svt_vjp_batch(A, Zb, ts[k])
                tbar[k] += tb
                Ab = Ab + taus[k] * Dp
                Dnew = (1.0 - taus[k] / beta) * Dp + Ab / beta
                nlen = N if ax == 1 else M
                xb = lift_adj(Ab, w, p, vc, J, nlen)
                Kbar = Kbar + fftc(xb, axis=ax)          # adjoint of the inverse hybrid transform
                if ax == 1:
                    Dbar_r = Dnew
                else:
                    Dbar_c = Dnew
        else:
            Dbar_r = np.zeros_like(Dr)
            Dbar_c = np.zeros_like(Dc)
        # X-update of iteration k: K = (lam U Y + beta (F_m a_r + F_n a_c)) / den
        if lam > 0:
            den = lam * Uf + den_b
            safe = np.where(den != 0, den, 1.0)
            Sb = np.where(den != 0, beta * Kbar / safe, 0.0)
            Ybar = Ybar + np.where(den != 0, lam * Uf * Kbar / safe, 0.0)
        else:
            safe = np.where(den_b != 0, den_b, 1.0)
            Sb = np.where((Uf > 0) | (den_b == 0), 0.0, beta * Kbar / safe)
            Ybar = Ybar + np.where(Uf > 0, Kbar, 0.0)
        ar = ifftc(Sb, axis=1)
        ac = ifftc(Sb, axis=2)
        Ebar_r = lift_rows(ar, s.wN, p, vc)
        Ebar_c = lift_cols(ac, s.wM, p, vc)
        # E_{k-1} = Z_{k-1} - D_{k-1} / beta: D_{k-1}'s cotangent gets -Ebar / beta in the
        # next (earlier) step through Dp = Dbar - Ebar / beta.
    return tbar, taubar, Ybar
