"""SPIRiT operator G and the X-update of SHLR-S / SHLR-SV (Eq. 3, Eq. 6, Eq. 15).

Test infrastructure only (see ``oracle/__init__.py``).

G models every k-space sample of coil j as a linear combination of the
samples of all coils in a ksize x ksize neighbourhood (the sample itself
excluded), with one kernel per coil pair:
    (G K)_j[m, n] = sum_{j', a, b} g[j, j', a, b] K_j'[m + a - h, n + b - h],   h = ksize // 2,
taken circularly in k-space, so that in the image domain G is a pixelwise
J x J matrix (the form the paper's "SPIRiT operator in image domain" takes).

Readings (the paper gives neither the kernel size nor the calibration):
* ksize = 5; the kernel is calibrated on the ACS block (the n_acs centre rows
  of k-space, all columns) from every kernel position that fits inside the
  block, by Tikhonov-regularised least squares per target coil with weight
  reg * trace(A^H A) / (number of unknowns), reg = 1e-3.
* The X-update (Eq. 15 with the lambda_1 (G - I)^* (G - I) term) is solved in
  k-space by conjugate gradients on the normal equations
      (lambda U + beta d + lambda_1 (G - I)^H (G - I)) K = lambda U Y + beta (lift adjoints),
  to a relative residual of 1e-12, from the previous iterate.  lambda must
  be finite (no hard data consistency with the SPIRiT term).
"""
from __future__ import annotations

import numpy as np


def calibrate(Y, n_acs, ksize=5, reg=1e-3):
    """Kernel g [J][J][ksize][ksize] from the ACS rows of k-space Y [J][M][N]."""
    Y = np.asarray(Y, dtype=np.complex128)
    J, M, N = Y.shape
    h = ksize // 2
    r0 = M // 2 - n_acs // 2
    r1 = r0 + n_acs
    rows = []
    for m in range(r0 + h, r1 - h):
        for n in range(h, N - h):
            rows.append(Y[:, m - h:m + h + 1, n - h:n + h + 1].reshape(-1))
    A = np.asarray(rows)
    kk = ksize * ksize
    g = np.zeros((J, J, ksize, ksize), dtype=np.complex128)
    for j in range(J):
        tgt = j * kk + h * ksize + h
        cols = np.array([q for q in range(J * kk) if q != tgt])
        As, b = A[:, cols], A[:, tgt]
        C = As.conj().T @ As
        lam = reg * np.trace(C).real / C.shape[0]
        x = np.linalg.solve(C + lam * np.eye(len(cols)), As.conj().T @ b)
        full = np.zeros(J * kk, dtype=np.complex128)
        full[cols] = x
        g[j] = full.reshape(J, ksize, ksize)
    return g


def apply_g(K, g):
    """(G K) by the circular k-space correlation in the module docstring (one
    circular shift of every coil per kernel offset, then the J x J kernel
    weights of that offset)."""
    K = np.asarray(K, dtype=np.complex128)
    ks = g.shape[-1]
    h = ks // 2
    out = np.zeros_like(K)
    for a in range(ks):
        for b in range(ks):
            w = g[:, :, a, b]
            if np.any(w):
                out += np.einsum("jk,kmn->jmn", w, np.roll(K, (-(a - h), -(b - h)), axis=(1, 2)))
    return out


def apply_gh(V, g):
    """Adjoint G^H of apply_g (transposed conjugate kernel weights, opposite shifts)."""
    V = np.asarray(V, dtype=np.complex128)
    ks = g.shape[-1]
    h = ks // 2
    out = np.zeros_like(V)
    for a in range(ks):
        for b in range(ks):
            w = g[:, :, a, b]
            if np.any(w):
                out += np.roll(np.einsum("jk,jmn->kmn", np.conj(w), V), (a - h, b - h), axis=(1, 2))
    return out


def normal_op(K, diag, lam1, g):
    """diag * K + lam1 (G - I)^H (G - I) K (diag = lambda U + beta d, broadcast)."""
    R = apply_g(K, g) - K
    return diag * K + lam1 * (apply_gh(R, g) - R)


def cg(apply_A, rhs, x0, tol=1e-12, max_iter=2000):
    """Conjugate gradients for the Hermitian positive definite apply_A."""
    x = x0.copy()
    r = rhs - apply_A(x)
    p = r.copy()
    rr = np.vdot(r, r).real
    nb = np.vdot(rhs, rhs).real
    it = 0
    while it < max_iter and rr > tol * tol * nb:
        Ap = apply_A(p)
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it
