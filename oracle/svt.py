"""Singular value thresholding (Eqs. 16-17, S8-S9).

Test infrastructure only (see ``oracle/__init__.py``).

S_t(A) = U diag(max(sigma - t, 0)) V^H, the proximal map of t*||.||_* , taken
from a full SVD (``numpy.linalg.svd``, a library step).  Z is unique even when
the singular vectors are not (S_t is a spectral function), so comparisons
are made on Z, never on U or V.  sigma = t maps to 0.
"""
from __future__ import annotations

import numpy as np


def svt(A, t):
    """Batched S_t over the last two axes of A (complex)."""
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    s = np.maximum(s - t, 0.0)
    return (U * s[..., None, :]) @ Vh


def svt_rank(A, t):
    """Number of singular values strictly above t, per matrix."""
    s = np.linalg.svd(A, compute_uv=False)
    return (s > t).sum(axis=-1)


def nuclear_norm(A):
    return np.linalg.svd(A, compute_uv=False).sum(axis=-1)


# ------------------------------------------------------------------ reverse
def _shrink_odd(mu, t):
    """The odd extension g(mu) = sign(mu) max(|mu| - t, 0) of the shrinkage."""
    return np.sign(mu) * np.maximum(np.abs(mu) - t, 0.0)


def svt_vjp(A, Zbar, t, guard=1e-9):
    """Reverse-mode derivative of Z = S_t(A) for one matrix, in FP64.

    Written independently of the Gram-matrix form: S_t(A) is the top-right
    block of g(H) for the Hermitian dilation H = [[0, A], [A^H, 0]] (whose
    eigenvalues are +-sigma_i and zeros) and the odd shrinkage g of
    ``_shrink_odd``.  For a Hermitian matrix function the Daleckii-Krein
    theorem gives Dg(H)[E] = Q (Gamma o (Q^H E Q)) Q^H with H = Q diag(mu) Q^H
    and Gamma_ij the first divided difference of g at (mu_i, mu_j) (g'(mu)
    where the two agree).  Dg(H) is self-adjoint for the real inner product
    Re tr(X^H Y), so with the cotangent Zbar of the top-right block,
        Abar = [Dg(H)[[[0, Zbar], [Zbar^H, 0]]]]_{top-right},
        tbar = Re tr(Zbar^H dS_t/dt),  dg/dt = -sign(mu) [|mu| > t].
    Returns (Abar, tbar)."""
    A = np.asarray(A, dtype=np.complex128)
    Zbar = np.asarray(Zbar, dtype=np.complex128)
    m, n = A.shape
    H = np.zeros((m + n, m + n), dtype=np.complex128)
    H[:m, m:] = A
    H[m:, :m] = A.conj().T
    mu, Q = np.linalg.eigh(H)
    g = _shrink_odd(mu, t)
    dg = (np.abs(mu) > t).astype(np.float64)
    dmu = mu[:, None] - mu[None, :]
    scale = np.maximum(np.abs(mu)[:, None], np.abs(mu)[None, :])
    close = np.abs(dmu) <= guard * np.maximum(scale, 1.0)
    safe = np.where(close, 1.0, dmu)
    Gam = np.where(close, 0.5 * (dg[:, None] + dg[None, :]), (g[:, None] - g[None, :]) / safe)
    Eb = np.zeros_like(H)
    Eb[:m, m:] = Zbar
    Eb[m:, :m] = Zbar.conj().T
    W = Q @ (Gam * (Q.conj().T @ Eb @ Q)) @ Q.conj().T
    Abar = W[:m, m:]
    dZdt = (Q * (-np.sign(mu) * dg)[None, :]) @ Q.conj().T
    tbar = float(np.real(np.vdot(Zbar, dZdt[:m, m:])))
    return Abar, tbar
