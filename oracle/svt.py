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
