"""Image-quality metrics (Sec. IV; Eq. S10).  Test infrastructure only."""
from __future__ import annotations

import numpy as np


def ssos(X, coil_axis=0):
    """Square root of the sum of squares over coils."""
    return np.sqrt(np.sum(np.abs(X) ** 2, axis=coil_axis))


def rlne(x, xhat):
    """Relative l2 norm error ||x - xhat||_2 / ||x||_2 (Eq. S10)."""
    x = np.asarray(x).ravel()
    xhat = np.asarray(xhat).ravel()
    return float(np.linalg.norm(x - xhat) / np.linalg.norm(x))


def rel_l2(a, ref):
    """||a - ref||_F / ||ref||_F."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(ref)) / np.linalg.norm(ref))
