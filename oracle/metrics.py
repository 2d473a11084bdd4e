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


# ----------------------------------------------------------------- MSSIM
def gaussian_window(size=11, sigma=1.5):
    """Normalised 2D Gaussian window (the MSSIM local window; the paper does not
    fix it: the usual 11 x 11, sigma = 1.5 is taken)."""
    r = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-0.5 * (r / sigma) ** 2)
    w = np.outer(g, g)
    return w / w.sum()


def mssim(A, B, L=None, size=11, sigma=1.5, k1=0.01, k2=0.03):
    """Mean structural similarity (Eq. in Sec. S3) of reference A and image B
    (real, 2D): the local means, variances and covariance are Gaussian-weighted
    over every window that fits inside the image ("valid" positions), C1 =
    (k1 L)^2, C2 = (k2 L)^2 with L the dynamic range (default: max of A).
    Window statistics by scipy.signal.correlate2d (a library step)."""
    from scipy.signal import correlate2d
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    L = float(A.max()) if L is None else float(L)
    C1, C2 = (k1 * L) ** 2, (k2 * L) ** 2
    w = gaussian_window(size, sigma)
    f = lambda x: correlate2d(x, w, mode="valid")
    mu_a, mu_b = f(A), f(B)
    saa = f(A * A) - mu_a ** 2
    sbb = f(B * B) - mu_b ** 2
    sab = f(A * B) - mu_a * mu_b
    ssim = ((2 * mu_a * mu_b + C1) * (2 * sab + C2)) / ((mu_a ** 2 + mu_b ** 2 + C1) * (saa + sbb + C2))
    return float(ssim.mean())


# ----------------------------------------------------------------- T2 fit
def t2_fit(S, te_ms, t2_range=(1.0, 1000.0)):
    """Pixel-by-pixel nonlinear least-squares fit of S_l = M0 exp(-TE_l / T2)
    (Sec. IV, T2 mapping) to magnitudes S [L][...] at echo times te_ms [L].
    Each pixel: scipy.optimize.least_squares (a library step) from the
    log-linear fit.  Returns (T2, M0) with T2 = NaN outside t2_range or where
    the data are not positive (the paper excludes T2 outside a reasonable
    range without stating it; the range is a reading)."""
    from scipy.optimize import least_squares
    S = np.asarray(S, dtype=np.float64)
    te = np.asarray(te_ms, dtype=np.float64)
    shp = S.shape[1:]
    flat = S.reshape(S.shape[0], -1)
    T2 = np.full(flat.shape[1], np.nan)
    M0 = np.full(flat.shape[1], np.nan)
    for p in range(flat.shape[1]):
        s = flat[:, p]
        if not (s > 0).all():
            continue
        slope, icpt = np.polyfit(te, np.log(s), 1)
        r0 = -slope if slope < 0 else 1.0 / t2_range[1]
        x0 = np.array([np.exp(icpt), r0])               # (M0, R2 = 1 / T2)
        res = least_squares(lambda x: x[0] * np.exp(-te * x[1]) - s, x0, method="lm", xtol=1e-15, ftol=1e-15,
                            gtol=1e-15, max_nfev=2000)
        m0, r2 = res.x
        if r2 > 0 and t2_range[0] <= 1.0 / r2 <= t2_range[1]:
            T2[p], M0[p] = 1.0 / r2, m0
    return T2.reshape(shp), M0.reshape(shp)
