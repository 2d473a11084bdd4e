"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only *simulates acquisitions*: phantoms, smooth phase, coil
sensitivities, T2 decay along echoes, sampling masks, complex noise, and the
forward acquisition ``Y = U * (F2D(S_j * image) + noise)``.  It holds none of
the reconstruction method's arithmetic (no Hankel lift, SVT, adjoint or data
consistency).  The forward 2D/1D Fourier transforms used to synthesise
k-space are NumPy's FFT with the centred unitary convention that the
reconstruction assumes (DC at index N/2), because an acquisition has to be
simulated somehow; the reconstruction side never calls into this module.

Every generator takes an explicit ``numpy.random.Generator`` or seed, so the
same call produces the same arrays on any machine.

Array conventions (all C-contiguous):
  2D data   : [J][M][N]       complex, row index m (dim 1), column index n (dim 2)
  param data: [L][J][M][N]    complex, echo l outermost; m = FE, n = PE
  masks     : [M][N] (2D) or [L][M][N] (parameter imaging), uint8 0/1
"""
from __future__ import annotations

import numpy as np

from .configs import ACS_SWEEP, CONFIGS, Workload, get_config, unrolled_batch, unrolled_instance  # noqa: F401


# ---------------------------------------------------------------- transforms
def _fftc(x, axes):
    """Centred unitary DFT used only to simulate acquisition."""
    x = np.fft.ifftshift(x, axes=axes)
    x = np.fft.fftn(x, axes=axes, norm="ortho")
    return np.fft.fftshift(x, axes=axes)


def _ifftc(x, axes):
    x = np.fft.ifftshift(x, axes=axes)
    x = np.fft.ifftn(x, axes=axes, norm="ortho")
    return np.fft.fftshift(x, axes=axes)


# ------------------------------------------------------------------ phantoms
def _grid(M, N):
    y = (np.arange(M) - M / 2) / M        # [-0.5, 0.5)
    x = (np.arange(N) - N / 2) / N
    return np.meshgrid(y, x, indexing="ij")


def ellipse_phantom(M, N, rng, n_ellipses=10):
    """Sum of ``n_ellipses`` random filled ellipses, intensities in (0.1, 1].

    The image is zero outside a centred disc covering 90% of the FOV width.
    """
    Y, X = _grid(M, N)
    img = np.zeros((M, N))
    for _ in range(n_ellipses):
        cy, cx = rng.uniform(-0.25, 0.25, size=2)
        ay, ax = rng.uniform(0.04, 0.30, size=2)
        th = rng.uniform(0, np.pi)
        amp = rng.uniform(0.1, 1.0)
        if amp <= 0.1:
            amp = 0.1 + 1e-6
        c, s = np.cos(th), np.sin(th)
        u = ((X - cx) * c + (Y - cy) * s) / ax
        v = (-(X - cx) * s + (Y - cy) * c) / ay
        img += amp * ((u * u + v * v) <= 1.0)
    img *= (X * X + Y * Y) <= 0.45 ** 2
    m = img.max()
    return img / m if m > 0 else img


def smooth_phase(M, N, rng, max_rad=0.5):
    """Random 2D quadratic phase map scaled so that max |phase| <= max_rad."""
    Y, X = _grid(M, N)
    a = rng.standard_normal(6)
    ph = a[0] + a[1] * X + a[2] * Y + a[3] * X * X + a[4] * X * Y + a[5] * Y * Y
    return ph * (max_rad / max(np.abs(ph).max(), 1e-12))


def coil_maps(J, M, N, rng, ring=0.6, width=0.4):
    """Smooth complex Gaussian coil sensitivities normalised to sum |S_j|^2 = 1.

    Coil j is a Gaussian bump of std ``width`` (in FOV units) centred on a
    ring of radius ``ring`` with a small random linear phase.
    """
    Y, X = _grid(M, N)
    S = np.empty((J, M, N), dtype=np.complex128)
    off = rng.uniform(0, 2 * np.pi)
    for j in range(J):
        ang = off + 2 * np.pi * j / J
        cy, cx = ring * np.sin(ang), ring * np.cos(ang)
        mag = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * width ** 2))
        kx, ky = rng.uniform(-0.5, 0.5, size=2)
        S[j] = mag * np.exp(1j * (kx * X + ky * Y) * np.pi)
    S /= np.sqrt((np.abs(S) ** 2).sum(axis=0, keepdims=True))
    return S


# --------------------------------------------------------------------- masks
def mask_1d_random(M, N, R, n_acs, rng, axis=0):
    """1D Cartesian mask: ``n_acs`` centre lines plus uniformly random lines.

    Lines are indexed along ``axis`` (0: k_m lines, each a full row of N
    samples; 1: k_n lines).  Total lines = round(size / R).
    """
    size = M if axis == 0 else N
    total = int(round(size / R))
    lines = np.zeros(size, dtype=bool)
    c0 = size // 2 - n_acs // 2
    lines[c0:c0 + n_acs] = True
    rest = np.flatnonzero(~lines)
    need = max(total - int(lines.sum()), 0)
    lines[rng.choice(rest, size=need, replace=False)] = True
    m = np.zeros((M, N), dtype=np.uint8)
    if axis == 0:
        m[lines, :] = 1
    else:
        m[:, lines] = 1
    return m


def mask_1d_gaussian(M, N, R, n_center, rng, axis=0, sigma_frac=0.25):
    """1D Cartesian mask with Gaussian line density plus ``n_center`` centre lines."""
    size = M if axis == 0 else N
    total = int(round(size / R))
    lines = np.zeros(size, dtype=bool)
    c0 = size // 2 - n_center // 2
    lines[c0:c0 + n_center] = True
    k = np.arange(size) - size / 2
    p = np.exp(-0.5 * (k / (sigma_frac * size)) ** 2)
    p[lines] = 0
    p /= p.sum()
    need = max(total - int(lines.sum()), 0)
    lines[rng.choice(size, size=need, replace=False, p=p)] = True
    m = np.zeros((M, N), dtype=np.uint8)
    if axis == 0:
        m[lines, :] = 1
    else:
        m[:, lines] = 1
    return m


def mask_1d_uniform(M, N, R, n_center, axis=0, shift=0):
    """Uniform (regular) 1D Cartesian mask: every R-th line counted from the
    centre line (offset by ``shift``), plus ``n_center`` centre (ACS) lines."""
    size = M if axis == 0 else N
    R = int(round(R))
    c = size // 2
    lines = ((np.arange(size) - c - shift) % R) == 0
    c0 = c - n_center // 2
    lines[c0:c0 + n_center] = True
    m = np.zeros((M, N), dtype=np.uint8)
    if axis == 0:
        m[lines, :] = 1
    else:
        m[:, lines] = 1
    return m


def partial_fourier(mask, frac, axis=0):
    """Partial Fourier: keep the first ceil(frac * size) lines along ``axis``
    (which contain the centre for frac > 1/2) and drop the rest of the
    high-frequency side."""
    m = mask.copy()
    size = m.shape[axis]
    keep = int(np.ceil(frac * size))
    sl = [slice(None)] * m.ndim
    sl[axis] = slice(keep, size)
    m[tuple(sl)] = 0
    return m


def acs_sweep_masks(M, N, rate, acs_lines, seed, axis=0):
    """1D Gaussian-density Cartesian masks, all at the same total sampling rate,
    that differ in the number of centre (ACS) lines: {n_acs: mask}."""
    out = {}
    for n_acs in acs_lines:
        rng = np.random.default_rng(seed)
        out[int(n_acs)] = mask_1d_gaussian(M, N, 1.0 / rate, int(n_acs), rng, axis=axis)
    return out


def mask_poisson_2d(M, N, R, rng, acs=8, max_tries=30):
    """2D Poisson-disc mask (dart throwing) with an ``acs`` x ``acs`` centre block.

    The minimum distance is found by bisection so the sampled fraction is
    close to 1/R.
    """
    target = M * N / R

    def throw(r):
        order = rng.permutation(M * N)
        taken = np.zeros((M, N), dtype=bool)
        occ = np.zeros((M, N), dtype=bool)
        ri = int(np.ceil(r))
        yy, xx = np.mgrid[-ri:ri + 1, -ri:ri + 1]
        disc = (yy * yy + xx * xx) < r * r
        dy, dx = yy[disc], xx[disc]
        for idx in order:
            i, j = divmod(int(idx), N)
            if occ[i, j]:
                continue
            taken[i, j] = True
            occ[np.clip(i + dy, 0, M - 1), np.clip(j + dx, 0, N - 1)] = True
        return taken

    lo, hi = 0.5, 8.0
    best = None
    for _ in range(max_tries):
        r = 0.5 * (lo + hi)
        t = throw(r)
        t[M // 2 - acs // 2:M // 2 + acs // 2, N // 2 - acs // 2:N // 2 + acs // 2] = True
        cnt = t.sum()
        if best is None or abs(cnt - target) < abs(best.sum() - target):
            best = t
        if abs(cnt - target) <= 0.01 * target:
            break
        if cnt > target:
            lo = r
        else:
            hi = r
    return best.astype(np.uint8)


# ------------------------------------------------------------- acquisitions
def multicoil_image(J, M, N, seed, max_phase=0.5):
    """Coil images S_j * (phantom * exp(i*phase)) : [J][M][N] complex128."""
    rng = np.random.default_rng(seed)
    img = ellipse_phantom(M, N, rng) * np.exp(1j * smooth_phase(M, N, rng, max_phase))
    S = coil_maps(J, M, N, rng)
    return S * img[None]


def acquire_2d(coil_img, mask, sigma_n, seed):
    """Zero-filled k-space Y = U * (F2D(x_j) + sigma_n * CN(0,1)) : [J][M][N]."""
    rng = np.random.default_rng(seed + 7919)
    K = _fftc(coil_img, axes=(-2, -1))
    if sigma_n > 0:
        K = K + sigma_n * (rng.standard_normal(K.shape) + 1j * rng.standard_normal(K.shape)) / np.sqrt(2)
    return K * mask[None]


def t2_series(J, M, N, L, te_ms, seed, t2_range=(20.0, 200.0), max_phase=0.5):
    """Multi-echo coil images [L][J][M][N]: S_j * M0 * exp(-TE_l / T2) * exp(i*phase).

    M0 is the phantom magnitude; T2 is drawn per pixel, uniform in ``t2_range`` ms.
    """
    rng = np.random.default_rng(seed)
    m0 = ellipse_phantom(M, N, rng)
    ph = smooth_phase(M, N, rng, max_phase)
    S = coil_maps(J, M, N, rng)
    t2 = rng.uniform(t2_range[0], t2_range[1], size=(M, N))
    te = np.asarray(te_ms, dtype=np.float64)
    decay = np.exp(-te[:, None, None] / t2[None])                     # [L][M][N]
    img = m0[None] * decay * np.exp(1j * ph)[None]                     # [L][M][N]
    return S[None] * img[:, None], t2, m0


def acquire_param(series, masks, sigma_n, seed):
    """Hybrid parameter data Y^Parameter: k-space masked per echo, then 1D
    inverse FT along FE (dim m).  ``masks`` is [L][M][N].  Returns [L][J][M][N]."""
    rng = np.random.default_rng(seed + 7919)
    K = _fftc(series, axes=(-2, -1))
    if sigma_n > 0:
        K = K + sigma_n * (rng.standard_normal(K.shape) + 1j * rng.standard_normal(K.shape)) / np.sqrt(2)
    K = K * masks[:, None]
    return _ifftc(K, axes=(-2,))


# --------------------------------------------------------------- workloads
def make_inputs(cfg, small=None):
    """Build (Y, mask, truth) for a :class:`Workload`.

    ``small`` optionally overrides (J, M, N) to get a reduced-size case with
    the same recipe.  Y is normalised by 1/max|Y| (the same factor is applied
    to ``truth``), so the regularisation parameters of the config apply.
    Returns a dict with keys Y (complex128), mask (uint8), truth (complex128).
    """
    J, M, N = cfg.J, cfg.M, cfg.N
    if small is not None:
        J, M, N = small
    rng_mask = np.random.default_rng(cfg.seed + 101)
    if cfg.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV"):
        x = multicoil_image(J, M, N, cfg.seed)
        if cfg.mask == "gauss1d":
            mask = mask_1d_gaussian(M, N, cfg.R, cfg.n_acs, rng_mask)
        elif cfg.mask == "random1d":
            mask = mask_1d_random(M, N, cfg.R, cfg.n_acs, rng_mask)
        elif cfg.mask == "poisson2d":
            mask = mask_poisson_2d(M, N, cfg.R, rng_mask, acs=cfg.n_acs)
        elif cfg.mask == "uniform1d":
            mask = mask_1d_uniform(M, N, cfg.R, cfg.n_acs)
        elif cfg.mask == "full":
            mask = np.ones((M, N), dtype=np.uint8)
        else:
            raise ValueError(cfg.mask)
        if cfg.pf < 1.0:
            mask = partial_fourier(mask, cfg.pf, axis=0)
        Y = acquire_2d(x, mask, cfg.sigma_n, cfg.seed)
        s = 1.0 / np.abs(Y).max()
        return {"Y": Y * s, "mask": mask, "truth": x * s}
    # parameter imaging: masks along PE (dim n), one per echo
    L = cfg.L
    te = [cfg.te_ms * (l + 1) for l in range(L)]
    series, _, _ = t2_series(J, M, N, L, te, cfg.seed)
    masks = np.empty((L, M, N), dtype=np.uint8)
    for l in range(L):
        r = np.random.default_rng(cfg.seed + l)
        if cfg.mask == "full":
            masks[l] = 1
        elif cfg.mask == "uniform1d":
            masks[l] = mask_1d_uniform(M, N, cfg.R, cfg.n_acs, axis=1, shift=l)   # echo-varying offsets
        else:
            masks[l] = mask_1d_random(M, N, cfg.R, cfg.n_acs, r, axis=1)
        if cfg.pf < 1.0:
            masks[l] = partial_fourier(masks[l], cfg.pf, axis=1)
    Y = acquire_param(series, masks, cfg.sigma_n, cfg.seed)
    s = 1.0 / np.abs(Y).max()
    return {"Y": Y * s, "mask": masks, "truth": series * s}
