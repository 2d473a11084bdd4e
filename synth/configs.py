"""Named synthetic workloads (sizes, seeds, sampling and solver parameters).

Each workload mirrors the shape and structure of one of the paper's
experiments (multi-coil 2D brain k-space; multi-echo T2 data) with a seeded
ellipse phantom in place of the in-vivo scans, which are not available.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict, replace


@dataclass(frozen=True)
class Workload:
    name: str
    model: str            # "SHLR", "SHLR_V", "SHLR_P", "SHLR_VP"
    J: int
    M: int
    N: int
    L: int = 1
    window: int = 8
    window_param: int = 4
    weight: int = 1       # 0: W = I ; 1: circular finite-difference filter
    mask: str = "random1d"  # random1d, gauss1d, uniform1d, poisson2d, full
    R: float = 4.0
    n_acs: int = 24
    pf: float = 1.0       # partial Fourier: fraction of the phase-encoding lines kept
    sigma_n: float = 0.0
    seed: int = 1
    te_ms: float = 10.0
    n_iter: int = 30
    lam: float = 1.0e4    # data-term weight lambda (<= 0 : hard data consistency)
    lam2: float = 2.0     # parameter-dimension weight lambda_2
    lam1: float = 1000.0  # SPIRiT weight lambda_1 (SHLR-S / SHLR-SV)
    spirit_k: int = 5     # SPIRiT kernel size
    spirit_reg: float = 1e-3   # SPIRiT calibration Tikhonov weight (relative)
    cg_iters: int = 30    # CG iterations of the SHLR-S / SHLR-SV X-update on the GPU
    beta: float = 1.0
    tau: float = 1.0
    d_init: float = 1.0

    def to_dict(self):
        return asdict(self)

    def with_(self, **kw):
        return replace(self, **kw)


CONFIGS = {
    # 4-coil 64x64, plain SHLR, 1D Gaussian-density Cartesian R=3 + 8 centre lines
    "shlr_4c_64": Workload(name="shlr_4c_64", model="SHLR", J=4, M=64, N=64, window=8,
                           mask="gauss1d", R=3.0, n_acs=8, sigma_n=0.0, seed=1,
                           beta=20.0, tau=20.0),
    # 12-coil 256x256 parallel imaging, 1D random R=4 + 24 ACS, noise 1e-3
    "shlr_12c_256": Workload(name="shlr_12c_256", model="SHLR", J=12, M=256, N=256, window=16,
                             mask="random1d", R=4.0, n_acs=24, sigma_n=1e-3, seed=2,
                             beta=20.0, tau=20.0),
    # same data, SHLR-V (conjugate-symmetric virtual coils), 2D Poisson-disc R=5
    "shlrv_12c_256": Workload(name="shlrv_12c_256", model="SHLR_V", J=12, M=256, N=256, window=16,
                              mask="poisson2d", R=5.0, n_acs=8, sigma_n=1e-3, seed=2,
                              beta=20.0, tau=20.0),
    # 8-coil 192x192 x 8 echoes T2 series, SHLR-VP, echo-varying 1D random R=6 + 8 ACS
    "shlrvp_8c_192_8e": Workload(name="shlrvp_8c_192_8e", model="SHLR_VP", J=8, M=192, N=192, L=8,
                                 window=12, window_param=4, mask="random1d", R=6.0, n_acs=8,
                                 sigma_n=1e-3, seed=4, te_ms=10.0, beta=20.0, tau=20.0, lam2=2.0),
    # the bench workload's data and mask with the SPIRiT term (Eq. 3 / Eq. 6): SHLR-S and
    # SHLR-SV, 5x5 kernel calibrated on the 24 ACS lines, X-update by 30 CG iterations
    "shlrs_12c_256": Workload(name="shlrs_12c_256", model="SHLR_S", J=12, M=256, N=256, window=16,
                              mask="random1d", R=4.0, n_acs=24, sigma_n=1e-3, seed=2,
                              beta=20.0, tau=20.0, lam1=1e3),
    "shlrsv_12c_256": Workload(name="shlrsv_12c_256", model="SHLR_SV", J=12, M=256, N=256, window=16,
                               mask="random1d", R=4.0, n_acs=24, sigma_n=1e-3, seed=2,
                               beta=20.0, tau=20.0, lam1=1e2),
    # the paper's further parallel-imaging patterns on the 12-coil 256x256 data:
    # uniform R = 6 with 20 ACS lines; that pattern with 3/4 partial Fourier; the
    # Gaussian Cartesian pattern (rate ~0.34) with 3/4 partial Fourier; the 2D
    # Poisson-disc pattern with 4/5 partial Fourier (SHLR-V)
    "shlr_12c_256_uniform6": Workload(name="shlr_12c_256_uniform6", model="SHLR", J=12, M=256, N=256,
                                      window=16, mask="uniform1d", R=6.0, n_acs=20, sigma_n=1e-3, seed=2,
                                      beta=20.0, tau=20.0),
    "shlr_12c_256_uniform6_pf34": Workload(name="shlr_12c_256_uniform6_pf34", model="SHLR", J=12, M=256, N=256,
                                           window=16, mask="uniform1d", R=6.0, n_acs=20, pf=0.75, sigma_n=1e-3,
                                           seed=2, beta=20.0, tau=20.0),
    "shlr_12c_256_gauss_pf34": Workload(name="shlr_12c_256_gauss_pf34", model="SHLR", J=12, M=256, N=256,
                                        window=16, mask="gauss1d", R=2.94, n_acs=24, pf=0.75, sigma_n=1e-3,
                                        seed=2, beta=20.0, tau=20.0),
    "shlrv_12c_256_poisson_pf45": Workload(name="shlrv_12c_256_poisson_pf45", model="SHLR_V", J=12, M=256,
                                           N=256, window=16, mask="poisson2d", R=5.0, n_acs=8, pf=0.8,
                                           sigma_n=1e-3, seed=2, beta=20.0, tau=20.0),
}

# the ACS-line sweep: Gaussian Cartesian masks of one sampling rate, different ACS counts
ACS_SWEEP = dict(rate=0.34, acs_lines=(8, 12, 16, 20, 24, 28, 32))


def get_config(name: str) -> Workload:
    return CONFIGS[name]


def unrolled_batch(n_inst: int = 16, n_iter: int = 10, window: int = 16, n_acs: int = 24):
    """The uneven batch of the differentiable unrolled reconstruction: n_inst
    SHLR instances with M = N in 128..320 and 8..32 coils (every size and
    coil count of the lists appears), window 16 (C p = 16 J up to 512
    columns), 1D random masks R = 4 with 24 ACS lines, noise 1e-3, n_iter
    unrolled iterations (the parallel-imaging recipe of the 12-coil workload).
    Deterministic: instance i takes sizes[i % 6], coils[3 i % 5]."""
    sizes = [128, 160, 192, 240, 256, 320]
    coils = [8, 12, 16, 24, 32]
    out = []
    for i in range(n_inst):
        n = sizes[i % len(sizes)]
        out.append(Workload(name=f"unrolled_{i:02d}", model="SHLR", J=coils[(3 * i) % len(coils)], M=n, N=n,
                            window=window, mask="random1d", R=4.0, n_acs=n_acs, sigma_n=1e-3, seed=500 + i,
                            beta=20.0, tau=20.0, n_iter=n_iter))
    return out


def unrolled_instance(name: str) -> Workload:
    """Instance `unrolled_NN` of unrolled_batch()."""
    return unrolled_batch()[int(name.split("_")[1])]
