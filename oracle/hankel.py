"""Hankel lifts of the SHLR family and their real adjoints.

Test infrastructure only (see ``oracle/__init__.py``).

Definitions (Sec. III-A, Eq. 2 and Eq. 4):
* H maps v in C^N to the (N-p+1) x p Hankel matrix (H v)[i, c] = v[i + c].
  Reading: the paper fixes neither orientation nor window; rows index the
  position i, columns the window tap c, and channels are concatenated
  horizontally, so a lift with C channels is (N-p+1) x (C*p).
* H~ W~ F~ P_m X = [H W F x_{m,1}, ..., H W F x_{m,J}] (Eq. 2); the vectors
  handed to the functions below are already F^1D-transformed (a row of the
  hybrid array F^1D applied along that row), so the lift here applies W then H.
* H~_vc (Eq. 4) appends the channels H W (F x_j)^dagger, where dagger takes
  the complex conjugate and flips the vector about its centre.  Reading: the
  flip is the reversal i -> N-1-i, applied before W.
* The VC channels are antilinear in x, so adjoints are taken for the real
  inner product Re<a, b>.
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------ single vector
def hankel(v, p):
    """(H v)[i, c] = v[i + c] for 0 <= i < N-p+1, 0 <= c < p."""
    N = v.shape[-1]
    l = N - p + 1
    idx = np.arange(l)[:, None] + np.arange(p)[None, :]
    return v[..., idx]


def hankel_adjoint(E, N):
    """(H* E)[k] = sum over entries (i, c) with i + c = k of E[i, c]."""
    l, p = E.shape[-2], E.shape[-1]
    assert l + p - 1 == N
    out = np.zeros(E.shape[:-2] + (N,), dtype=np.result_type(E, np.complex128))
    for q in range(p):
        out[..., q:q + l] += E[..., :, q]
    return out


def dagger(v):
    """Conjugate and flip about the centre: v^dagger[i] = conj(v[N-1-i]) (Eq. 4)."""
    return np.conj(v[..., ::-1])


# ------------------------------------------------------------ channel lifts
def lift_vectors(V, w, p, vc):
    """Lift a set of J vectors V[..., j, :] (length N, already in the lift's
    Fourier domain) into [H(w V_1) ... H(w V_J) (| H(w V_1^+) ... H(w V_J^+))].

    ``w`` is None for the parameter-dimension lift (no W, Eq. 7/8).
    Returns [..., N-p+1, C*p] with C = J or 2J.
    """
    if w is None:
        w = np.ones(V.shape[-1])
    chans = [w * V]
    if vc:
        chans.append(w * dagger(V))
    V2 = np.concatenate(chans, axis=-2)                  # [..., C, N]
    H = hankel(V2, p)                                    # [..., C, l, p]
    H = np.moveaxis(H, -3, -2)                           # [..., l, C, p]
    return H.reshape(H.shape[:-2] + (H.shape[-2] * H.shape[-1],))


def lift_vectors_adjoint(E, w, p, vc, J, N):
    """Real adjoint of :func:`lift_vectors`: E [..., l, C*p] -> [..., J, N].

    Plain channel j : conj(w) * H*(E_j).
    VC channel j    : flip(w * conj(H*(E_{J+j})))   (the real adjoint of
                      v -> H(w * conj(flip v))).
    """
    if w is None:
        w = np.ones(N)
    l = N - p + 1
    C = 2 * J if vc else J
    Ec = E.reshape(E.shape[:-1] + (C, p))
    Ec = np.moveaxis(Ec, -2, -3)                         # [..., C, l, p]
    h = hankel_adjoint(Ec, N)                            # [..., C, N]
    out = np.conj(w) * h[..., :J, :]
    if vc:
        out = out + (w * np.conj(h[..., J:, :]))[..., ::-1]
    return out


# ------------------------------------------------- 2D row / column lifts
def lift_rows(R, w, p, vc):
    """Row lifts of Eq. 2 / Eq. 4 for all m.

    R is the hybrid array F^1D applied along n (R = F_m^* K): [J][M][N].
    Returns [M][N-p+1][C*p]."""
    V = np.moveaxis(R, 1, 0)                             # [M][J][N]
    return lift_vectors(V, w, p, vc)


def lift_rows_adjoint(E, w, p, vc, J, N):
    """Adjoint of :func:`lift_rows`: [M][l][Cp] -> hybrid [J][M][N]."""
    out = lift_vectors_adjoint(E, w, p, vc, J, N)        # [M][J][N]
    return np.moveaxis(out, 0, 1)


def lift_cols(Cc, w, p, vc):
    """Column lifts for all n.  Cc = F_n^* K is F^1D along m: [J][M][N].
    Returns [N][M-p+1][C*p]."""
    V = np.transpose(Cc, (2, 0, 1))                      # [N][J][M]
    return lift_vectors(V, w, p, vc)


def lift_cols_adjoint(E, w, p, vc, J, M):
    """Adjoint of :func:`lift_cols`: [N][l][Cp] -> hybrid [J][M][N]."""
    out = lift_vectors_adjoint(E, w, p, vc, J, M)        # [N][J][M]
    return np.transpose(out, (1, 2, 0))


# -------------------------------------------- parameter imaging (Eq. 7/8)
def lift_pe(Kp, w, p, vc):
    """PE lifts H~(_vc) W~ F~ Q_l X_m for every (m, l) (Eq. 7 / 8).

    Kp is X already transformed along PE (the k_n domain): [L][J][M][N].
    Returns [M*L][N-p+1][C*p] ordered (m, l)."""
    L, J, M, N = Kp.shape
    V = np.transpose(Kp, (2, 0, 1, 3)).reshape(M * L, J, N)
    return lift_vectors(V, w, p, vc)


def lift_pe_adjoint(E, w, p, vc, L, J, M, N):
    out = lift_vectors_adjoint(E, w, p, vc, J, N)        # [M*L][J][N]
    return np.transpose(out.reshape(M, L, J, N), (1, 2, 0, 3))


def lift_param(Xi, pP):
    """Parameter-dimension lifts H~ P_n X_m for every (m, n) (Eq. 7 / 8): the
    echo vector (length L) of each coil at image position (m, n), no F, no W.

    Xi is the image [L][J][M][N].  Returns [M*N][L-pP+1][J*pP] ordered (m, n)."""
    L, J, M, N = Xi.shape
    V = np.transpose(Xi, (2, 3, 1, 0)).reshape(M * N, J, L)
    return lift_vectors(V, None, pP, False)


def lift_param_adjoint(E, pP, L, J, M, N):
    out = lift_vectors_adjoint(E, None, pP, False, J, L)  # [M*N][J][L]
    return np.transpose(out.reshape(M, N, J, L), (3, 2, 0, 1))
