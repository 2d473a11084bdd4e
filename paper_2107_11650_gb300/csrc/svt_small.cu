// Singular value thresholding (Eqs. 16-17, S8-S9) of many tiny lifted matrices,
// one warp per matrix, everything in registers.
//
// The parameter-dimension lifts of SHLR-P / SHLR-VP (Eq. 7/8) are (L - pP + 1)
// x (J pP) matrices, 5 x 32 for 8 echoes, 8 coils and pP = 4, and there is one
// per image pixel (36 864 for 192 x 192).  A CTA-per-matrix eigensolver leaves
// such a matrix one warp's worth of work in a 512-thread block; here each lane
// of a warp holds element e (and e + 32) of the s <= SMALL_S columns of
// B = A or A^T and the whole s x s rotation matrix Q:
//   one-sided Jacobi B Q = W (W^H W diagonal), the same rotation formulas and
//   stopping rule as k_jacobi (pair inner products by warp reduction; the
//   rotation of Q is replicated in every lane, so it needs no communication);
//   sigma_q = ||w_q||, h_q = max(1 - t / sigma_q, 0),
//   Z = sum_q h_q w_q q_q^H  (= U diag((sigma - t)_+) V^H),
// followed by the same epilogue as the other SVT paths: Z written out, or the
// multiplier update D <- D + tau (A - D/beta - Z), E = Z - D/beta (Eqs. 13-14).
#include "selr_internal.cuh"

#define SMALL_S 8           // largest s handled (templates for s <= 2, 4, 6, 8)
#define SMALL_E 2           // elements per lane: len <= 64
#define SMALL_WARPS 4

__device__ __forceinline__ float sw_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool small_frozen(const Group &g, int mat, const int *active) {
    if (!active) return false;
    if (g.kind == G_PE) return active[g.aoff + mat / g.L] == 0;
    if (g.kind == G_PARAM) return active[g.aoff + mat / g.N] == 0;
    return false;
}

template <int S>
__global__ void __launch_bounds__(SMALL_WARPS * 32) k_svt_small(GroupSet gs, int mat_begin, int mat_count, SvtArgs a) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int m = blockIdx.x * SMALL_WARPS + wib;
    if (m >= mat_count) return;                       // whole warp
    int mat;
    const int gi = find_group(gs, mat_begin + m, &mat);
    const Group &g = gs.g[gi];
    if (small_frozen(g, mat, a.active)) return;
    const int n = g.s, len = g.len;
    const long long base = g.off + (long long)mat * n * len;
    cf w[S][SMALL_E];
    cf q[S][S];                           // q[c][k]: component c of v_k
#pragma unroll
    for (int c = 0; c < S; ++c) {
#pragma unroll
        for (int k = 0; k < SMALL_E; ++k) {
            const int e = lane + 32 * k;
            w[c][k] = (c < n && e < len) ? a.B0[base + (long long)c * len + e] : mk(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < S; ++k) q[c][k] = mk(c == k ? 1.f : 0.f, 0.f);
    }
    int sweeps = 0;
    bool converged = false;
    for (sweeps = 1; sweeps <= a.max_sweeps; ++sweeps) {
        int rot = 0;
#pragma unroll
        for (int p = 0; p < S - 1; ++p) {
#pragma unroll
            for (int r = p + 1; r < S; ++r) {
                if (r >= n) continue;                 // uniform across the warp
                float aa = 0.f, bb = 0.f, cr = 0.f, ci = 0.f;
#pragma unroll
                for (int k = 0; k < SMALL_E; ++k) {
                    const cf x = w[p][k], y = w[r][k];
                    aa = fmaf(x.x, x.x, fmaf(x.y, x.y, aa));
                    bb = fmaf(y.x, y.x, fmaf(y.y, y.y, bb));
                    cr = fmaf(x.x, y.x, fmaf(x.y, y.y, cr));
                    ci = fmaf(x.x, y.y, fmaf(-x.y, y.x, ci));
                }
                aa = sw_sum(aa);
                bb = sw_sum(bb);
                cr = sw_sum(cr);
                ci = sw_sum(ci);
                const float d = sqrtf(cr * cr + ci * ci);
                if (!(d > a.tol * sqrtf(aa * bb)) || d == 0.f) continue;
                rot = 1;
                const float zeta = (bb - aa) / (2.f * d);
                const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                const float cs = rsqrtf(fmaf(tt, tt, 1.f));
                const float sn = cs * tt;
                const float snr = sn * cr / d, sni = sn * ci / d;
                // x' = cs x - (snr - i sni) y ; y' = (snr + i sni) x + cs y (columns p, r of W and Q)
#pragma unroll
                for (int k = 0; k < SMALL_E; ++k) {
                    const cf x = w[p][k], y = w[r][k];
                    w[p][k] = mk(cs * x.x - (snr * y.x + sni * y.y), cs * x.y - (snr * y.y - sni * y.x));
                    w[r][k] = mk(cs * y.x + (snr * x.x - sni * x.y), cs * y.y + (snr * x.y + sni * x.x));
                }
#pragma unroll
                for (int c = 0; c < S; ++c) {
                    const cf x = q[c][p], y = q[c][r];
                    q[c][p] = mk(cs * x.x - (snr * y.x + sni * y.y), cs * x.y - (snr * y.y - sni * y.x));
                    q[c][r] = mk(cs * y.x + (snr * x.x - sni * x.y), cs * y.y + (snr * x.y + sni * x.x));
                }
            }
        }
        if (!rot) { converged = true; break; }
    }
    // h_k = max(1 - t / sigma_k, 0)
    float h[S];
    int rank = 0;
    const float t = g.thresh;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        float s2 = 0.f;
#pragma unroll
        for (int j = 0; j < SMALL_E; ++j) s2 = fmaf(w[k][j].x, w[k][j].x, fmaf(w[k][j].y, w[k][j].y, s2));
        const float sg = sqrtf(sw_sum(s2));
        if (!isfinite(sg)) bad = true;
        h[k] = (k < n && sg > t) ? 1.f - t / sg : 0.f;
        if (k < n && sg > t) ++rank;
    }
    if (lane == 0) {
        if (bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
        if (!converged) atomicOr(a.status, (unsigned)ST_NOCONV);
        if (a.mat_status) a.mat_status[g.moff + mat] = converged ? sweeps : -a.max_sweeps;
        if (a.rank_out) a.rank_out[g.moff + mat] = rank;
    }
    const float ib = 1.f / a.beta;
#pragma unroll
    for (int j = 0; j < SMALL_E; ++j) {
        const int e = lane + 32 * j;
        if (e >= len) continue;
#pragma unroll
        for (int c = 0; c < S; ++c) {
            if (c >= n) continue;
            // Z[e][c] = sum_k h_k w_k[e] conj(q[c][k])
            float zr = 0.f, zi = 0.f;
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const cf x = w[k][j], v = q[c][k];
                zr = fmaf(h[k], x.x * v.x + x.y * v.y, zr);
                zi = fmaf(h[k], x.y * v.x - x.x * v.y, zi);
            }
            const long long vi = base + (long long)c * len + e;
            if (a.mode == 0) {
                if (a.z_natural) {
                    const int rr = g.trans ? c : e, cc = g.trans ? e : c;
                    a.Zout[base + (long long)rr * g.cols + cc] = mk(zr, zi);
                } else {
                    a.Zout[vi] = mk(zr, zi);
                }
            } else {
                const cf A = a.B0[vi];
                const cf Dv = a.D[vi];
                const cf Dn = mk(Dv.x + a.tau * (A.x - Dv.x * ib - zr), Dv.y + a.tau * (A.y - Dv.y * ib - zi));
                a.D[vi] = Dn;
                a.E[vi] = mk(zr - Dn.x * ib, zi - Dn.y * ib);
            }
        }
    }
}

bool svt_small_fits(const Group &g) { return g.s <= SMALL_S && g.len <= 32 * SMALL_E; }

cudaError_t launch_svt_small(const GroupSet &gs, int mat_begin, int mat_count, const SvtArgs &a, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    for (int k = 0; k < gs.n; ++k)
        if (!svt_small_fits(gs.g[k])) return cudaErrorInvalidValue;
    int smax = 0;
    for (int k = 0; k < gs.n; ++k) smax = max(smax, gs.g[k].s);
    const int blocks = (mat_count + SMALL_WARPS - 1) / SMALL_WARPS;
    if (smax <= 2) k_svt_small<2><<<blocks, SMALL_WARPS * 32, 0, st>>>(gs, mat_begin, mat_count, a);
    else if (smax <= 4) k_svt_small<4><<<blocks, SMALL_WARPS * 32, 0, st>>>(gs, mat_begin, mat_count, a);
    else if (smax <= 6) k_svt_small<6><<<blocks, SMALL_WARPS * 32, 0, st>>>(gs, mat_begin, mat_count, a);
    else k_svt_small<8><<<blocks, SMALL_WARPS * 32, 0, st>>>(gs, mat_begin, mat_count, a);
    return cudaGetLastError();
}
