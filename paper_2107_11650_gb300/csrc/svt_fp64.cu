// FP64 re-solve of the SVT (Eqs. 16-17, S8-S9) for the matrices that the FP32
// eigensolver flags as near-degenerate at the threshold.
//
// The eigensolver works on G = B^H B in FP32, whose eigenvalues carry an
// absolute error of order eps_32 * lambda_max.  When t^2 lies below the
// resolution floor F = 64 eps_32 lambda_max and G has eigenvalues between t^2
// and F, which singular values exceed t, and by how much, is not determined in
// FP32 (k_eigvec marks such a matrix with rank -1 and the FP32 apply kernels
// skip it).  This kernel then computes S_t of the matrix in FP64 by one-sided
// (Hestenes) Jacobi on B itself, W = B Q, sigma_i = ||w_i||,
//     S_t(B) = sum_{sigma_i > t} (1 - t / sigma_i) / sigma_i^2 w_i (w_i^H B),
// and writes the same outputs as the FP32 apply (Z, or the multiplier update
// D <- D + tau (A - D / beta - Z), E = Z - D / beta of Eqs. 13-14) and the rank.
// FP64 runs at a small fraction of the FP32 rate on this GPU, so a flagged
// matrix costs about 0.1 s; on the reconstructions' own lifts nothing is
// flagged (their sigma_max / t stays below ~200).
//
// Launch: gridDim.x CTAs, each with its own FP64 work copy (slot) in global
// memory; CTA b owns every gridDim.x-th matrix of the launch from b on, reads
// their flags in parallel and solves the flagged ones.
#include "selr_internal.cuh"

#include <float.h>

#define F64_THREADS 512
#define F64_WARPS (F64_THREADS / 32)
#define F64_SWEEPS 40
#define F64_TOL 1e-14
#define F64_MAXLEN 512

__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool frozen64(const Group &g, int mat, const int *active) {
    if (!active) return false;
    if (g.kind == G_PE) return active[g.aoff + mat / g.L] == 0;
    if (g.kind == G_PARAM) return active[g.aoff + mat / g.N] == 0;
    return false;
}

// Orthogonalise columns x and y (length len, FP64) in place; 1 if rotated.
__device__ int rot64(double2 *x, double2 *y, int len, int lane) {
    double a = 0.0, b = 0.0, cr = 0.0, ci = 0.0;
    for (int e = lane; e < len; e += 32) {
        const double2 xv = x[e], yv = y[e];
        a = fma(xv.x, xv.x, fma(xv.y, xv.y, a));
        b = fma(yv.x, yv.x, fma(yv.y, yv.y, b));
        cr = fma(xv.x, yv.x, fma(xv.y, yv.y, cr));
        ci = fma(xv.x, yv.y, fma(-xv.y, yv.x, ci));
    }
    a = wsum_d(a);
    b = wsum_d(b);
    cr = wsum_d(cr);
    ci = wsum_d(ci);
    const double d = sqrt(cr * cr + ci * ci);
    if (!(d > F64_TOL * sqrt(a * b)) || d == 0.0) return 0;
    const double zeta = (b - a) / (2.0 * d);
    const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
    const double cs = 1.0 / sqrt(fma(t, t, 1.0));
    const double sn = cs * t;
    const double snr = sn * cr / d, sni = sn * ci / d;
    for (int e = lane; e < len; e += 32) {
        const double2 xv = x[e], yv = y[e];
        double2 xn, yn;
        xn.x = cs * xv.x - (snr * yv.x + sni * yv.y);
        xn.y = cs * xv.y - (snr * yv.y - sni * yv.x);
        yn.x = cs * yv.x + (snr * xv.x - sni * xv.y);
        yn.y = cs * yv.y + (snr * xv.y + sni * xv.x);
        x[e] = xn;
        y[e] = yn;
    }
    return 1;
}

__device__ __forceinline__ void rr_pair64(int P, int r, int i, int *p, int *q) {
    if (i == 0) { *p = 0; *q = 1 + r; return; }
    const int n1 = P - 1;
    *p = 1 + (r + i) % n1;
    *q = 1 + (r - i + n1) % n1;
}

__global__ void __launch_bounds__(F64_THREADS) k_svt_fp64(GroupSet gs, int mat_begin, int mat_count, EigArgs ea,
                                                          SvtArgs a, double2 *work, long long slot_elems) {
    __shared__ int s_rot;
    __shared__ double s_sig[1024];
    __shared__ int s_list[F64_THREADS];
    __shared__ int s_cnt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double2 *W = work + (long long)blockIdx.x * slot_elems;
    // This CTA owns matrices q = blockIdx.x + gridDim.x * j.  Their flags are read F64_THREADS at a
    // time (one per thread) and the flagged ones of each chunk are then solved one after another.
    const int nmine = blockIdx.x < mat_count ? (mat_count - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    for (int base = 0; base < nmine; base += F64_THREADS) {
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        if (base + tid < nmine) {
            const int q = blockIdx.x + gridDim.x * (base + tid);
            int m;
            const Group &gq = gs.g[find_group(gs, mat_begin + q, &m)];
            if (!frozen64(gq, m, a.active) && ea.rank[gq.moff + m] < 0) s_list[atomicAdd(&s_cnt, 1)] = q;
        }
        __syncthreads();
        const int cnt = s_cnt;
        for (int li = 0; li < cnt; ++li) {
            int mat;
            const int gi = find_group(gs, mat_begin + s_list[li], &mat);
            const Group &g = gs.g[gi];
            const int n = g.s, len = g.len;
            if (len > F64_MAXLEN || (long long)n * len > slot_elems || n > 1024) {
                if (tid == 0) atomicOr(a.status, (unsigned)ST_NOCONV);
                continue;
            }
            const cf *B = ea.B0 + g.off + (long long)mat * n * len;
            for (long long i = tid; i < (long long)n * len; i += F64_THREADS)
                W[i] = make_double2((double)B[i].x, (double)B[i].y);
            __syncthreads();
            const int P = n + (n & 1);
            bool conv = false;
            for (int sweep = 0; sweep < F64_SWEEPS && !conv; ++sweep) {
                if (tid == 0) s_rot = 0;
                __syncthreads();
                for (int r = 0; r < P - 1; ++r) {
                    int mine = 0;
                    for (int i = warp; i < P / 2; i += F64_WARPS) {
                        int p, q;
                        rr_pair64(P, r, i, &p, &q);
                        if (p < n && q < n) mine += rot64(W + (long long)p * len, W + (long long)q * len, len, lane);
                    }
                    if (lane == 0 && mine) atomicAdd(&s_rot, mine);
                    __syncthreads();
                }
                conv = s_rot == 0;
                __syncthreads();
            }
            if (!conv && tid == 0) atomicOr(a.status, (unsigned)ST_NOCONV);
            // singular values
            for (int i = warp; i < n; i += F64_WARPS) {
                double s2 = 0.0;
                for (int e = lane; e < len; e += 32) s2 = fma(W[(long long)i * len + e].x, W[(long long)i * len + e].x,
                                                              fma(W[(long long)i * len + e].y, W[(long long)i * len + e].y, s2));
                s2 = wsum_d(s2);
                if (lane == 0) s_sig[i] = sqrt(s2);
            }
            __syncthreads();
            const double t = (double)g.thresh;
            int r = 0;
            for (int i = 0; i < n; ++i) r += s_sig[i] > t ? 1 : 0;
            if (tid == 0) {
                ea.rank[g.moff + mat] = r;
                if (ea.rank_acc) ea.rank_acc[g.moff + mat] += (unsigned long long)r;
                if (a.rank_out) a.rank_out[g.moff + mat] = r;
            }
            // column c of Z (vector-major): z_c = sum_i g_i (w_i^H b_c) w_i, one warp per column,
            // each lane holding elements e = lane + 32 u
            const float ib = 1.f / a.beta;
            for (int c = warp; c < n; c += F64_WARPS) {
                double2 z[F64_MAXLEN / 32];
    #pragma unroll
                for (int u = 0; u < F64_MAXLEN / 32; ++u) z[u] = make_double2(0.0, 0.0);
                const cf *bc = B + (long long)c * len;
                for (int i = 0; i < n; ++i) {
                    const double si = s_sig[i];
                    if (!(si > t)) continue;                   // warp-uniform
                    const double2 *wi = W + (long long)i * len;
                    double dr = 0.0, di = 0.0;                 // w_i^H b_c
                    for (int e = lane; e < len; e += 32) {
                        const double2 w = wi[e];
                        const double bx = (double)bc[e].x, by = (double)bc[e].y;
                        dr = fma(w.x, bx, fma(w.y, by, dr));
                        di = fma(w.x, by, fma(-w.y, bx, di));
                    }
                    dr = wsum_d(dr);
                    di = wsum_d(di);
                    const double gi_ = (1.0 - t / si) / (si * si);
                    dr *= gi_;
                    di *= gi_;
    #pragma unroll
                    for (int u = 0; u < F64_MAXLEN / 32; ++u) {
                        const int e = lane + 32 * u;
                        if (e < len) {
                            const double2 w = wi[e];
                            z[u].x = fma(w.x, dr, fma(-w.y, di, z[u].x));
                            z[u].y = fma(w.x, di, fma(w.y, dr, z[u].y));
                        }
                    }
                }
    #pragma unroll
                for (int u = 0; u < F64_MAXLEN / 32; ++u) {
                    const int e = lane + 32 * u;
                    if (e >= len) continue;
                    const long long vi = g.off + (long long)mat * n * len + (long long)c * len + e;
                    const cf zf = mk((float)z[u].x, (float)z[u].y);
                    if (a.mode == 0) {
                        if (a.z_natural) {
                            int rr, cc;
                            if (g.trans) { rr = c; cc = e; } else { rr = e; cc = c; }
                            a.Zout[g.off + (long long)mat * n * len + (long long)rr * g.cols + cc] = zf;
                        } else {
                            a.Zout[vi] = zf;
                        }
                    } else {
                        const cf A = bc[e];
                        const cf Dv = a.D[vi];
                        cf Dn;
                        Dn.x = Dv.x + a.tau * (A.x - Dv.x * ib - zf.x);
                        Dn.y = Dv.y + a.tau * (A.y - Dv.y * ib - zf.y);
                        a.D[vi] = Dn;
                        a.E[vi] = mk(zf.x - Dn.x * ib, zf.y - Dn.y * ib);
                    }
                }
            }
            __syncthreads();
        }
        __syncthreads();                                   // s_cnt / s_list reused by the next chunk
    }
}

cudaError_t launch_svt_fp64(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, const SvtArgs &a,
                            void *work, long long slot_elems, int slots, cudaStream_t st) {
    if (mat_count <= 0 || !work || slots <= 0) return cudaSuccess;
    k_svt_fp64<<<slots, F64_THREADS, 0, st>>>(gs, mat_begin, mat_count, ea, a, (double2 *)work, slot_elems);
    return cudaGetLastError();
}
