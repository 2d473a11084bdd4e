// Singular value thresholding S_t (Eqs. 16-17, S8-S9) of every lifted matrix,
// and the fused multiplier / adjoint-input update (Eqs. 13-14).
//
// Method.  For a matrix A (rows x cols) let B be A (cols <= rows) or A^T,
// stored vector-major: its s = min(rows, cols) columns of length len.
// One-sided (Hestenes) Jacobi rotates pairs of columns of B until all are
// mutually orthogonal: B Q = W, W^H W = diag(sigma^2), Q unitary, so the
// sigma_i = ||w_i|| are the singular values and u_i = w_i / sigma_i the
// corresponding singular vectors of B.  Then
//     S_t(B) = sum_{sigma_i > t} (1 - t / sigma_i) / sigma_i^2 * w_i (w_i^H B),
// which needs W and the original B but never Q.  S_t(A^T) = S_t(A)^T.
// Working on B directly (no Gram matrix) keeps the FP32 error at the level of
// eps * sigma_max instead of eps * sigma_max^2 / sigma.
//
// Rotation of a pair (x, y): a = ||x||^2, b = ||y||^2, c = x^H y = |c| e^{i phi};
// zeta = (b - a) / (2|c|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// cs = 1 / sqrt(1 + t^2), sn = cs t;
//     x <- cs x - sn e^{-i phi} y,   y <- sn e^{i phi} x + cs y,
// which makes x^H y = 0 (a <- a - t|c|, b <- b + t|c|).  A pair is rotated only
// while |c| > tol sqrt(a b); a sweep that rotates nothing ends the loop.
//
// Scheduling.  One CTA per matrix; one warp per column pair.  If all s
// columns fit in shared memory, rounds of the circle (round-robin) ordering
// run on the resident matrix.  Otherwise the columns are split into blocks of
// bc columns held two at a time: a sweep visits every block pair (I, J) once,
// rotating I x J cross pairs in bc rounds (pair (k, (k + r) mod P)), and each
// block's internal pairs once (on its first visit).  The sweep count is
// capped; a matrix that hits the cap is flagged (SELR_ERR_NO_CONVERGENCE).
#include "selr_internal.cuh"

#define JAC_THREADS 1024
#define JAC_WARPS (JAC_THREADS / 32)
#define APPLY_THREADS 256
#define APPLY_TC 16
#define APPLY_CH 16

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Is the matrix `mat` of group g frozen (parameter models, converged FE position)?
__device__ __forceinline__ bool frozen(const Group &g, int mat, const int *active) {
    if (!active) return false;
    if (g.kind == G_PE) return active[g.aoff + mat / g.L] == 0;
    if (g.kind == G_PARAM) return active[g.aoff + mat / g.N] == 0;
    return false;
}

// Orthogonalise columns x and y (length len) in place; returns 1 if rotated.
// The rotation is chosen from the first dlen entries and applied to all len
// (dlen < len: Jacobi on [B; I], which accumulates the rotations below B).
__device__ __forceinline__ int rotate_pair(cf *x, cf *y, int len, int dlen, float tol, int lane) {
    float a = 0.f, b = 0.f, cr = 0.f, ci = 0.f;
    for (int e = lane; e < dlen; e += 32) {
        const cf xv = x[e], yv = y[e];
        a = fmaf(xv.x, xv.x, fmaf(xv.y, xv.y, a));
        b = fmaf(yv.x, yv.x, fmaf(yv.y, yv.y, b));
        cr = fmaf(xv.x, yv.x, fmaf(xv.y, yv.y, cr));
        ci = fmaf(xv.x, yv.y, fmaf(-xv.y, yv.x, ci));
    }
    a = warp_sum(a);
    b = warp_sum(b);
    cr = warp_sum(cr);
    ci = warp_sum(ci);
    const float d = sqrtf(cr * cr + ci * ci);
    if (!(d > tol * sqrtf(a * b)) || d == 0.f) return 0;
    const float zeta = (b - a) / (2.f * d);
    const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
    const float cs = rsqrtf(fmaf(t, t, 1.f));
    const float sn = cs * t;
    const float pr = cr / d, pi = ci / d;           // e^{i phi}
    // sn e^{-i phi} and sn e^{i phi}
    const float snr = sn * pr, sni = sn * pi;
    for (int e = lane; e < len; e += 32) {
        const cf xv = x[e], yv = y[e];
        // x' = cs x - (snr - i sni) y ; y' = (snr + i sni) x + cs y
        cf xn, yn;
        xn.x = cs * xv.x - (snr * yv.x + sni * yv.y);
        xn.y = cs * xv.y - (snr * yv.y - sni * yv.x);
        yn.x = cs * yv.x + (snr * xv.x - sni * xv.y);
        yn.y = cs * yv.y + (snr * xv.y + sni * xv.x);
        x[e] = xn;
        y[e] = yn;
    }
    return 1;
}

// Circle-method pair i of round r among P (even) players.
__device__ __forceinline__ void rr_pair(int P, int r, int i, int *p, int *q) {
    if (i == 0) { *p = 0; *q = 1 + r; return; }
    const int n1 = P - 1;
    *p = 1 + (r + i) % n1;
    *q = 1 + (r - i + n1) % n1;
}

__device__ void copy_in(cf *dst, const cf *src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
__device__ void copy_out(cf *dst, const cf *src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Round-robin sweep over the `cnt` columns starting at `base` (smem).
__device__ void intra_rounds(cf *base, int cnt, int len, int dlen, float tol, int *rot) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (cnt < 2) return;
    const int P = cnt + (cnt & 1);
    for (int r = 0; r < P - 1; ++r) {
        int mine = 0;
        for (int i = warp; i < P / 2; i += JAC_WARPS) {
            int p, q;
            rr_pair(P, r, i, &p, &q);
            if (p < cnt && q < cnt)
                mine += rotate_pair(base + (long long)p * len, base + (long long)q * len, len, dlen, tol, lane);
        }
        if (lane == 0 && mine) atomicAdd(rot, mine);
        __syncthreads();
    }
}

// All cross pairs between block I (cntI columns at bI) and block J (cntJ at bJ).
__device__ void cross_rounds(cf *bI, int cntI, cf *bJ, int cntJ, int len, int dlen, float tol, int *rot) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = max(cntI, cntJ);
    for (int r = 0; r < P; ++r) {
        int mine = 0;
        for (int k = warp; k < P; k += JAC_WARPS) {
            const int q = (k + r) % P;
            if (k < cntI && q < cntJ)
                mine += rotate_pair(bI + (long long)k * len, bJ + (long long)q * len, len, dlen, tol, lane);
        }
        if (lane == 0 && mine) atomicAdd(rot, mine);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(JAC_THREADS, 1)
k_jacobi(GroupSet gs, int mat_begin, SvtArgs a, int cap_vecs_bytes) {
    extern __shared__ cf jsm[];
    __shared__ int rot;
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    if (frozen(g, mat, a.active)) return;
    const int s = g.s, len = g.len, dlen = g.dlen > 0 ? g.dlen : g.len;
    cf *W = a.W + g.off + (long long)mat * s * len;
    const int cap = cap_vecs_bytes / (int)(len * sizeof(cf));   // columns that fit in smem
    int sweeps = 0;
    bool converged = false;
    if (s <= cap) {
        copy_in(jsm, W, s * len);
        __syncthreads();
        for (sweeps = 1; sweeps <= a.max_sweeps; ++sweeps) {
            if (threadIdx.x == 0) rot = 0;
            __syncthreads();
            intra_rounds(jsm, s, len, dlen, a.tol, &rot);
            const int r = rot;
            __syncthreads();
            if (r == 0) { converged = true; break; }
        }
        copy_out(W, jsm, s * len);
    } else {
        const int bc = cap / 2;
        const int nb = (s + bc - 1) / bc;
        cf *slotI = jsm, *slotJ = jsm + (long long)bc * len;
        for (sweeps = 1; sweeps <= a.max_sweeps; ++sweeps) {
            if (threadIdx.x == 0) rot = 0;
            __syncthreads();
            for (int I = 0; I < nb; ++I) {
                const int cI = min(bc, s - I * bc);
                copy_in(slotI, W + (long long)I * bc * len, cI * len);
                __syncthreads();
                intra_rounds(slotI, cI, len, dlen, a.tol, &rot);
                for (int J = I + 1; J < nb; ++J) {
                    const int cJ = min(bc, s - J * bc);
                    copy_in(slotJ, W + (long long)J * bc * len, cJ * len);
                    __syncthreads();
                    cross_rounds(slotI, cI, slotJ, cJ, len, dlen, a.tol, &rot);
                    copy_out(W + (long long)J * bc * len, slotJ, cJ * len);
                    __syncthreads();
                }
                copy_out(W + (long long)I * bc * len, slotI, cI * len);
                __syncthreads();
            }
            const int r = rot;
            __syncthreads();
            if (r == 0) { converged = true; break; }
        }
    }
    __syncthreads();
    // singular values = column norms of the orthogonalised matrix
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool bad = false;
    for (int v = warp; v < s; v += JAC_WARPS) {
        float acc = 0.f;
        for (int e = lane; e < dlen; e += 32) {
            const cf x = W[(long long)v * len + e];
            acc = fmaf(x.x, x.x, fmaf(x.y, x.y, acc));
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const float sg = sqrtf(acc);
            a.sigma[g.soff + (long long)mat * s + v] = sg;
            if (!isfinite(sg)) bad = true;
        }
    }
    if (bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    if (threadIdx.x == 0) {
        if (a.mat_status) a.mat_status[g.moff + mat] = converged ? sweeps : -a.max_sweeps;
        if (!converged) atomicOr(a.status, (unsigned)ST_NOCONV);
    }
}

static int g_jacobi_smem = 0;
static bool g_apply_attr = false;

cudaError_t launch_jacobi(const GroupSet &gs, int mat_begin, int mat_count, const SvtArgs &a, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    if (g_jacobi_smem == 0) return cudaErrorNotReady;
    // Use only as much shared memory as the largest matrix needs (resident case)
    size_t need = 0;
    for (int k = 0; k < gs.n; ++k) need = max(need, (size_t)gs.g[k].s * gs.g[k].len * sizeof(cf));
    const int smem = (int)min(need, (size_t)g_jacobi_smem);
    k_jacobi<<<mat_count, JAC_THREADS, smem, st>>>(gs, mat_begin, a, smem);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ apply
// Z_B[:, c] = sum_{sigma_i > t} coef_i w_i (w_i^H B0[:, c]),  coef_i = (1 - t/sigma_i)/sigma_i^2,
// for a tile of APPLY_TC columns c; then either write Z or do the ADMM update
//   D <- D + tau (A - D/beta - Z),  E <- Z - D/beta   (A = B0 = lift(X) + D_old/beta).
__global__ void __launch_bounds__(APPLY_THREADS)
k_svt_apply(GroupSet gs, int mat_begin, SvtArgs a) {
    extern __shared__ cf asm_[];
    __shared__ int sel[1024];
    __shared__ float coef[1024];
    __shared__ int nsel;
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    if (frozen(g, mat, a.active)) return;
    const int s = g.s, len = g.len;
    const int c0 = blockIdx.y * APPLY_TC;
    if (c0 >= s) return;
    const int tc = min(APPLY_TC, s - c0);
    const long long mb = g.off + (long long)mat * s * len;
    const float t = g.thresh;
    cf *B0t = asm_;                                  // [APPLY_TC][len]
    cf *Wc = asm_ + APPLY_TC * len;                  // [APPLY_CH][len]
    cf *Ys = Wc + APPLY_CH * len;                    // [APPLY_CH][APPLY_TC]

    if (threadIdx.x == 0) {
        int n = 0;
        for (int i = 0; i < s; ++i) {
            const float sg = a.sigma[g.soff + (long long)mat * s + i];
            if (sg > t) {
                sel[n] = i;
                coef[n] = (1.f - t / sg) / (sg * sg);
                ++n;
            }
        }
        nsel = n;
        if (a.rank_out && blockIdx.y == 0) a.rank_out[g.moff + mat] = n;
    }
    for (int i = threadIdx.x; i < tc * len; i += APPLY_THREADS) B0t[i] = a.B0[mb + (long long)c0 * len + i];
    __syncthreads();
    const int r = nsel;
    constexpr int MAXE = (APPLY_TC * 512 + APPLY_THREADS - 1) / APPLY_THREADS;
    const int nel = tc * len;
    cf z[MAXE];
#pragma unroll
    for (int k = 0; k < MAXE; ++k) z[k] = mk(0.f, 0.f);

    for (int i0 = 0; i0 < r; i0 += APPLY_CH) {
        const int ch = min(APPLY_CH, r - i0);
        for (int i = threadIdx.x; i < ch * len; i += APPLY_THREADS) {
            const int k = i / len, e = i - k * len;
            Wc[i] = a.W[mb + (long long)sel[i0 + k] * len + e];
        }
        __syncthreads();
        {
            const int k = threadIdx.x / APPLY_TC, c = threadIdx.x - k * APPLY_TC;
            if (k < ch && c < tc) {
                float yr = 0.f, yi = 0.f;
                const cf *wk = Wc + k * len, *bc = B0t + c * len;
                for (int e = 0; e < len; ++e) {
                    const cf wv = wk[e], bv = bc[e];
                    yr = fmaf(wv.x, bv.x, fmaf(wv.y, bv.y, yr));
                    yi = fmaf(wv.x, bv.y, fmaf(-wv.y, bv.x, yi));
                }
                const float cf_ = coef[i0 + k];
                Ys[k * APPLY_TC + c] = mk(yr * cf_, yi * cf_);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < MAXE; ++kk) {
            const int idx = threadIdx.x + kk * APPLY_THREADS;
            if (idx < nel) {
                const int c = idx / len, e = idx - c * len;
                cf acc = z[kk];
                for (int k = 0; k < ch; ++k) acc = cadd(acc, cmul(Wc[k * len + e], Ys[k * APPLY_TC + c]));
                z[kk] = acc;
            }
        }
        __syncthreads();
    }
    const float ib = 1.f / a.beta;
#pragma unroll
    for (int kk = 0; kk < MAXE; ++kk) {
        const int idx = threadIdx.x + kk * APPLY_THREADS;
        if (idx < nel) {
            const int c = idx / len, e = idx - c * len;
            const long long vi = mb + (long long)(c0 + c) * len + e;
            if (a.mode == 0) {
                if (a.z_natural) {
                    int rr, cc;
                    if (g.trans) { rr = c0 + c; cc = e; } else { rr = e; cc = c0 + c; }
                    a.Zout[g.off + (long long)mat * s * len + (long long)rr * g.cols + cc] = z[kk];
                } else {
                    a.Zout[vi] = z[kk];
                }
            } else {
                const cf A = B0t[idx];
                const cf Dv = a.D[vi];
                cf Dn;
                Dn.x = Dv.x + a.tau * (A.x - Dv.x * ib - z[kk].x);
                Dn.y = Dv.y + a.tau * (A.y - Dv.y * ib - z[kk].y);
                a.D[vi] = Dn;
                a.E[vi] = mk(z[kk].x - Dn.x * ib, z[kk].y - Dn.y * ib);
            }
        }
    }
}

cudaError_t launch_svt_apply(const GroupSet &gs, int mat_begin, int mat_count, const SvtArgs &a, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    int maxlen = 0, maxs = 0;
    for (int k = 0; k < gs.n; ++k) { maxlen = max(maxlen, gs.g[k].len); maxs = max(maxs, gs.g[k].s); }
    if (maxlen > 512 || maxs > 1024) return cudaErrorInvalidValue;
    const size_t smem = sizeof(cf) * ((APPLY_TC + APPLY_CH) * (size_t)maxlen + APPLY_CH * APPLY_TC);
    if (!g_apply_attr) return cudaErrorNotReady;
    dim3 grid(mat_count, (maxs + APPLY_TC - 1) / APPLY_TC);
    k_svt_apply<<<grid, APPLY_THREADS, smem, st>>>(gs, mat_begin, a);
    return cudaGetLastError();
}

// Called at plan creation (outside any stream capture): opt the SVT kernels
// into large dynamic shared memory.
cudaError_t svt_init_attributes() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int jsm = optin - 1024;   // leave room for the static shared counter
    e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, jsm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_svt_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(cf) * ((APPLY_TC + APPLY_CH) * 512 + APPLY_CH * APPLY_TC)));
    if (e != cudaSuccess) return e;
    g_jacobi_smem = jsm;
    g_apply_attr = true;
    return cudaSuccess;
}

