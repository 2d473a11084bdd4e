// Reverse-mode pieces of the unrolled reconstruction: the vector-Jacobian
// product of the SVT (Eqs. 16-17) through the Daleckii-Krein formula, the
// X-update (Eq. 15) scaling, and small batched linear-algebra helpers.
//
// SVT VJP.  For B (len x s, s <= len) with G = B^H B = V diag(lambda) V^H,
//     Z = S_t(B) = B h(G),   h(lambda) = max(1 - t / sqrt(lambda), 0).
// For a cotangent Zbar (real inner product Re tr(Zbar^H dZ)):
//     Bbar = Zbar h(G) + B (Gbar + Gbar^H),
//     Gbar = V [Gamma o (V^H B^H Zbar V)] V^H,
//     Gamma_ij = (h(lambda_i) - h(lambda_j)) / (lambda_i - lambda_j)
//               (h'(lambda_i) where lambda_i = lambda_j),
//     tbar = -Re sum_{lambda_i > t^2} (V^H B^H Zbar V)_ii / sqrt(lambda_i).
// dh(G) follows the Daleckii-Krein theorem for the matrix function h; the
// divided difference is the 1 / (sigma_i^2 - sigma_j^2) term of the
// singular-vector derivative, guarded by evaluating it in a form without
// cancellation (k_gamma).  The eigenpairs of G come from one-sided Jacobi on
// [B; I] (k_augment, k_jacobi with rotations chosen on B, k_split_aug): the
// accumulated rotations Q stay orthonormal inside clusters of small singular
// values, where eigenvectors from inverse iteration would not.  Each FP32
// rotation is unitary only to O(u), so after ~sweeps * s rotations Q^H Q - I
// reaches ~1e-5; one Newton-Schulz (polar) step [BQ; Q] <- [BQ; Q](3I - Q^H Q)/2
// squares that error away and keeps the top block equal to B Q.  Then
// lambda_i = ||B v_i||^2.
#include "selr_internal.cuh"

#include <float.h>

// ------------------------------------------------------------------- GEMM
// C[b] = alpha op(A[b]) op(B[b]) + beta C[b] for row-major complex matrices.
// op: 0 = N, 1 = T (transpose), 2 = H (conjugate transpose), 3 = C (conjugate).
// A: op(A) is m x k; B: op(B) is k x n; lda/ldb/ldc are row strides of the
// stored matrices, sa/sb/sc batch strides (elements).
#define GM_T 32
#define GM_K 16
__device__ __forceinline__ cf opload(const cf *M, int op, long long ld, int r, int c) {
    // element (r, c) of op(M)
    cf v = (op == 0 || op == 3) ? M[(long long)r * ld + c] : M[(long long)c * ld + r];
    if (op == 2 || op == 3) v.y = -v.y;
    return v;
}

__global__ void __launch_bounds__(256) k_cgemm(int m, int n, int k, cf alpha, const cf *A, int opa, long long lda,
                                               long long sa, const cf *B, int opb, long long ldb, long long sb,
                                               cf beta, cf *C, long long ldc, long long sc) {
    __shared__ cf As[GM_K][GM_T + 1], Bs[GM_K][GM_T + 1];
    const int b = blockIdx.z;
    const cf *Ab = A + (long long)b * sa, *Bb = B + (long long)b * sb;
    cf *Cb = C + (long long)b * sc;
    const int r0 = blockIdx.y * GM_T, c0 = blockIdx.x * GM_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;     // 2x2 outputs per thread
    float ar[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, ai[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < k; k0 += GM_K) {
        for (int idx = threadIdx.x; idx < GM_K * GM_T; idx += 256) {
            const int kk = idx % GM_K, rr = idx / GM_K;
            const int gk = k0 + kk;
            As[kk][rr] = (r0 + rr < m && gk < k) ? opload(Ab, opa, lda, r0 + rr, gk) : mk(0.f, 0.f);
            Bs[kk][rr] = (c0 + rr < n && gk < k) ? opload(Bb, opb, ldb, gk, c0 + rr) : mk(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GM_K; ++kk) {
            const cf a0 = As[kk][ty], a1 = As[kk][ty + 16], b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            const cf aa[2] = {a0, a1}, bb[2] = {b0, b1};
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    ar[u][w] = fmaf(aa[u].x, bb[w].x, fmaf(-aa[u].y, bb[w].y, ar[u][w]));
                    ai[u][w] = fmaf(aa[u].x, bb[w].y, fmaf(aa[u].y, bb[w].x, ai[u][w]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            const int r = r0 + ty + 16 * u, c = c0 + tx + 16 * w;
            if (r < m && c < n) {
                const cf acc = mk(ar[u][w], ai[u][w]);
                cf out = cmul(alpha, acc);
                if (beta.x != 0.f || beta.y != 0.f) out = cadd(out, cmul(beta, Cb[(long long)r * ldc + c]));
                Cb[(long long)r * ldc + c] = out;
            }
        }
}

cudaError_t launch_cgemm(int batch, int m, int n, int k, cf alpha, const cf *A, int opa, long long lda, long long sa,
                         const cf *B, int opb, long long ldb, long long sb, cf beta, cf *C, long long ldc,
                         long long sc, cudaStream_t st) {
    if (batch <= 0 || m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((n + GM_T - 1) / GM_T, (m + GM_T - 1) / GM_T, batch);
    k_cgemm<<<grid, 256, 0, st>>>(m, n, k, alpha, A, opa, lda, sa, B, opb, ldb, sb, beta, C, ldc, sc);
    return cudaGetLastError();
}

// ------------------------------------------------------------- SVT VJP parts
__device__ __forceinline__ float hfun(float lam, float t) {
    const float sg = sqrtf(fmaxf(lam, 0.f));
    return sg > t ? 1.f - t / sg : 0.f;
}

// M[b][i][j] <- Gamma_ij M[b][i][j] (eigenvalues in any order).  Written in
// sigma = sqrt(lambda) so that no difference of nearly equal numbers is formed:
//   both above t:  (h(l_i) - h(l_j)) / (l_i - l_j) = t / (s_i s_j (s_i + s_j))
//                  (at s_i = s_j this is h'(lambda) = t / (2 s^3): no guard needed);
//   one above t:   h(l_i) / (l_i - l_j) with l_i > t^2 >= l_j;   none: 0.
__global__ void k_gamma(int s, const float *lam, float t, cf *M, long long sm, long long sl) {
    const int b = blockIdx.y;
    const float *lb = lam + (long long)b * sl;
    cf *Mb = M + (long long)b * sm;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < s * s; idx += gridDim.x * blockDim.x) {
        const int i = idx / s, j = idx - i * s;
        const float li = fmaxf(lb[i], 0.f), lj = fmaxf(lb[j], 0.f);
        const float si = sqrtf(li), sj = sqrtf(lj);
        const bool ai = si > t, aj = sj > t;
        float gmm = 0.f;
        if (ai && aj) gmm = t / (si * sj * (si + sj));
        else if (ai) gmm = (1.f - t / si) / (li - lj);
        else if (aj) gmm = (1.f - t / sj) / (lj - li);
        Mb[idx] = cscale(Mb[idx], gmm);
    }
}

// Vs[b][q][i] = f(lam[b][q]) * V[b][q][i] with f = h (mode 0) or 1/sqrt(lam) on the
// selected pairs (mode 1: lam > t^2, else 0).  V stored eigenvector-major.
__global__ void k_scale_vecs(int s, const float *lam, float t, const cf *V, cf *Vs, long long sv, long long sl,
                             int mode) {
    const int b = blockIdx.y;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < s * s; idx += gridDim.x * blockDim.x) {
        const int q = idx / s;
        const float l = lam[(long long)b * sl + q];
        const float sg = sqrtf(fmaxf(l, 0.f));
        float f;
        if (mode == 0) f = hfun(l, t);
        else f = sg > t ? 1.f / sg : 0.f;
        Vs[(long long)b * sv + idx] = cscale(V[(long long)b * sv + idx], f);
    }
}

// out[b] = -Re sum_i (V^H C V)_ii / sqrt(lam_i) over lam_i > t^2, summed over b into
// *tbar (single block, fixed order => deterministic).  Ct holds V^H C V.
__global__ void k_tbar(int batch, int s, const float *lam, float t, const cf *Ct, long long sm, long long sl,
                       float *tbar) {
    __shared__ double red[256];
    double acc = 0.0;
    for (long long idx = threadIdx.x; idx < (long long)batch * s; idx += blockDim.x) {
        const int b = (int)(idx / s), i = (int)(idx - (long long)b * s);
        const double sg = sqrt((double)fmaxf(lam[(long long)b * sl + i], 0.f));
        if (sg > t) acc -= (double)Ct[(long long)b * sm + (long long)i * s + i].x / sg;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *tbar = (float)red[0];
}

// M <- M + M^H (square, per batch), in place on the lower/upper pairs.
__global__ void k_herm_sum(int s, cf *M, long long sm) {
    const int b = blockIdx.y;
    cf *Mb = M + (long long)b * sm;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < s * s; idx += gridDim.x * blockDim.x) {
        const int i = idx / s, j = idx - i * s;
        if (j > i) continue;
        const cf a = Mb[(long long)i * s + j], c = Mb[(long long)j * s + i];
        const cf v = mk(a.x + c.x, a.y - c.y);
        Mb[(long long)i * s + j] = v;
        Mb[(long long)j * s + i] = cconj(v);
    }
}

cudaError_t launch_gamma(int batch, int s, const float *lam, float t, cf *M, long long sm, long long sl,
                         cudaStream_t st) {
    dim3 grid((s * s + 255) / 256, batch);
    k_gamma<<<grid, 256, 0, st>>>(s, lam, t, M, sm, sl);
    return cudaGetLastError();
}
cudaError_t launch_scale_vecs(int batch, int s, const float *lam, float t, const cf *V, cf *Vs, long long sv,
                              long long sl, int mode, cudaStream_t st) {
    dim3 grid((s * s + 255) / 256, batch);
    k_scale_vecs<<<grid, 256, 0, st>>>(s, lam, t, V, Vs, sv, sl, mode);
    return cudaGetLastError();
}
cudaError_t launch_tbar(int batch, int s, const float *lam, float t, const cf *Ct, long long sm, long long sl,
                        float *tbar, cudaStream_t st) {
    k_tbar<<<1, 256, 0, st>>>(batch, s, lam, t, Ct, sm, sl, tbar);
    return cudaGetLastError();
}
cudaError_t launch_herm_sum(int batch, int s, cf *M, long long sm, cudaStream_t st) {
    dim3 grid((s * s + 255) / 256, batch);
    k_herm_sum<<<grid, 256, 0, st>>>(s, M, sm);
    return cudaGetLastError();
}

// ---------------------------------------------------------- BLAS-1 helpers
// out = a x + b y (+ c z), complex64 arrays of n elements (y, z may be null).
__global__ void k_axpbypcz(long long n, float a, const cf *x, float b, const cf *y, float c, const cf *z, cf *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        cf v = cscale(x[i], a);
        if (y) v = cadd(v, cscale(y[i], b));
        if (z) v = cadd(v, cscale(z[i], c));
        out[i] = v;
    }
}
cudaError_t launch_axpbypcz(long long n, float a, const cf *x, float b, const cf *y, float c, const cf *z, cf *out,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = min((n + 255) / 256, (long long)152 * 8);
    k_axpbypcz<<<(unsigned)blocks, 256, 0, st>>>(n, a, x, b, y, c, z, out);
    return cudaGetLastError();
}

// *out = Re <x, y> = sum Re(conj(x_i) y_i), fixed-order two-level reduction.
__global__ void k_dot_partial(long long n, const cf *x, const cf *y, double *part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)x[i].x * y[i].x + (double)x[i].y * y[i].y;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_dot_final(int nb, const double *part, float *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < nb; ++i) a += part[i];
        *out = (float)a;
    }
}
#define DOT_BLOCKS 304
cudaError_t launch_dot_re(long long n, const cf *x, const cf *y, double *part, float *out, cudaStream_t st) {
    k_dot_partial<<<DOT_BLOCKS, 256, 0, st>>>(n, x, y, part);
    k_dot_final<<<1, 32, 0, st>>>(DOT_BLOCKS, part, out);
    return cudaGetLastError();
}

// X-update VJP: out[i] = beta Kbar[i] / den(i) where den = lambda U + beta (d_a + d_b)
// (hard consistency: out = Kbar / (d_a + d_b) on unsampled points, 0 on sampled ones);
// zero where den == 0.  ybar (nullable) receives lambda U Kbar / den.
__global__ void k_dc_vjp(DcArgs a, const cf *Kbar, cf *out, cf *ybar) {
    const long long total = (long long)a.L * a.J * a.M * a.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int kn = (int)(i % a.N);
        const long long r1 = i / a.N;
        const int m = (int)(r1 % a.M);
        const int l = (int)(r1 / ((long long)a.M * a.J));
        const float u = a.mask[((long long)l * a.M + m) * a.N + kn] ? 1.f : 0.f;
        const float dd = a.da[kn] + (a.model2d ? a.db[m] : a.db[l]);
        const cf kb = Kbar[i];
        cf o = mk(0.f, 0.f), yb = mk(0.f, 0.f);
        if (a.lambda > 0.f) {
            const float den = a.lambda * u + a.beta * dd;
            if (den != 0.f) {
                o = cscale(kb, a.beta / den);
                yb = cscale(kb, a.lambda * u / den);
            }
        } else if (u > 0.f) {
            yb = kb;
        } else if (dd != 0.f) {
            o = cscale(kb, 1.f / dd);
        }
        out[i] = o;
        if (ybar) ybar[i] = yb;
    }
}
cudaError_t launch_dc_vjp(const DcArgs &a, const cf *Kbar, cf *out, cf *ybar, cudaStream_t st) {
    const long long total = (long long)a.L * a.J * a.M * a.N;
    const long long blocks = min((total + 255) / 256, (long long)152 * 8);
    k_dc_vjp<<<(unsigned)blocks, 256, 0, st>>>(a, Kbar, out, ybar);
    return cudaGetLastError();
}

// ------------------------------------------------- Jacobi on [B; I] (VJP)
// aug[b][q] = [Bt[b][q][0..len); e_q] : column q of B followed by column q of
// the identity, so that one-sided Jacobi with rotations chosen on the first
// len entries leaves [B Q; Q] (Q unitary, B Q with orthogonal columns).
__global__ void k_augment(int s, int len, const cf *Bt, cf *aug) {
    const int b = blockIdx.y;
    const int L = len + s;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)s * L;
         idx += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(idx / L), e = (int)(idx - (long long)q * L);
        cf v;
        if (e < len) v = Bt[(long long)b * s * len + (long long)q * len + e];
        else v = mk(e - len == q ? 1.f : 0.f, 0.f);
        aug[(long long)b * s * L + idx] = v;
    }
}
cudaError_t launch_augment(int batch, int s, int len, const cf *Bt, cf *aug, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    const long long per = (long long)s * (len + s);
    dim3 grid((unsigned)min((per + 255) / 256, 64LL), batch);
    k_augment<<<grid, 256, 0, st>>>(s, len, Bt, aug);
    return cudaGetLastError();
}

// Vt[b][q][i] = Q[i][q] (eigenvector-major, row stride s, batch stride s*s) and
// lam[b][q] = ||(B Q)[:, q]||^2: the eigenpairs of G = B^H B.  One warp per q.
__global__ void k_split_aug(int s, int len, const cf *aug, cf *Vt, float *lam) {
    const int b = blockIdx.y;
    const int L = len + s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = blockIdx.x * nw + warp; q < s; q += gridDim.x * nw) {
        const cf *col = aug + (long long)b * s * L + (long long)q * L;
        float acc = 0.f;
        for (int e = lane; e < len; e += 32) acc = fmaf(col[e].x, col[e].x, fmaf(col[e].y, col[e].y, acc));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) lam[(long long)b * s + q] = acc;
        for (int i = lane; i < s; i += 32) Vt[(long long)b * s * s + (long long)q * s + i] = col[len + i];
    }
}
cudaError_t launch_split_aug(int batch, int s, int len, const cf *aug, cf *Vt, float *lam, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    dim3 grid((unsigned)((s + 7) / 8), batch);
    k_split_aug<<<grid, 256, 0, st>>>(s, len, aug, Vt, lam);
    return cudaGetLastError();
}

// M[b] <- M[b] + v I (square s x s, row stride s, batch stride sm).
__global__ void k_add_diag(int s, cf *M, long long sm, float v) {
    const int b = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x)
        M[(long long)b * sm + (long long)i * s + i].x += v;
}
cudaError_t launch_add_diag(int batch, int s, cf *M, long long sm, float v, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    dim3 grid((unsigned)((s + 255) / 256), batch);
    k_add_diag<<<grid, 256, 0, st>>>(s, M, sm, v);
    return cudaGetLastError();
}

// ------------------------------------------------------- low-rank reverse mode
// With r = #{lambda > t^2} pairs (v_q, lambda_q) of G = B^H B, sigma_q = sqrt(lambda_q),
// h_q = 1 - t / sigma_q, u_q = B v_q, g_q = Zbar v_q and C = B^H Zbar, the blocks of
// Gamma o (V^H C V) that involve eigenvectors below the threshold reduce to the
// resolvents R_q = sum_{lambda_j <= t^2} v_j v_j^H / (lambda_q - lambda_j):
//     y_q = R_q C^H v_q = R_q Zbar^H u_q,     z_q = R_q C v_q = R_q B^H g_q,
//     Gbar = V1 (Gamma11 o C11) V1^H + sum_q h_q (v_q y_q^H + z_q v_q^H),
//     C11_pq = u_p^H g_q,  Gamma11_pq = t / (s_p s_q (s_p + s_q)),
// so with M2 = Gamma11 o (C11 + C11^H) and x_q = h_q (y_q + z_q):
//     Bbar = Zbar h(G) + B (Gbar + Gbar^H)
//          = sum_q [h_q g_q + sum_p u_p M2_pq + B x_q] v_q^H + sum_q u_q x_q^H,
//     S_t(B) = sum_q h_q u_q v_q^H,   tbar = -Re sum_q C11_qq / sigma_q.
// Everything is O(r s len) besides the eigensolver and the 2 r resolvent solves
// (k_resolvent).  Per-matrix slots: vm-sized (s len) at g.off + mat s len for U, Gv
// (r x len), V, X (r x s), M2 (r x r), Ab (r x len); 2 s len for W, Y (2 r x s).
#define LR_QB 8
#define LR_THREADS 256

__device__ __forceinline__ float lr_wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(LR_THREADS) k_lr_front(GroupSet gs, const cf *Bt, const cf *Zt, const cf *V,
                                                         const int *rank, cf *U, cf *Gv, cf *W) {
    extern __shared__ __align__(16) cf lsm[];
    int mat;
    const int gi = find_group(gs, blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int n = g.s, len = g.len, r = rank[g.moff + mat];
    const long long base = g.off + (long long)mat * n * len;
    cf *vq = lsm, *us = lsm + LR_QB * n, *gq = us + LR_QB * len;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = LR_THREADS / 32;
    for (int q0 = 0; q0 < r; q0 += LR_QB) {
        const int qc = min(LR_QB, r - q0);
        for (int idx = tid; idx < LR_QB * n; idx += LR_THREADS) {
            const int qq = idx / n, i = idx - qq * n;
            vq[idx] = qq < qc ? V[base + (long long)(q0 + qq) * n + i] : mk(0.f, 0.f);
        }
        __syncthreads();
        for (int e = tid; e < len; e += LR_THREADS) {
            float ur[LR_QB], ui[LR_QB], gr[LR_QB], gi_[LR_QB];
#pragma unroll
            for (int qq = 0; qq < LR_QB; ++qq) ur[qq] = ui[qq] = gr[qq] = gi_[qq] = 0.f;
            for (int i = 0; i < n; ++i) {
                const cf b = Bt[base + (long long)i * len + e], z = Zt[base + (long long)i * len + e];
#pragma unroll
                for (int qq = 0; qq < LR_QB; ++qq) {
                    const cf v = vq[qq * n + i];
                    ur[qq] = fmaf(b.x, v.x, fmaf(-b.y, v.y, ur[qq]));
                    ui[qq] = fmaf(b.x, v.y, fmaf(b.y, v.x, ui[qq]));
                    gr[qq] = fmaf(z.x, v.x, fmaf(-z.y, v.y, gr[qq]));
                    gi_[qq] = fmaf(z.x, v.y, fmaf(z.y, v.x, gi_[qq]));
                }
            }
#pragma unroll
            for (int qq = 0; qq < LR_QB; ++qq) {
                us[qq * len + e] = mk(ur[qq], ui[qq]);
                gq[qq * len + e] = mk(gr[qq], gi_[qq]);
                if (qq < qc) {
                    U[base + (long long)(q0 + qq) * len + e] = mk(ur[qq], ui[qq]);
                    Gv[base + (long long)(q0 + qq) * len + e] = mk(gr[qq], gi_[qq]);
                }
            }
        }
        __syncthreads();
        // w1_q[i] = sum_e conj(Zbar[e][i]) u_q[e],  w2_q[i] = sum_e conj(B[e][i]) g_q[e]
        for (int i = warp; i < n; i += nw) {
            float a1r[LR_QB], a1i[LR_QB], a2r[LR_QB], a2i[LR_QB];
#pragma unroll
            for (int qq = 0; qq < LR_QB; ++qq) a1r[qq] = a1i[qq] = a2r[qq] = a2i[qq] = 0.f;
            for (int e = lane; e < len; e += 32) {
                const cf z = Zt[base + (long long)i * len + e], b = Bt[base + (long long)i * len + e];
#pragma unroll
                for (int qq = 0; qq < LR_QB; ++qq) {
                    const cf u = us[qq * len + e], gg = gq[qq * len + e];
                    a1r[qq] = fmaf(z.x, u.x, fmaf(z.y, u.y, a1r[qq]));
                    a1i[qq] = fmaf(z.x, u.y, fmaf(-z.y, u.x, a1i[qq]));
                    a2r[qq] = fmaf(b.x, gg.x, fmaf(b.y, gg.y, a2r[qq]));
                    a2i[qq] = fmaf(b.x, gg.y, fmaf(-b.y, gg.x, a2i[qq]));
                }
            }
#pragma unroll
            for (int qq = 0; qq < LR_QB; ++qq) {
                const float s1r = lr_wsum(a1r[qq]), s1i = lr_wsum(a1i[qq]);
                const float s2r = lr_wsum(a2r[qq]), s2i = lr_wsum(a2i[qq]);
                if (lane == 0 && qq < qc) {
                    W[2 * base + (long long)(2 * (q0 + qq)) * n + i] = mk(s1r, s1i);
                    W[2 * base + (long long)(2 * (q0 + qq) + 1) * n + i] = mk(s2r, s2i);
                }
            }
        }
        __syncthreads();
    }
}

// C11 = U^H Gv (r x r), M2 = Gamma11 o (C11 + C11^H), tpart[mat] = -Re sum_q C11_qq / sigma_q.
__global__ void __launch_bounds__(LR_THREADS) k_lr_mid(GroupSet gs, const cf *U, const cf *Gv, const float *lam,
                                                       const int *rank, float t, cf *C11, cf *M2, double *tpart) {
    int mat;
    const int gi = find_group(gs, blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int n = g.s, len = g.len, r = rank[g.moff + mat];
    const long long base = g.off + (long long)mat * n * len;
    const float *lm = lam + g.soff + (long long)mat * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = LR_THREADS / 32;
    for (int pq = warp; pq < r * r; pq += nw) {
        const int p = pq / r, q = pq - p * r;
        float cr = 0.f, ci = 0.f;
        for (int e = lane; e < len; e += 32) {
            const cf u = U[base + (long long)p * len + e], gg = Gv[base + (long long)q * len + e];
            cr = fmaf(u.x, gg.x, fmaf(u.y, gg.y, cr));
            ci = fmaf(u.x, gg.y, fmaf(-u.y, gg.x, ci));
        }
        cr = lr_wsum(cr);
        ci = lr_wsum(ci);
        if (lane == 0) C11[base + pq] = mk(cr, ci);
    }
    __syncthreads();
    for (int pq = tid; pq < r * r; pq += LR_THREADS) {
        const int p = pq / r, q = pq - p * r;
        const float sp = sqrtf(fmaxf(lm[p], 0.f)), sq = sqrtf(fmaxf(lm[q], 0.f));
        const float gam = t / (sp * sq * (sp + sq));
        const cf a = C11[base + pq], b = C11[base + (long long)q * r + p];
        M2[base + pq] = mk(gam * (a.x + b.x), gam * (a.y - b.y));
    }
    if (tid == 0) {
        double acc = 0.0;
        for (int q = 0; q < r; ++q) acc -= (double)C11[base + (long long)q * r + q].x / sqrt((double)fmaxf(lm[q], 0.f));
        tpart[g.moff + mat] = acc;
    }
}

// x_q = h_q (y_q + z_q);  a_q = h_q g_q + sum_p u_p M2_pq + B x_q.
__global__ void __launch_bounds__(LR_THREADS) k_lr_back(GroupSet gs, const cf *Bt, const cf *U, const cf *Gv,
                                                        const cf *M2, const cf *Yv, const float *lam, const int *rank,
                                                        float t, cf *X, cf *Ab) {
    extern __shared__ __align__(16) cf lsm[];
    int mat;
    const int gi = find_group(gs, blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int n = g.s, len = g.len, r = rank[g.moff + mat];
    const long long base = g.off + (long long)mat * n * len;
    const float *lm = lam + g.soff + (long long)mat * n;
    cf *xs = lsm;                       // LR_QB x n
    const int tid = threadIdx.x;
    for (int q0 = 0; q0 < r; q0 += LR_QB) {
        const int qc = min(LR_QB, r - q0);
        for (int idx = tid; idx < LR_QB * n; idx += LR_THREADS) {
            const int qq = idx / n, i = idx - qq * n;
            cf x = mk(0.f, 0.f);
            if (qq < qc) {
                const int q = q0 + qq;
                const float sg = sqrtf(fmaxf(lm[q], 0.f));
                const float h = sg > t ? 1.f - t / sg : 0.f;
                const cf y = Yv[2 * base + (long long)(2 * q) * n + i], z = Yv[2 * base + (long long)(2 * q + 1) * n + i];
                x = mk(h * (y.x + z.x), h * (y.y + z.y));
                X[base + (long long)q * n + i] = x;
            }
            xs[idx] = x;
        }
        __syncthreads();
        for (int e = tid; e < len; e += LR_THREADS) {
            float ar[LR_QB], ai[LR_QB];
#pragma unroll
            for (int qq = 0; qq < LR_QB; ++qq) ar[qq] = ai[qq] = 0.f;
            for (int i = 0; i < n; ++i) {
                const cf b = Bt[base + (long long)i * len + e];
#pragma unroll
                for (int qq = 0; qq < LR_QB; ++qq) {
                    const cf x = xs[qq * n + i];
                    ar[qq] = fmaf(b.x, x.x, fmaf(-b.y, x.y, ar[qq]));
                    ai[qq] = fmaf(b.x, x.y, fmaf(b.y, x.x, ai[qq]));
                }
            }
            for (int p = 0; p < r; ++p) {
                const cf u = U[base + (long long)p * len + e];
#pragma unroll
                for (int qq = 0; qq < LR_QB; ++qq) {
                    if (qq < qc) {
                        const cf m = M2[base + (long long)p * r + q0 + qq];
                        ar[qq] = fmaf(u.x, m.x, fmaf(-u.y, m.y, ar[qq]));
                        ai[qq] = fmaf(u.x, m.y, fmaf(u.y, m.x, ai[qq]));
                    }
                }
            }
#pragma unroll
            for (int qq = 0; qq < LR_QB; ++qq) {
                if (qq < qc) {
                    const int q = q0 + qq;
                    const float sg = sqrtf(fmaxf(lm[q], 0.f));
                    const float h = sg > t ? 1.f - t / sg : 0.f;
                    const cf gg = Gv[base + (long long)q * len + e];
                    Ab[base + (long long)q * len + e] = mk(ar[qq] + h * gg.x, ai[qq] + h * gg.y);
                }
            }
        }
        __syncthreads();
    }
}

// Bbar^T[v][e] = sum_q a_q[e] conj(v_q[v]) + u_q[e] conj(x_q[v]);
// Zt[v][e] (if non-null) = sum_q h_q u_q[e] conj(v_q[v]).  Block: 32 e x 8 v.
__global__ void __launch_bounds__(LR_THREADS) k_lr_out(GroupSet gs, const cf *U, const cf *Ab, const cf *V,
                                                       const cf *X, const float *lam, const int *rank, float t,
                                                       cf *Bbart, cf *Zt) {
    int mat;
    const int gi = find_group(gs, blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int n = g.s, len = g.len, r = rank[g.moff + mat];
    const long long base = g.off + (long long)mat * n * len;
    const float *lm = lam + g.soff + (long long)mat * n;
    const int e = blockIdx.y * 32 + (threadIdx.x & 31);
    const int v = blockIdx.z * 8 + (threadIdx.x >> 5);
    if (e >= len || v >= n) return;
    float br = 0.f, bi = 0.f, zr = 0.f, zi = 0.f;
    for (int q = 0; q < r; ++q) {
        const cf a = Ab[base + (long long)q * len + e], u = U[base + (long long)q * len + e];
        const cf vv = V[base + (long long)q * n + v], x = X[base + (long long)q * n + v];
        // a conj(vv) + u conj(x)
        br = fmaf(a.x, vv.x, fmaf(a.y, vv.y, br));
        bi = fmaf(a.y, vv.x, fmaf(-a.x, vv.y, bi));
        br = fmaf(u.x, x.x, fmaf(u.y, x.y, br));
        bi = fmaf(u.y, x.x, fmaf(-u.x, x.y, bi));
        if (Zt) {
            const float sg = sqrtf(fmaxf(lm[q], 0.f));
            const float h = sg > t ? 1.f - t / sg : 0.f;
            zr = fmaf(h, u.x * vv.x + u.y * vv.y, zr);
            zi = fmaf(h, u.y * vv.x - u.x * vv.y, zi);
        }
    }
    Bbart[base + (long long)v * len + e] = mk(br, bi);
    if (Zt) Zt[base + (long long)v * len + e] = mk(zr, zi);
}

// *out = sum of nm per-matrix partials in index order (single block).
__global__ void k_sum_partials(int nm, const double *part, float *out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nm; i += blockDim.x) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)red[0];
}

static bool g_lr_attr = false;

cudaError_t launch_lowrank_vjp(const GroupSet &gs, int nmat, const cf *Bt, const cf *Zt, const cf *V, const float *lam,
                               const int *rank, float t, const LrBuffers &b, float *tbar, cf *Bbart, cf *Zout_t,
                               const EigArgs &ea, cudaStream_t st) {
    if (nmat <= 0) return cudaSuccess;
    int nmax = 0, lmax = 0;
    for (int k = 0; k < gs.n; ++k) { nmax = max(nmax, gs.g[k].s); lmax = max(lmax, gs.g[k].len); }
    const size_t sm_front = sizeof(cf) * LR_QB * ((size_t)nmax + 2 * lmax);
    const size_t sm_back = sizeof(cf) * LR_QB * (size_t)nmax;
    cudaError_t e = cudaSuccess;
    if (!g_lr_attr) {
        e = cudaFuncSetAttribute(k_lr_front, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        g_lr_attr = true;
    }
    k_lr_front<<<nmat, LR_THREADS, sm_front, st>>>(gs, Bt, Zt, V, rank, b.U, b.Gv, b.W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_lr_mid<<<nmat, LR_THREADS, 0, st>>>(gs, b.U, b.Gv, lam, rank, t, b.C11, b.M2, b.tpart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_resolvent(gs, nmat, ea, b.W, b.Y, st)) != cudaSuccess) return e;
    k_lr_back<<<nmat, LR_THREADS, sm_back, st>>>(gs, Bt, b.U, b.Gv, b.M2, b.Y, lam, rank, t, b.X, b.Ab);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid(nmat, (lmax + 31) / 32, (nmax + 7) / 8);
    k_lr_out<<<grid, LR_THREADS, 0, st>>>(gs, b.U, b.Ab, V, b.X, lam, rank, t, Bbart, Zout_t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_sum_partials<<<1, 256, 0, st>>>(nmat, b.tpart, tbar);
    return cudaGetLastError();
}
