// Singular value thresholding through the Hermitian eigenproblem of the Gram
// matrix, computing only the eigenpairs above the threshold (Eqs. 16-17,
// S8-S9).
//
// For B (len x s, the shorter side as columns, vector-major storage):
//     G = B^H B = V diag(lambda) V^H,   sigma_i = sqrt(lambda_i),
//     S_t(B) = sum_{sigma_i > t} (1 - t / sigma_i) (B v_i) v_i^H,
// so only the eigenpairs with lambda_i > t^2 are needed.  On the lifted Hankel
// matrices of the reconstruction only a few percent of the s singular values
// exceed t, so the eigensolver is built to find exactly those:
//   k_gram      G (lower triangle, packed by columns) = B^H B.
//   k_heig      one CTA per matrix: Householder reduction of G to a Hermitian
//               tridiagonal (Householder vectors kept in the packed buffer),
//               diagonal phase scaling to a real symmetric tridiagonal T,
//               Sturm count of the eigenvalues above t^2, 32-way multisection
//               of each of them (one warp per eigenvalue), inverse iteration
//               for their eigenvectors with modified Gram-Schmidt inside
//               clusters of close eigenvalues, and back-transformation.
//   k_apply_eig Z = sum_i g_i (B v_i) v_i^H per tile of rows of B, fused with
//               the multiplier update D <- D + tau (A - D/beta - Z) and
//               E = Z - D/beta (Eqs. 13-14), or writing Z.
// No step is iterative beyond the fixed bisection / inverse-iteration counts,
// so the work is bounded by construction.
#include "selr_internal.cuh"

#include <float.h>

#define EIG_THREADS 512
#define EIG_WARPS (EIG_THREADS / 32)
#define EIG_SMEM_MAX_N 224       // packed G of order <= 224 stays in shared memory
#define EIG_MAXR_CHUNK 32        // eigenvectors handled per back-transformation pass
#define INV_ITERS 4

__device__ __forceinline__ long long colstart(int j, int n) { return (long long)j * (2 * n - j + 1) / 2; }

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one float (all threads get the result).
__device__ float bsum(float v, float *red) {
    v = wsum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float t = 0.f;
    if (l < EIG_WARPS) t = red[l];
    t = wsum(t);
    return t;
}

__device__ __forceinline__ bool is_frozen(const Group &g, int mat, const int *active) {
    if (!active) return false;
    if (g.kind == G_PE) return active[mat / g.L] == 0;
    if (g.kind == G_PARAM) return active[mat / g.N] == 0;
    return false;
}

// ------------------------------------------------------------------- Gram
// One CTA computes a 64x64 block (I >= J) of G = B^H B for one matrix.
#define GR_T 64
#define GR_K 16
__global__ void __launch_bounds__(256) k_gram(GroupSet gs, int mat_begin, const cf *B0, cf *Gp,
                                               const int *active) {
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    if (is_frozen(g, mat, active)) return;
    const int n = g.s, len = g.len;
    const int nb = (n + GR_T - 1) / GR_T;
    // blockIdx.y enumerates lower blocks (bi >= bj)
    int bi = 0, bj = 0, q = blockIdx.y;
    if (q >= nb * (nb + 1) / 2) return;
    while (q > bi) { q -= bi + 1; ++bi; }
    bj = q;
    const cf *B = B0 + g.off + (long long)mat * n * len;
    __shared__ cf sI[GR_K][GR_T + 1], sJ[GR_K][GR_T + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4x4 outputs each
    float accr[4][4], acci[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) accr[a][b] = acci[a][b] = 0.f;
    const int i0 = bi * GR_T, j0 = bj * GR_T;
    for (int e0 = 0; e0 < len; e0 += GR_K) {
        for (int idx = threadIdx.x; idx < GR_K * GR_T; idx += 256) {
            const int v = idx / GR_K, e = idx - v * GR_K;   // e fastest -> coalesced along the vector
            const int ee = e0 + e;
            cf xi = mk(0.f, 0.f), xj = mk(0.f, 0.f);
            if (ee < len) {
                if (i0 + v < n) xi = B[(long long)(i0 + v) * len + ee];
                if (j0 + v < n) xj = B[(long long)(j0 + v) * len + ee];
            }
            sI[e][v] = xi;
            sJ[e][v] = xj;
        }
        __syncthreads();
#pragma unroll 4
        for (int e = 0; e < GR_K; ++e) {
            cf a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = sI[e][ty + 16 * u]; b[u] = sJ[e][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    // conj(a) * b
                    accr[u][w] = fmaf(a[u].x, b[w].x, fmaf(a[u].y, b[w].y, accr[u][w]));
                    acci[u][w] = fmaf(a[u].x, b[w].y, fmaf(-a[u].y, b[w].x, acci[u][w]));
                }
        }
        __syncthreads();
    }
    cf *G = Gp + g.poff + (long long)mat * ((long long)n * (n + 1) / 2);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * w;
            if (i < n && j < n && i >= j) G[colstart(j, n) + (i - j)] = mk(accr[u][w], acci[u][w]);
        }
}

// ------------------------------------------------------- tridiagonal tools
// Number of eigenvalues of the real symmetric tridiagonal (d, f) below x.
__device__ __forceinline__ int sturm_lt(const float *d, const float *f2, int n, float x, float pivmin) {
    int cnt = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++cnt;
    for (int k = 1; k < n; ++k) {
        q = (d[k] - x) - f2[k - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        if (q < 0.f) ++cnt;
    }
    return cnt;
}

// Solve (T - lam I) y = z in place (z -> y) by Gaussian elimination with
// partial pivoting on the tridiagonal (d, f).  u0/u1/u2 are the diagonals of
// U, lm the multipliers, piv the row interchanges; all length n.  The
// current row always has two entries (c0 at column k, c1 at column k+1):
//   no swap: l = f_k / c0, U_k = (c0, c1, 0),          row' = (a_{k+1} - l c1, f_{k+1})
//   swap:    l = c0 / f_k, U_k = (f_k, a_{k+1}, f_{k+1}), row' = (c1 - l a_{k+1}, -l f_{k+1})
// A zero pivot is replaced by `tiny` (inverse iteration wants a huge, not
// infinite, growth).
__device__ void tri_solve(const float *d, const float *f, int n, float lam, float *z, float *u0, float *u1,
                          float *u2, float *lm, unsigned char *piv, float tiny) {
    float c0 = d[0] - lam, c1 = n > 1 ? f[0] : 0.f;
    for (int k = 0; k < n - 1; ++k) {
        const float fk = f[k];
        const float an = d[k + 1] - lam;
        const float fn = k + 1 < n - 1 ? f[k + 1] : 0.f;
        if (fabsf(c0) >= fabsf(fk)) {
            if (c0 == 0.f) c0 = tiny;
            const float l = fk / c0;
            u0[k] = c0; u1[k] = c1; u2[k] = 0.f; lm[k] = l; piv[k] = 0;
            c0 = an - l * c1;
            c1 = fn;
        } else {
            const float l = c0 / fk;
            u0[k] = fk; u1[k] = an; u2[k] = fn; lm[k] = l; piv[k] = 1;
            c0 = c1 - l * an;
            c1 = -l * fn;
        }
    }
    if (c0 == 0.f) c0 = tiny;
    u0[n - 1] = c0; u1[n - 1] = 0.f; u2[n - 1] = 0.f;
    for (int k = 0; k < n - 1; ++k) {
        if (piv[k]) {
            const float t = z[k];
            z[k] = z[k + 1];
            z[k + 1] = t - lm[k] * z[k + 1];
        } else {
            z[k + 1] -= lm[k] * z[k];
        }
    }
    z[n - 1] /= u0[n - 1];
    if (n > 1) z[n - 2] = (z[n - 2] - u1[n - 2] * z[n - 1]) / u0[n - 2];
    for (int k = n - 3; k >= 0; --k) z[k] = (z[k] - u1[k] * z[k + 1] - u2[k] * z[k + 2]) / u0[k];
}

// ------------------------------------------------------------------ k_heig
__global__ void __launch_bounds__(EIG_THREADS, 1) k_heig(GroupSet gs, int mat_begin, EigArgs a) {
    extern __shared__ float esm[];
    __shared__ float red[EIG_WARPS];
    __shared__ float s_tau;
    __shared__ cf s_alpha;
    __shared__ int s_r;
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    if (is_frozen(g, mat, a.active)) return;
    const int n = g.s;
    const long long pk = (long long)n * (n + 1) / 2;
    cf *Gglob = a.Gp + g.poff + (long long)mat * pk;
    const bool in_smem = n <= EIG_SMEM_MAX_N;
    // shared layout: [v n][p n][ph n] cf, [d n][f n][f^2 n][tau n] float, then the packed
    // G (if it fits); the eigen stage reuses the packed region as scratch.
    cf *vb = (cf *)esm;
    cf *pb = vb + n;
    cf *ph = pb + n;
    float *dd = (float *)(ph + n);
    float *ff = dd + n;
    float *f2 = ff + n;
    float *taus = f2 + n;
    float *work = taus + n;
    cf *Gs = in_smem ? (cf *)work : Gglob;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float t2 = g.thresh * g.thresh;
    float *lam_out = a.lam + g.soff + (long long)mat * n;
    cf *V = a.V + g.off + (long long)mat * n * g.len;   // room for s vectors of length s <= len
    int *rank_out = a.rank + g.moff + mat;

    if (in_smem)
        for (long long i = tid; i < pk; i += EIG_THREADS) Gs[i] = Gglob[i];
    __syncthreads();

    // ---- Householder reduction to Hermitian tridiagonal (lower)
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        cf *col = Gs + colstart(k, n) + 1;     // x = G[k+1 .. n-1][k]
        float xn2 = 0.f;
        for (int i = tid; i < m; i += EIG_THREADS) xn2 += cabs2(col[i]);
        xn2 = bsum(xn2, red);
        const cf x0 = col[0];
        const float ax0 = sqrtf(cabs2(x0));
        const float rest = xn2 - ax0 * ax0;
        if (tid == 0) {
            if (!(rest > 1e-30f * xn2) || xn2 == 0.f) {
                s_tau = 0.f;
                s_alpha = x0;
            } else {
                const float xnorm = sqrtf(xn2);
                const cf phs = ax0 > 0.f ? mk(x0.x / ax0, x0.y / ax0) : mk(1.f, 0.f);
                s_alpha = mk(-phs.x * xnorm, -phs.y * xnorm);
                s_tau = 1.f / (xn2 + xnorm * ax0);          // 2 / v^H v
                vb[0] = mk(phs.x * (ax0 + xnorm), phs.y * (ax0 + xnorm));
            }
        }
        __syncthreads();
        const float tau = s_tau;
        if (tid == 0) taus[k] = tau;
        cf *hv = Gglob + colstart(k, n) + 1;   // Householder vector k stored in place of column k
        if (tau == 0.f) {
            if (tid == 0) { vb[0] = mk(0.f, 0.f); ph[k] = s_alpha; }
            __syncthreads();
            continue;
        }
        for (int i = tid + 1; i < m; i += EIG_THREADS) vb[i] = col[i];
        __syncthreads();
        for (int i = tid; i < m; i += EIG_THREADS) hv[i] = vb[i];
        if (tid == 0) ph[k] = s_alpha;        // sub-diagonal entry e_k (temporarily in ph)
        // p = tau * Gt v over trailing rows/cols k+1 .. n-1 (trailing index i <-> row k+1+i)
        for (int i = tid; i < m; i += EIG_THREADS) {
            const int I = k + 1 + i;
            float sr = 0.f, si = 0.f;
            for (int j = 0; j <= i; ++j) {          // G(I, J) stored, J = k+1+j <= I
                const cf gv = Gs[colstart(k + 1 + j, n) + (I - (k + 1 + j))];
                const cf v = vb[j];
                sr += gv.x * v.x - gv.y * v.y;
                si += gv.x * v.y + gv.y * v.x;
            }
            const cf *ci = Gs + colstart(I, n);
            for (int j = i + 1; j < m; ++j) {       // conj(G(J, I)), J > I
                const cf gv = ci[j - i];
                const cf v = vb[j];
                sr += gv.x * v.x + gv.y * v.y;
                si += gv.x * v.y - gv.y * v.x;
            }
            pb[i] = mk(tau * sr, tau * si);
        }
        __syncthreads();
        float kv = 0.f;
        for (int i = tid; i < m; i += EIG_THREADS) kv += vb[i].x * pb[i].x + vb[i].y * pb[i].y;   // Re(v^H p)
        kv = bsum(kv, red);
        const float K = 0.5f * tau * kv;
        for (int i = tid; i < m; i += EIG_THREADS) pb[i] = mk(pb[i].x - K * vb[i].x, pb[i].y - K * vb[i].y);  // w
        __syncthreads();
        // rank-2 update of the trailing lower triangle: G(I,J) -= v_i conj(w_j) + w_i conj(v_j)
        for (int j = warp; j < m; j += EIG_WARPS) {
            const cf vj = vb[j], wj = pb[j];
            cf *cj = Gs + colstart(k + 1 + j, n);
            for (int i = j + lane; i < m; i += 32) {
                const cf vi = vb[i], wi = pb[i];
                cf gv = cj[i - j];
                gv.x -= vi.x * wj.x + vi.y * wj.y + wi.x * vj.x + wi.y * vj.y;
                gv.y -= vi.y * wj.x - vi.x * wj.y + wi.y * vj.x - wi.x * vj.y;
                cj[i - j] = gv;
            }
        }
        __syncthreads();
    }
    // diagonal, last sub-diagonal
    for (int k = tid; k < n; k += EIG_THREADS) dd[k] = Gs[colstart(k, n)].x;
    if (tid == 0) {
        if (n >= 2) ph[n - 2] = Gs[colstart(n - 2, n) + 1];
        if (n >= 2) taus[n - 2] = 0.f;
        taus[n - 1] = 0.f;
    }
    __syncthreads();
    // phases making the tridiagonal real: f_k = |e_k|, ph_{k+1} = ph_k e_k / |e_k|
    if (tid == 0) {
        cf cur = mk(1.f, 0.f);
        for (int k = 0; k < n; ++k) {
            const cf e = k + 1 < n ? ph[k] : mk(0.f, 0.f);
            const float ae = sqrtf(cabs2(e));
            ph[k] = cur;
            if (k + 1 < n) {
                ff[k] = ae;
                f2[k] = ae * ae;
                if (ae > 0.f) cur = cmul(cur, mk(e.x / ae, e.y / ae));
            }
        }
        if (n >= 1) { ff[n - 1] = 0.f; f2[n - 1] = 0.f; }
    }
    __syncthreads();

    // ---- eigenvalues above t^2
    float gl = 0.f, gu = 0.f, fmax2 = 0.f;
    if (tid == 0) {
        gl = FLT_MAX; gu = -FLT_MAX;
        for (int k = 0; k < n; ++k) {
            const float r0 = (k > 0 ? ff[k - 1] : 0.f) + (k + 1 < n ? ff[k] : 0.f);
            gl = fminf(gl, dd[k] - r0);
            gu = fmaxf(gu, dd[k] + r0);
            fmax2 = fmaxf(fmax2, f2[k]);
        }
        red[0] = gl; red[1] = gu; red[2] = fmax2;
    }
    __syncthreads();
    gl = red[0]; gu = red[1]; fmax2 = red[2];
    const float tnorm = fmaxf(fabsf(gl), fabsf(gu));
    const float pivmin = FLT_MIN * fmaxf(1.f, fmax2);
    if (tid == 0) {
        const int below = (t2 >= gu) ? n : sturm_lt(dd, f2, n, t2, pivmin);
        s_r = n - below;
    }
    __syncthreads();
    const int r = s_r;
    if (tid == 0) *rank_out = r;
    if (r == 0) return;
    // reuse shared memory beyond the tridiagonal arrays for the eigen stage
    float *lamv = work;                               // [r]
    int *clu = (int *)(lamv + n);                     // cluster start flags [r]
    float *zv = (float *)(clu + n);                   // [min(r, chunk)][n] real eigenvectors of T
    // multisection: warp per eigenvalue (q-th largest, ascending index n-1-q)
    for (int q = warp; q < r; q += EIG_WARPS) {
        const int j = n - 1 - q;
        float lo = fmaxf(gl, t2), hi = gu;
        hi = hi + 2.f * FLT_EPSILON * fabsf(hi) + pivmin;
        for (int it = 0; it < 12; ++it) {
            const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
            const int c = sturm_lt(dd, f2, n, x, pivmin);
            const unsigned msk = __ballot_sync(0xffffffffu, c <= j);
            const int nb = __popc(msk);
            const float nlo = nb > 0 ? lo + (hi - lo) * (float)nb / 33.f : lo;
            const float nhi = nb < 32 ? lo + (hi - lo) * (float)(nb + 1) / 33.f : hi;
            lo = nlo;
            hi = nhi;
            if (hi - lo <= 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + pivmin) break;
        }
        if (lane == 0) lamv[q] = 0.5f * (lo + hi);
    }
    __syncthreads();
    // clusters of close eigenvalues (descending order) and distinctness perturbation
    if (tid == 0) {
        const float ortol = 1e-3f * tnorm;
        const float sep = 10.f * FLT_EPSILON * tnorm;
        for (int q = 0; q < r; ++q) {
            if (q > 0 && lamv[q - 1] - lamv[q] < sep) lamv[q] = lamv[q - 1] - sep;
            clu[q] = (q == 0) || (lamv[q - 1] - lamv[q] > ortol) ? 1 : 0;
        }
    }
    __syncthreads();
    for (int q = tid; q < r; q += EIG_THREADS) lam_out[q] = lamv[q];
    // eigenvectors in chunks of EIG_MAXR_CHUNK: inverse iteration + MGS within clusters,
    // then back-transformation v = Q P z.
    float *scratch = zv + (long long)EIG_MAXR_CHUNK * n;   // per warp: 4n floats + n bytes
    for (int q0 = 0; q0 < r; q0 += EIG_MAXR_CHUNK) {
        const int qc = min(EIG_MAXR_CHUNK, r - q0);
        // a warp owns a cluster (its members in this chunk, in order); cluster starts are
        // re-opened at the chunk boundary (members of a split cluster are orthogonalised
        // against earlier members of the same chunk only).
        for (int w = warp; w < qc; w += EIG_WARPS) {
            const int q = q0 + w;
            const bool starts = (w == 0) || clu[q];
            if (!starts) continue;
            int end = w + 1;
            while (end < qc && !clu[q0 + end]) ++end;
            float *u0 = scratch + (long long)warp * (4 * n + n / 4 + 1);
            float *u1 = u0 + n, *u2 = u1 + n, *lm = u2 + n;
            unsigned char *piv = (unsigned char *)(lm + n);
            for (int mbr = w; mbr < end; ++mbr) {
                float *z = zv + (long long)mbr * n;
                const float lm_ = lamv[q0 + mbr];
                for (int i = lane; i < n; i += 32)
                    z[i] = 1.f + 0.25f * (float)(((i * 7919 + (q0 + mbr) * 104729) % 997) - 498) / 498.f;
                __syncwarp();
                for (int it = 0; it < INV_ITERS; ++it) {
                    if (lane == 0) tri_solve(dd, ff, n, lm_, z, u0, u1, u2, lm, piv, FLT_EPSILON * tnorm + pivmin);
                    __syncwarp();
                    // orthogonalise against earlier members of the cluster
                    for (int o = w; o < mbr; ++o) {
                        const float *zo = zv + (long long)o * n;
                        float dot = 0.f;
                        for (int i = lane; i < n; i += 32) dot += zo[i] * z[i];
                        dot = wsum(dot);
                        for (int i = lane; i < n; i += 32) z[i] -= dot * zo[i];
                        __syncwarp();
                    }
                    float nrm = 0.f;
                    for (int i = lane; i < n; i += 32) nrm += z[i] * z[i];
                    nrm = wsum(nrm);
                    const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
                    for (int i = lane; i < n; i += 32) z[i] *= inv;
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        // back-transformation: y = P z (complex), then y <- H_k y for k = n-3 .. 0.
        cf *Yc = (cf *)scratch;                                    // [qc][n]
        for (long long idx = tid; idx < (long long)qc * n; idx += EIG_THREADS) {
            const int w = (int)(idx / n), i = (int)(idx - (long long)w * n);
            Yc[idx] = cscale(ph[i], zv[(long long)w * n + i]);
        }
        __syncthreads();
        for (int k = n - 3; k >= 0; --k) {
            const float tau = taus[k];
            if (tau == 0.f) continue;
            const int m = n - k - 1;
            const cf *hv = Gglob + colstart(k, n) + 1;
            for (int i = tid; i < m; i += EIG_THREADS) vb[i] = hv[i];
            __syncthreads();
            for (int w = warp; w < qc; w += EIG_WARPS) {
                cf *y = Yc + (long long)w * n + k + 1;
                float sr = 0.f, si = 0.f;
                for (int i = lane; i < m; i += 32) {          // v^H y
                    const cf v = vb[i], yy = y[i];
                    sr += v.x * yy.x + v.y * yy.y;
                    si += v.x * yy.y - v.y * yy.x;
                }
                sr = wsum(sr) * tau;
                si = wsum(si) * tau;
                for (int i = lane; i < m; i += 32) {
                    const cf v = vb[i];
                    y[i].x -= v.x * sr - v.y * si;
                    y[i].y -= v.x * si + v.y * sr;
                }
            }
            __syncthreads();
        }
        for (long long idx = tid; idx < (long long)qc * n; idx += EIG_THREADS) {
            const int w = (int)(idx / n), i = (int)(idx - (long long)w * n);
            const cf y = Yc[idx];
            if (!isfinite(y.x) || !isfinite(y.y)) atomicOr(a.status, (unsigned)ST_NONFINITE);
            V[(long long)(q0 + w) * n + i] = y;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- apply
#define AP_ET 16
#define AP_CH 16
#define AP_THREADS 256
__global__ void __launch_bounds__(AP_THREADS) k_apply_eig(GroupSet gs, int mat_begin, EigArgs ea, SvtArgs a) {
    extern __shared__ cf xsm[];
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    if (is_frozen(g, mat, a.active)) return;
    const int n = g.s, len = g.len;
    const int e0 = blockIdx.y * AP_ET;
    if (e0 >= len) return;
    const int et = min(AP_ET, len - e0);
    const long long mb = g.off + (long long)mat * n * len;
    const int r = ea.rank[g.moff + mat];
    const float t = g.thresh;
    cf *Bt = xsm;                          // [n][AP_ET]
    cf *Vc = Bt + (long long)n * AP_ET;    // [AP_CH][n]
    cf *Yc = Vc + (long long)AP_CH * n;    // [AP_ET][AP_CH]
    __shared__ float gcoef[AP_CH];
    for (int idx = threadIdx.x; idx < n * AP_ET; idx += AP_THREADS) {
        const int c = idx / AP_ET, e = idx - c * AP_ET;
        Bt[idx] = e < et ? a.B0[mb + (long long)c * len + e0 + e] : mk(0.f, 0.f);
    }
    if (blockIdx.y == 0 && threadIdx.x == 0 && a.rank_out) a.rank_out[g.moff + mat] = r;
    __syncthreads();
    constexpr int MAXE = (512 * AP_ET + AP_THREADS - 1) / AP_THREADS;    // n <= 512
    const int nel = n * AP_ET;
    cf z[MAXE];
#pragma unroll
    for (int k = 0; k < MAXE; ++k) z[k] = mk(0.f, 0.f);
    const cf *V = ea.V + g.off + (long long)mat * n * len;
    const float *lam = ea.lam + g.soff + (long long)mat * n;
    for (int i0 = 0; i0 < r; i0 += AP_CH) {
        const int ch = min(AP_CH, r - i0);
        for (int idx = threadIdx.x; idx < ch * n; idx += AP_THREADS) Vc[idx] = V[(long long)i0 * n + idx];
        if (threadIdx.x < ch) {
            const float sg = sqrtf(fmaxf(lam[i0 + threadIdx.x], 0.f));
            gcoef[threadIdx.x] = sg > t ? 1.f - t / sg : 0.f;
        }
        __syncthreads();
        // Y[e][k] = g_k * sum_c B[e][c] V_k[c]
        for (int idx = threadIdx.x; idx < AP_ET * AP_CH; idx += AP_THREADS) {
            const int k = idx / AP_ET, e = idx - k * AP_ET;
            float yr = 0.f, yi = 0.f;
            if (k < ch) {
                const cf *vk = Vc + (long long)k * n;
                for (int c = 0; c < n; ++c) {
                    const cf b = Bt[c * AP_ET + e], v = vk[c];
                    yr = fmaf(b.x, v.x, fmaf(-b.y, v.y, yr));
                    yi = fmaf(b.x, v.y, fmaf(b.y, v.x, yi));
                }
                yr *= gcoef[k];
                yi *= gcoef[k];
            }
            Yc[e * AP_CH + k] = mk(yr, yi);
        }
        __syncthreads();
        // Z[c][e] += sum_k Y[e][k] conj(V_k[c])
#pragma unroll
        for (int kk = 0; kk < MAXE; ++kk) {
            const int idx = threadIdx.x + kk * AP_THREADS;
            if (idx < nel) {
                const int c = idx / AP_ET, e = idx - c * AP_ET;
                cf acc = z[kk];
                for (int k = 0; k < ch; ++k) {
                    const cf y = Yc[e * AP_CH + k], v = Vc[(long long)k * n + c];
                    acc.x = fmaf(y.x, v.x, fmaf(y.y, v.y, acc.x));
                    acc.y = fmaf(y.y, v.x, fmaf(-y.x, v.y, acc.y));
                }
                z[kk] = acc;
            }
        }
        __syncthreads();
    }
    const float ib = 1.f / a.beta;
#pragma unroll
    for (int kk = 0; kk < MAXE; ++kk) {
        const int idx = threadIdx.x + kk * AP_THREADS;
        if (idx < nel) {
            const int c = idx / AP_ET, e = idx - c * AP_ET;
            if (e >= et) continue;
            const long long vi = mb + (long long)c * len + e0 + e;
            if (a.mode == 0) {
                if (a.z_natural) {
                    int rr, cc;
                    if (g.trans) { rr = c; cc = e0 + e; } else { rr = e0 + e; cc = c; }
                    a.Zout[g.off + (long long)mat * n * len + (long long)rr * g.cols + cc] = z[kk];
                } else {
                    a.Zout[vi] = z[kk];
                }
            } else {
                const cf A = Bt[idx];
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

// ---------------------------------------------------------------- launchers
static int g_eig_smem_max = 0;

cudaError_t eig_init_attributes() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    g_eig_smem_max = optin - 2048;
    e = cudaFuncSetAttribute(k_heig, cudaFuncAttributeMaxDynamicSharedMemorySize, g_eig_smem_max);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_apply_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, g_eig_smem_max);
}

// shared bytes needed by k_heig for order n
static size_t heig_smem(int n) {
    const size_t pk = (size_t)n * (n + 1) / 2;
    const bool in_smem = n <= EIG_SMEM_MAX_N;
    size_t b = 3 * (size_t)n * sizeof(cf) + 4 * (size_t)n * sizeof(float);
    const size_t gbytes = (in_smem ? pk : 0) * sizeof(cf);
    // eigen stage: lam [n] + clu [n] + z [chunk][n] + per-warp (4n + n/4 + 1) floats, or Y [chunk][n] cf
    const size_t per_warp = (4 * (size_t)n + n / 4 + 1) * sizeof(float);
    const size_t st1 = 2 * (size_t)n * 4 + (size_t)EIG_MAXR_CHUNK * n * sizeof(float) +
                       (size_t)EIG_WARPS * per_warp;
    const size_t st2 = 2 * (size_t)n * 4 + (size_t)EIG_MAXR_CHUNK * n * sizeof(float) +
                       (size_t)EIG_MAXR_CHUNK * n * sizeof(cf);
    const size_t st = st1 > st2 ? st1 : st2;
    return b + (gbytes > st ? gbytes : st);
}

cudaError_t launch_gram(const GroupSet &gs, int mat_begin, int mat_count, const cf *B0, cf *Gp,
                        const int *active, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    int maxnb = 0;
    for (int k = 0; k < gs.n; ++k) {
        const int nb = (gs.g[k].s + GR_T - 1) / GR_T;
        maxnb = max(maxnb, nb * (nb + 1) / 2);
    }
    dim3 grid(mat_count, maxnb);
    k_gram<<<grid, 256, 0, st>>>(gs, mat_begin, B0, Gp, active);
    return cudaGetLastError();
}

cudaError_t launch_heig(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    if (g_eig_smem_max == 0) return cudaErrorNotReady;
    size_t smem = 0;
    for (int k = 0; k < gs.n; ++k) smem = max(smem, heig_smem(gs.g[k].s));
    if (smem > (size_t)g_eig_smem_max) return cudaErrorInvalidValue;
    k_heig<<<mat_count, EIG_THREADS, smem, st>>>(gs, mat_begin, ea);
    return cudaGetLastError();
}

cudaError_t launch_apply_eig(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, const SvtArgs &a,
                             cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    if (g_eig_smem_max == 0) return cudaErrorNotReady;
    int maxlen = 0, maxn = 0;
    for (int k = 0; k < gs.n; ++k) { maxlen = max(maxlen, gs.g[k].len); maxn = max(maxn, gs.g[k].s); }
    if (maxn > 512) return cudaErrorInvalidValue;
    const size_t smem = sizeof(cf) * ((size_t)maxn * AP_ET + (size_t)AP_CH * maxn + AP_ET * AP_CH);
    dim3 grid(mat_count, (maxlen + AP_ET - 1) / AP_ET);
    k_apply_eig<<<grid, AP_THREADS, smem, st>>>(gs, mat_begin, ea, a);
    return cudaGetLastError();
}
