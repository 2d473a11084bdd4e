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
//   k_tridiag   one CTA per matrix: Householder reduction of G to a Hermitian
//               tridiagonal (Householder vectors kept in the packed buffer),
//               with the rank-2 update of each step fused into the next
//               step's matrix-vector product (one pass over the matrix per
//               step); k_tridiag_g is the same reduction on global memory for
//               orders that do not fit in shared memory.
//   k_sb1, k_sb2  the two-stage alternative to k_tridiag (orders 48 .. 192, opt-in): G to a
//               Hermitian band of half-bandwidth 16 by blocked panels, then the band to
//               tridiagonal by bulge chasing (see the section before k_eigvec).
//   k_eigvec    diagonal phase scaling to a real symmetric tridiagonal T,
//               Sturm count of the eigenvalues above t^2, 32-way multisection
//               of each of them (one warp per eigenvalue), inverse iteration
//               for their eigenvectors (one thread per vector) with modified
//               Gram-Schmidt inside clusters of close eigenvalues, and
//               back-transformation with batches of reflectors.
//               EigArgs::zsave keeps the tridiagonal-basis eigenvectors.  With
//               EigArgs::allp every eigenpair is computed: clusters of close
//               eigenvalues then span several chunks of vectors, so each
//               inverse-iteration pass also orthogonalises (twice, modified
//               Gram-Schmidt) against the members of the same cluster found in
//               earlier chunks, read back from zsave.
//   k_resolvent the resolvent solves of the reverse-mode derivative (see
//               launch_resolvent in selr_internal.cuh): P^H Q^H, projection off
//               the computed eigenvectors, a tridiagonal solve per right-hand
//               side, projection, Q P.
//   k_apply_eig Z = sum_i g_i (B v_i) v_i^H per tile of rows of B, fused with
//               the multiplier update D <- D + tau (A - D/beta - Z) and
//               E = Z - D/beta (Eqs. 13-14), or writing Z.
// No step is iterative beyond the fixed bisection / inverse-iteration counts,
// so the work is bounded by construction.
#include "selr_internal.cuh"

#include <float.h>
#include <type_traits>

#define EIG_THREADS 512
#define EIG_WARPS (EIG_THREADS / 32)
#define EIG_SMEM_MAX_N 208       // packed G of order <= 208 stays in shared memory
#define INV_ITERS 4
#define EV_HB 8                  // Householder reflectors staged per back-transformation batch
#define TB 4                     // trailing columns per pass of the tridiagonal sweep (8 sums per reduction)

__device__ __forceinline__ long long colstart(int j, int n) { return (long long)j * (2 * n - j + 1) / 2; }

__host__ __device__ inline size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide maximum of one non-negative float (all threads get the result).
__device__ float bmax(float v, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float t = 0.f;
    if (l < EIG_WARPS) t = red[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}

// Squared norm below which a Householder column counts as already reduced:
// (eps max_i G_ii)^2 (G is positive semidefinite, so |G_ij| <= max_i G_ii), and
// never below 1e-36 so that tau = 1 / (|x|^2 + |x| |x_0|) stays finite.  Rank-
// deficient Gram matrices leave trailing columns of ~1e-20 whose squared norms
// are denormal; dropping them perturbs T by less than eps ||G||.
__device__ __forceinline__ float reflector_floor(float gmax) {
    const float f = FLT_EPSILON * gmax;
    return fmaxf(f * f, 1e-36f);
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
    if (g.kind == G_PE) return active[g.aoff + mat / g.L] == 0;
    if (g.kind == G_PARAM) return active[g.aoff + mat / g.N] == 0;
    return false;
}

// 8-byte asynchronous global -> shared copy (src_bytes 0: the destination is zero-filled and
// nothing is read).
__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Transpose-reduce over the lanes: lane L ends with the lane total of value (L >> 1) & 15 of
// a[16] (four halving exchanges, then one plain one: 16 shuffles for 16 sums).
__device__ __forceinline__ float treduce16(const float (&a)[16], int lane) {
    float b8[8], b4[4], b2[2];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool hi = lane & 16;
        b8[q] = (hi ? a[q + 8] : a[q]) + __shfl_xor_sync(0xffffffffu, hi ? a[q] : a[q + 8], 16);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool hi = lane & 8;
        b4[q] = (hi ? b8[q + 4] : b8[q]) + __shfl_xor_sync(0xffffffffu, hi ? b8[q] : b8[q + 4], 8);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const bool hi = lane & 4;
        b2[q] = (hi ? b4[q + 2] : b4[q]) + __shfl_xor_sync(0xffffffffu, hi ? b4[q] : b4[q + 2], 4);
    }
    const bool hi = lane & 2;
    const float s = (hi ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, hi ? b2[0] : b2[1], 2);
    return s + __shfl_xor_sync(0xffffffffu, s, 1);
}

// Lane L ends with the lane total of value (L >> 3) & 3 of a[4].
__device__ __forceinline__ float treduce4(const float (&a)[4], int lane) {
    const bool h16 = lane & 16, h8 = lane & 8;
    const float b0 = (h16 ? a[2] : a[0]) + __shfl_xor_sync(0xffffffffu, h16 ? a[0] : a[2], 16);
    const float b1 = (h16 ? a[3] : a[1]) + __shfl_xor_sync(0xffffffffu, h16 ? a[1] : a[3], 16);
    float s = (h8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h8 ? b0 : b1, 8);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    return s + __shfl_xor_sync(0xffffffffu, s, 1);
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
// Number of eigenvalues of the real symmetric tridiagonal (d, f) below x.  The
// recurrence divides once per step along a chain of n dependent steps, so it uses
// the fast division (2 ulp): a count can only change where |q| is within rounding
// of the pivot floor, which moves the bisection point by O(eps |T|), well inside
// the bisection's own stopping width.
__device__ __forceinline__ int sturm_lt(const float *d, const float *f2, int n, float x, float pivmin) {
    int cnt = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++cnt;
#pragma unroll 4
    for (int k = 1; k < n; ++k) {
        q = (d[k] - x) - __fdividef(f2[k - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        if (q < 0.f) ++cnt;
    }
    return cnt;
}

// Solve (T - lam I) y = z in place (z -> y) by Gaussian elimination with
// partial pivoting on the tridiagonal (d, f).  u0/u1/u2 are the diagonals of
// U, lm the multipliers, piv the row interchanges; element k of each array is
// at index k * ST (arrays of several systems are interleaved so that the
// threads solving them touch distinct shared-memory banks).  The current row
// always has two entries (c0 at column k, c1 at column k+1):
//   no swap: l = f_k / c0, U_k = (c0, c1, 0),            row' = (a_{k+1} - l c1, f_{k+1})
//   swap:    l = c0 / f_k, U_k = (f_k, a_{k+1}, f_{k+1}), row' = (c1 - l a_{k+1}, -l f_{k+1})
// The factorisation is done once (factor = true) and reused.  A zero pivot is
// replaced by `tiny` (inverse iteration wants a huge, not infinite, growth).
template <int ST>
__device__ void tri_solve(const float *__restrict__ d, const float *__restrict__ f, int n, float lam,
                          float *__restrict__ z, float *__restrict__ u0, float *__restrict__ u1,
                          float *__restrict__ u2, float *__restrict__ lm, unsigned char *__restrict__ piv, float tiny,
                          bool factor) {
    if (factor) {
        float c0 = d[0] - lam, c1 = n > 1 ? f[0] : 0.f;
        for (int k = 0; k < n - 1; ++k) {
            const float fk = f[k];
            const float an = d[k + 1] - lam;
            const float fn = k + 1 < n - 1 ? f[k + 1] : 0.f;
            if (fabsf(c0) >= fabsf(fk)) {
                if (c0 == 0.f) c0 = tiny;
                const float rc = 1.f / c0;
                const float l = fk * rc;
                u0[k * ST] = rc; u1[k * ST] = c1; u2[k * ST] = 0.f; lm[k * ST] = l; piv[k * ST] = 0;
                c0 = an - l * c1;
                c1 = fn;
            } else {
                const float l = c0 / fk;
                u0[k * ST] = 1.f / fk; u1[k * ST] = an; u2[k * ST] = fn; lm[k * ST] = l; piv[k * ST] = 1;
                c0 = c1 - l * an;
                c1 = -l * fn;
            }
        }
        if (c0 == 0.f) c0 = tiny;
        u0[(n - 1) * ST] = 1.f / c0; u1[(n - 1) * ST] = 0.f; u2[(n - 1) * ST] = 0.f;
    }
    float zk = z[0];
    for (int k = 0; k < n - 1; ++k) {
        const float zn = z[(k + 1) * ST];
        if (piv[k * ST]) {
            z[k * ST] = zn;
            zk = zk - lm[k * ST] * zn;
        } else {
            z[k * ST] = zk;
            zk = zn - lm[k * ST] * zk;
        }
    }
    z[(n - 1) * ST] = zk;
    float x2 = z[(n - 1) * ST] * u0[(n - 1) * ST];
    z[(n - 1) * ST] = x2;
    if (n > 1) {
        float x1 = (z[(n - 2) * ST] - u1[(n - 2) * ST] * x2) * u0[(n - 2) * ST];
        z[(n - 2) * ST] = x1;
        for (int k = n - 3; k >= 0; --k) {
            const float x0 = (z[k * ST] - u1[k * ST] * x1 - u2[k * ST] * x2) * u0[k * ST];
            z[k * ST] = x0;
            x2 = x1;
            x1 = x0;
        }
    }
}

// ------------------------------------------------------------ tridiagonal
// Tridiagonal data of one matrix in the plan's `tri` buffer (4 floats per
// row): d[n] (real diagonal), tau[n] (reflector scales), e[n] complex
// sub-diagonal (e[k] = T[k+1][k]).
__device__ __forceinline__ float *tri_d(const EigArgs &a, const Group &g, int mat) {
    return a.tri + 4 * (g.soff + (long long)mat * g.s);
}

template <int RPL>
__device__ __forceinline__ cf pick(const cf (&v)[RPL], int t) {
    cf r = v[0];
#pragma unroll
    for (int u = 1; u < RPL; ++u)
        if (u == t) r = v[u];
    return r;
}

__device__ __forceinline__ cf shfl_cf(cf v, int src) {
    return mk(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Householder reduction G = Q T Q^H (lower, packed G in shared memory,
// n <= 32 * RPL).  Lane l of every warp owns rows l, l + 32, ... and keeps
// their entries of the current reflector v and of the previous step's v and
// w in registers; for the per-row phases thread i owns row i.  Step k, with
// the reflector v_k of column k already formed (by step k - 1, or before the
// first step for column 0):
//   1. every lane loads v_k for its rows;
//   2. every warp sweeps its share of the trailing columns j > k once,
//      applying the previous update G -= v w^H + w v^H and accumulating
//      p = G v with the updated values: stored entry G(i, j) adds G(i, j) v_j
//      to the row sum of p_i (registers, per-warp partials in shared memory)
//      and conj(G(i, j)) v_i to p_j (warp reduction, one column per warp, so
//      no atomics);
//   3. thread per row: p = tau (sum of partials), K = tau/2 Re(v^H p)
//      (block sum), w = p - K v;
//   4. thread per row: column k + 1 with this step's update applied, its
//      norm (block sum) and the next reflector v_{k+1}.
// Four barriers per step; the reflector is formed by all threads at once
// instead of by one warp while the others wait.
// Reflector: x = G[k+1:, k], alpha = -e^{i arg x0} ||x||, v = x - alpha e1,
// tau = 2 / v^H v, so (I - tau v v^H) x = alpha e1.
// Columns [0, c0) of the packed matrix stay in global memory and [c0, n) are held in
// shared memory: the smallest c0 for which the shared part, the work arrays of
// k_tridiag and alignment fit in `budget` bytes (0 when everything fits).
__host__ __device__ inline size_t tridiag_smem_c0(int n, int c0) {
    const long long pk = (long long)n * (n + 1) / 2, c0s = (long long)c0 * (2 * n - c0 + 1) / 2;
    return al16((size_t)(pk - c0s) * 8) + (size_t)(EIG_WARPS + 4) * n * 8 + (size_t)n * 4 + 16;
}
__host__ __device__ inline int tridiag_c0(int n, size_t budget) {
    int c0 = 0;
    while (c0 < n && tridiag_smem_c0(n, c0) > budget) ++c0;
    return c0;
}

template <int RPL, bool HYB, bool FULL>
__global__ void __launch_bounds__(EIG_THREADS, 1) k_tridiag(GroupSet gs, int mat_begin, EigArgs a, int budget) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ float red[EIG_WARPS], redk[EIG_WARPS], redx[EIG_WARPS];
    __shared__ cf s_x0, s_p1;
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    clear_flag_before_release(flag_of(a.vready, g, mat));
    pdl_release_dependents();
    if (is_frozen(g, mat, a.active)) return;
    wait_flag(flag_of(a.gready, g, mat), a.status, true);
    const int n = g.s;
    const long long pk = (long long)n * (n + 1) / 2;
    const int c0 = HYB ? tridiag_c0(n, (size_t)budget) : 0;   // columns kept in global memory
    const long long c0s = (long long)c0 * (2 * n - c0 + 1) / 2;
    cf *Gglob = a.Gp + g.poff + (long long)mat * pk;
    cf *Gs = (cf *)tsm;                                   // packed columns c0..n-1
    cf *Pw = Gs + al16((size_t)(pk - c0s) * 8) / 8;      // [EIG_WARPS][n] row-sum partials
    cf *Cs = Pw + (long long)EIG_WARPS * n;               // [n] column sums
    cf *vbuf0 = Cs + n, *vbuf1 = vbuf0 + n;               // v of this / previous step
    cf *wbuf0 = vbuf1 + n;                                // w of the previous step, then of this one
    int *cst = (int *)(wbuf0 + n);                        // [n] column offsets (global for j < c0)
    float *td = tri_d(a, g, mat), *ttau = td + n;
    cf *te = (cf *)(td + 2 * n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // pointer to element (j, j) of packed column j
    auto colp = [&](int j) -> cf * { return (HYB && j < c0) ? Gglob + cst[j] : Gs + cst[j]; };
    for (int j = tid; j < n; j += EIG_THREADS) {
        cst[j] = (int)(colstart(j, n) - (j >= c0 ? c0s : 0));
        vbuf0[j] = vbuf1[j] = wbuf0[j] = mk(0.f, 0.f);
    }
    for (long long i = c0s + tid; i < pk; i += EIG_THREADS) Gs[i - c0s] = Gglob[i];
    __syncthreads();
    float gmax = 0.f;
    for (int j = tid; j < n; j += EIG_THREADS) gmax = fmaxf(gmax, colp(j)[0].x);
    const float floor2 = reflector_floor(bmax(gmax, red));
    cf vo[RPL], wo[RPL], vn[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) vo[t] = wo[t] = vn[t] = mk(0.f, 0.f);
    cf *vcur = vbuf0, *vprev = vbuf1, *wv = wbuf0;
    // Thread-per-row phases: thread tid owns row ir = tid (n <= EIG_THREADS) and keeps its entry of
    // the current reflector in vr.
    const int ir = tid;
    cf vr = mk(0.f, 0.f);
    // Reflector of column c from its updated entries x (thread ir holds x_ir for ir >= c):
    // ||x[c+1:]||^2 and x_{c+1} are reduced over the block (one barrier), every thread forms tau,
    // alpha and its own v_ir in the same order, and v goes to vdst (all rows, zero above c + 1) and
    // to the Householder storage of column c in global memory.
    auto reflect = [&](int c, cf x, cf *vdst) -> float {
        float xn2 = (ir > c && ir < n) ? cabs2(x) : 0.f;
        xn2 = wsum(xn2);
        if (lane == 0) redx[warp] = xn2;
        if (ir == c + 1) s_x0 = x;
        __syncthreads();
        xn2 = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < EIG_WARPS; ++w2) xn2 += redx[w2];
        const cf x0 = s_x0;
        const float ax0 = sqrtf(cabs2(x0));
        const float rest = xn2 - ax0 * ax0;
        float tau = 0.f;
        cf alpha = x0, v0 = mk(0.f, 0.f);
        if (rest > 1e-30f * xn2 && xn2 > floor2) {
            const float xnorm = sqrtf(xn2);
            const cf phs = ax0 > 0.f ? mk(x0.x / ax0, x0.y / ax0) : mk(1.f, 0.f);
            alpha = mk(-phs.x * xnorm, -phs.y * xnorm);
            tau = 1.f / (xn2 + xnorm * ax0);
            v0 = mk(phs.x * (ax0 + xnorm), phs.y * (ax0 + xnorm));
        }
        cf v = mk(0.f, 0.f);
        if (ir > c && ir < n && tau != 0.f) v = ir == c + 1 ? v0 : x;
        if (ir < n) vdst[ir] = v;
        if (ir > c && ir < n) Gglob[colstart(c, n) + (ir - c)] = v;
        if (ir == c) {
            ttau[c] = tau;
            te[c] = alpha;
            td[c] = x.x;
        }
        vr = v;
        return tau;
    };
    float tau = 0.f, tau_prev = 0.f;
    if (n >= 3) {
        tau = reflect(0, ir < n ? colp(0)[ir] : mk(0.f, 0.f), vcur);
        __syncthreads();
    }
    for (int k = 0; k + 2 < n; ++k) {
        // ---- 1. this step's reflector v_k in the lanes' row slots
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            vn[t] = ((FULL || i < n)) ? vcur[i] : mk(0.f, 0.f);
        }
        // ---- 2. fused update + symv over the trailing columns
        const bool upd = tau_prev != 0.f;
        cf pa[RPL];
#pragma unroll
        for (int t = 0; t < RPL; ++t) pa[t] = mk(0.f, 0.f);
        // The sweep is instantiated twice (with and without the deferred update, which only
        // the first step lacks) so that the column loop carries no update branch, and every
        // complex multiply-add is an explicit FMA chain (a - b c - d e ... does not contract
        // into FMAs): 16 FMAs per element and step.
        auto sweep = [&](auto UPDC) {
        constexpr bool UPD = decltype(UPDC)::value;
        // TB columns per pass (j, j + 16, ...): their 2 TB column sums are reduced together
        // by a transpose-reduce butterfly (9 shuffles instead of 10 TB)
        for (int j0 = k + 1 + warp; j0 < n; j0 += TB * EIG_WARPS) {
            float acc[2 * TB];
#pragma unroll
            for (int c = 0; c < TB; ++c) {
                const int j = j0 + c * EIG_WARPS;
                float cr = 0.f, ci = 0.f;
                if (j < n) {                                       // warp-uniform
                    const cf voj = vprev[j], woj = wv[j], vnj = vcur[j];
                    cf *colj = colp(j) - j;
#pragma unroll
                    for (int t = 0; t < RPL; ++t) {
                        if (32 * t + 31 >= j && (FULL || 32 * t < n)) {       // warp-uniform: slot t has rows >= j
                            const int i = lane + 32 * t;
                            if (i >= j && (FULL || i < n)) {
                                cf gv = colj[i];
                                if (UPD) {
                                    gv.x = fmaf(-vo[t].x, woj.x, gv.x);
                                    gv.x = fmaf(-vo[t].y, woj.y, gv.x);
                                    gv.x = fmaf(-wo[t].x, voj.x, gv.x);
                                    gv.x = fmaf(-wo[t].y, voj.y, gv.x);
                                    gv.y = fmaf(-vo[t].y, woj.x, gv.y);
                                    gv.y = fmaf(vo[t].x, woj.y, gv.y);
                                    gv.y = fmaf(-wo[t].y, voj.x, gv.y);
                                    gv.y = fmaf(wo[t].x, voj.y, gv.y);
                                    colj[i] = gv;
                                }
                                pa[t].x = fmaf(gv.x, vnj.x, pa[t].x);
                                pa[t].x = fmaf(-gv.y, vnj.y, pa[t].x);
                                pa[t].y = fmaf(gv.x, vnj.y, pa[t].y);
                                pa[t].y = fmaf(gv.y, vnj.x, pa[t].y);
                                if (i > j) {                       // conj(G(i,j)) v_i -> p_j
                                    cr = fmaf(gv.x, vn[t].x, cr);
                                    cr = fmaf(gv.y, vn[t].y, cr);
                                    ci = fmaf(gv.x, vn[t].y, ci);
                                    ci = fmaf(-gv.y, vn[t].x, ci);
                                }
                            }
                        }
                    }
                }
                acc[2 * c] = cr;
                acc[2 * c + 1] = ci;
            }
            // butterfly: after the halving steps lane L holds value 4 b4 + 2 b3 + b2 (bits of L)
            // summed over its 8-lane group; the last two steps complete the sum
            float b4v[4], b3v[2], s1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool hi = lane & 16;
                const float send = hi ? acc[q] : acc[q + 4];
                const float keep = hi ? acc[q + 4] : acc[q];
                b4v[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const bool hi = lane & 8;
                const float send = hi ? b4v[q] : b4v[q + 2];
                const float keep = hi ? b4v[q + 2] : b4v[q];
                b3v[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
            }
            {
                const bool hi = lane & 4;
                const float send = hi ? b3v[0] : b3v[1];
                const float keep = hi ? b3v[1] : b3v[0];
                s1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
            s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
            if ((lane & 3) == 0) {
                const int v = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                const int j = j0 + (v >> 1) * EIG_WARPS;
                if (j < n) ((float *)Cs)[2 * j + (v & 1)] = s1;
            }
        }
        };
        if (upd) sweep(std::integral_constant<bool, true>());
        else sweep(std::integral_constant<bool, false>());
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            if ((FULL || 32 * t < n) && i >= k + 1 && (FULL || i < n)) Pw[(long long)warp * n + i] = pa[t];
        }
        __syncthreads();
        // ---- 3. p_ir = tau (row partials + column sum) and K = tau/2 Re(v^H p) (thread per row)
        cf p = mk(0.f, 0.f);
        float kv = 0.f;
        if (ir > k && ir < n) {
            float sr = Cs[ir].x, si = Cs[ir].y;
            for (int w2 = 0; w2 < EIG_WARPS; ++w2) {
                const cf q = Pw[(long long)w2 * n + ir];
                sr += q.x;
                si += q.y;
            }
            p = mk(tau * sr, tau * si);
            kv = vr.x * p.x + vr.y * p.y;
            if (ir == k + 1) s_p1 = p;
        }
        kv = wsum(kv);
        if (lane == 0) redk[warp] = kv;
        __syncthreads();
        float kvs = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < EIG_WARPS; ++w2) kvs += redk[w2];
        const float K = 0.5f * tau * kvs;
        const cf w = (ir > k && ir < n) ? mk(p.x - K * vr.x, p.y - K * vr.y) : mk(0.f, 0.f);
        if (ir < n) wv[ir] = w;
        // ---- 4. column k + 1 after this step's update G -= v w^H + w v^H, and its reflector
        float tau_next = 0.f;
        if (k + 3 < n) {                                           // block-uniform
            const cf p1 = s_p1, v1 = vcur[k + 1];
            const cf w1 = mk(p1.x - K * v1.x, p1.y - K * v1.y);
            cf x = mk(0.f, 0.f);
            if (ir > k && ir < n) {
                x = (colp(k + 1) - (k + 1))[ir];
                x.x -= vr.x * w1.x + vr.y * w1.y + w.x * v1.x + w.y * v1.y;
                x.y -= vr.y * w1.x - vr.x * w1.y + w.y * v1.x - w.x * v1.y;
            }
            tau_next = reflect(k + 1, x, vprev);
        } else {
            __syncthreads();
        }
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            wo[t] = ((FULL || i < n)) ? wv[i] : mk(0.f, 0.f);
            vo[t] = vn[t];
        }
        __syncthreads();
        tau_prev = tau;
        tau = tau_next;
        cf *tv = vprev; vprev = vcur; vcur = tv;
    }
    // ---- last step's update on the final 2x2 block, then the remaining d, e
    if (warp == 0) {
        for (int j = (n >= 2 ? n - 2 : 0); j < n; ++j) {
            const cf voj = vprev[j], woj = wv[j];
#pragma unroll
            for (int t = 0; t < RPL; ++t) {
                const int i = lane + 32 * t;
                if (tau_prev != 0.f && (FULL || 32 * t < n) && i >= j && (FULL || i < n)) {
                    cf *cj = colp(j) - j;
                    cf gv = cj[i];
                    gv.x -= vo[t].x * woj.x + vo[t].y * woj.y + wo[t].x * voj.x + wo[t].y * voj.y;
                    gv.y -= vo[t].y * woj.x - vo[t].x * woj.y + wo[t].y * voj.x - wo[t].x * voj.y;
                    cj[i] = gv;
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            if (n >= 2) {
                td[n - 2] = colp(n - 2)[0].x;
                te[n - 2] = colp(n - 2)[1];
                ttau[n - 2] = 0.f;
            }
            td[n - 1] = colp(n - 1)[0].x;
            te[n - 1] = mk(0.f, 0.f);
            ttau[n - 1] = 0.f;
        }
    }
    publish_flag(flag_of(a.ready, g, mat));
}

// Same reduction with G kept in global memory (orders too large for shared
// memory): one thread per row half for the symv, warp-per-column rank-2 update.
__global__ void __launch_bounds__(EIG_THREADS, 1) k_tridiag_g(GroupSet gs, int mat_begin, EigArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ float red[EIG_WARPS];
    __shared__ float s_tau;
    __shared__ cf s_alpha;
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    clear_flag_before_release(flag_of(a.vready, g, mat));
    pdl_release_dependents();
    if (is_frozen(g, mat, a.active)) return;
    wait_flag(flag_of(a.gready, g, mat), a.status, true);
    const int n = g.s;
    const long long pk = (long long)n * (n + 1) / 2;
    cf *Gs = a.Gp + g.poff + (long long)mat * pk;
    cf *vb = (cf *)tsm;
    cf *pb = vb + n;
    int *cst = (int *)(pb + n);
    float *td = tri_d(a, g, mat), *ttau = td + n;
    cf *te = (cf *)(td + 2 * n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < n; j += EIG_THREADS) cst[j] = (int)colstart(j, n);
    __syncthreads();
    float gmax = 0.f;
    for (int j = tid; j < n; j += EIG_THREADS) gmax = fmaxf(gmax, Gs[cst[j]].x);
    const float floor2 = reflector_floor(bmax(gmax, red));
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        cf *col = Gs + cst[k] + 1;
        float xn2 = 0.f;
        for (int i = tid; i < m; i += EIG_THREADS) xn2 += cabs2(col[i]);
        xn2 = bsum(xn2, red);
        const cf x0 = col[0];
        const float ax0 = sqrtf(cabs2(x0));
        const float rest = xn2 - ax0 * ax0;
        if (tid == 0) {
            td[k] = Gs[cst[k]].x;
            if (!(rest > 1e-30f * xn2) || !(xn2 > floor2)) {
                s_tau = 0.f;
                s_alpha = x0;
            } else {
                const float xnorm = sqrtf(xn2);
                const cf phs = ax0 > 0.f ? mk(x0.x / ax0, x0.y / ax0) : mk(1.f, 0.f);
                s_alpha = mk(-phs.x * xnorm, -phs.y * xnorm);
                s_tau = 1.f / (xn2 + xnorm * ax0);
                vb[0] = mk(phs.x * (ax0 + xnorm), phs.y * (ax0 + xnorm));
            }
            ttau[k] = s_tau;
            te[k] = s_alpha;
        }
        __syncthreads();
        const float tau = s_tau;
        if (tau == 0.f) {
            for (int i = tid; i < m; i += EIG_THREADS) col[i] = mk(0.f, 0.f);   // zero reflector
            __syncthreads();
            continue;
        }
        for (int i = tid + 1; i < m; i += EIG_THREADS) vb[i] = col[i];
        __syncthreads();
        for (int i = tid; i < m; i += EIG_THREADS) col[i] = vb[i];              // reflector in place
        // symv: two threads per row (halves of the row), loop bound padded to a multiple of
        // 32 so that every lane reaches the pair shuffle (inactive lanes add zeros)
        const int nrow2 = 2 * m, nrow2_pad = (nrow2 + 31) & ~31;
        for (int t2i = tid; t2i < nrow2_pad; t2i += EIG_THREADS) {
            const bool act = t2i < nrow2;
            const int i = t2i >> 1, half = t2i & 1;
            const int I = k + 1 + i;
            const int j0 = act ? (half ? (m >> 1) : 0) : 0, j1 = act ? (half ? m : (m >> 1)) : 0;
            float sr = 0.f, si = 0.f;
            int j = j0;
            for (; j < j1 && j <= i; ++j) {
                const int J = k + 1 + j;
                const cf gv = Gs[cst[J] + (I - J)];
                const cf v = vb[j];
                sr += gv.x * v.x - gv.y * v.y;
                si += gv.x * v.y + gv.y * v.x;
            }
            if (j < j1) {
                const cf *ci = Gs + cst[I];
                for (; j < j1; ++j) {
                    const cf gv = ci[j - i];
                    const cf v = vb[j];
                    sr += gv.x * v.x + gv.y * v.y;
                    si += gv.x * v.y - gv.y * v.x;
                }
            }
            sr += __shfl_xor_sync(0xffffffffu, sr, 1);
            si += __shfl_xor_sync(0xffffffffu, si, 1);
            if (act && !half) pb[i] = mk(tau * sr, tau * si);
        }
        __syncthreads();
        float kv = 0.f;
        for (int i = tid; i < m; i += EIG_THREADS) kv += vb[i].x * pb[i].x + vb[i].y * pb[i].y;
        kv = bsum(kv, red);
        const float K = 0.5f * tau * kv;
        for (int i = tid; i < m; i += EIG_THREADS) pb[i] = mk(pb[i].x - K * vb[i].x, pb[i].y - K * vb[i].y);
        __syncthreads();
        for (int j = warp; j < m; j += EIG_WARPS) {
            const cf vj = vb[j], wj = pb[j];
            cf *cj = Gs + cst[k + 1 + j];
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
    if (tid == 0) {
        if (n >= 2) {
            td[n - 2] = Gs[cst[n - 2]].x;
            te[n - 2] = Gs[cst[n - 2] + 1];
            ttau[n - 2] = 0.f;
        }
        td[n - 1] = Gs[cst[n - 1]].x;
        te[n - 1] = mk(0.f, 0.f);
        ttau[n - 1] = 0.f;
    }
    publish_flag(flag_of(a.ready, g, mat));
}

// ------------------------------------------- two-stage reduction (orders SB_NMIN .. SB_NMAX)
// The one-stage reduction above is a chain of n - 2 dependent Householder steps, each with
// block-wide reductions and a pass over the whole trailing matrix.  The two-stage form
// reduces G first to a Hermitian band of half-bandwidth b = SB_B with blocked reflectors
// (about n / b dependent panel steps; the trailing updates are rank-2b products with b-fold
// reuse of every loaded element), then the band to tridiagonal by bulge chasing.
//
// Stage 1, k_sb1 (one CTA per matrix, packed G in shared memory).  For the panel of columns
// c0 .. c0 + b - 1 and rows r0 = c0 + b .. n - 1 (m = n - r0 rows):
//   QR of the panel: nr = min(b, m - 1) reflectors H_t = I - tau_t v_t v_t^H, one warp per
//     panel column, one barrier per reflector (Q = H_0 ... H_{nr-1} = I - V T V^H);
//   S = V^H V and Y = V T, with T^-1 = diag(1 / tau) + (strict upper part of S), by a
//     triangular solve per row of V;
//   trailing update A <- Q^H A Q on rows / columns r0 .. n - 1 as
//     X = A Y,  M = Y^H X,  W = X - V M / 2,  A <- A - W V^H - V W^H.
// The band (diagonals 0 .. b) goes to the scratch, the reflectors to the packed buffer (column c
// holds v of the panel reflector of that column on rows c + b .. n - 1) and tau_c to the tau
// slots of the tridiagonal data.
//
// Stage 2, k_sb2 (one CTA of eight warps per matrix, the band with room for the bulge in
// shared memory).  Sweep j (j = 0 .. n - 3) has steps k = 1 .. sb_nsteps(n, j): step 1
// annihilates column j below its first sub-diagonal with a reflector on rows j + 1 .. j + b;
// step k > 1 annihilates the first column of the bulge the previous step left below the band
// (column j + 1 + (k - 2) b) on rows j + 1 + (k - 1) b .. j + k b.  Each reflector is applied
// from the left to the columns between that column and its window, from both sides to the
// window's diagonal block and from the right to the b rows below the window.  Step k of sweep
// j runs at time 3 j + k: the steps that share a time touch disjoint entries, and every entry
// a step reads was last written by a step of an earlier time, so a pair of warps per step
// with a barrier per time gives the same matrix as the sweeps run one after the other.  The
// reflectors are stored sweep-major; the tridiagonal d, e goes to the tridiagonal data.
//
// Back-transformation (k_eigvec with EigArgs::band): y = Q1 Q2 P z; Q2 = S_0 S_1 ... S_{n-3}
// with S_j the product of the (commuting: disjoint windows) reflectors of sweep j, applied for
// j = n - 3 .. 0; then the panel reflectors, as the one-stage reflectors with their first row
// b - 1 rows further down.

// Reduction mode 0 ("by order") takes the two-stage reduction from this order up: never, since
// the one-stage reduction was faster at order 192, the order measured (the autotuner still
// tries the two-stage reduction on each plan).
#define SB_AUTO_MIN (1 << 30)
#define SB1_THREADS 512
#define SB1_RPL 6                  // panel rows per lane: n - SB_B <= 32 SB1_RPL for n <= SB_NMAX

struct Sb1Layout {
    size_t gs, vd, xs, ys, sm, mm, total;
};
__host__ __device__ inline Sb1Layout sb1_layout(int n) {
    Sb1Layout L;
    const size_t mm = (size_t)(n > SB_B ? n - SB_B : 1);
    size_t o = 0;
    L.gs = o; o += al16((size_t)n * (n + 1) / 2 * 8);
    L.vd = o; o += al16(mm * SB_B * 8);
    L.xs = o; o += al16((mm * SB_B + SB_B) * 8);    // also the column-major reflectors of the QR
    L.ys = o; o += al16(mm * SB_B * 8);
    L.sm = o; o += SB_B * SB_B * 8;
    L.mm = o; o += SB_B * SB_B * 8;
    L.total = o;
    return L;
}

// Householder reflector of x (this warp's entries xs[q] at local rows lane + 32 q, rows < t0
// excluded, x0 on local row t0 < 32, in lane t0 slot 0): (I - tau v v^H) x = alpha e1 with
// v0 = phs (|x0| + ||x||) and v = x below; tau = 0 when the column is already reduced.
__device__ __forceinline__ void sb_reflector(float xn2, cf x0, float floor2, float *tau, cf *alpha, cf *v0) {
    const float ax0 = sqrtf(cabs2(x0));
    const float rest = xn2 - ax0 * ax0;
    *tau = 0.f;
    *alpha = x0;
    *v0 = mk(0.f, 0.f);
    if (rest > 1e-30f * xn2 && xn2 > floor2) {
        const float xnorm = sqrtf(xn2);
        const cf phs = ax0 > 0.f ? mk(x0.x / ax0, x0.y / ax0) : mk(1.f, 0.f);
        *alpha = mk(-phs.x * xnorm, -phs.y * xnorm);
        *tau = 1.f / (xn2 + xnorm * ax0);
        *v0 = mk(phs.x * (ax0 + xnorm), phs.y * (ax0 + xnorm));
    }
}

__global__ void __launch_bounds__(SB1_THREADS, 1) k_sb1(GroupSet gs, int mat_begin, EigArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ float red[EIG_WARPS];
    __shared__ float s_pt[SB_B];
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    clear_flag_before_release(flag_of(a.vready, g, mat));
    pdl_release_dependents();
    if (is_frozen(g, mat, a.active)) return;
    wait_flag(flag_of(a.gready, g, mat), a.status, true);
    const int n = g.s;
    const long long pk = (long long)n * (n + 1) / 2;
    cf *Gglob = a.Gp + g.poff + (long long)mat * pk;
    cf *band = a.sb + g.sboff + (long long)mat * sb_stride(n);
    float *ttau = tri_d(a, g, mat) + n;
    const Sb1Layout LY = sb1_layout(n);
    cf *Gs = (cf *)(tsm + LY.gs), *Vd = (cf *)(tsm + LY.vd), *Xs = (cf *)(tsm + LY.xs), *Ys = (cf *)(tsm + LY.ys);
    cf *Sm = (cf *)(tsm + LY.sm), *Mm = (cf *)(tsm + LY.mm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (long long i = tid; i < pk; i += SB1_THREADS) Gs[i] = Gglob[i];
    for (int j = tid; j < n; j += SB1_THREADS) ttau[j] = 0.f;
    __syncthreads();
    float gmax = 0.f;
    for (int j = tid; j < n; j += SB1_THREADS) gmax = fmaxf(gmax, Gs[colstart(j, n)].x);
    const float floor2 = reflector_floor(bmax(gmax, red));
    int c0 = 0;
    for (; c0 + SB_B < n - 1; c0 += SB_B) {
        const int r0 = c0 + SB_B, m = n - r0, nr = min(SB_B, m - 1);
        // ---- QR of the panel: warp w holds column cw = c0 + w, local rows lane + 32 q
        const int cw = c0 + warp;
        const cf *colw = Gs + colstart(cw, n) - cw;       // colw[i] = G(i, cw), i >= cw
        cf x[SB1_RPL];
#pragma unroll
        for (int q = 0; q < SB1_RPL; ++q) {
            const int i = lane + 32 * q;
            x[q] = i < m ? colw[r0 + i] : mk(0.f, 0.f);
        }
        // reflectors column-major in the X buffer (odd column stride: the transposition below reads
        // a row across the columns without bank conflicts)
        cf *Vc = Xs;
        const int vst = (m & 1) ? m : m + 1;
        for (int t = 0; t < nr; ++t) {
            const cf *vs = Vc + t * vst;
            if (warp == t) {
                float xn2 = 0.f;
#pragma unroll
                for (int q = 0; q < SB1_RPL; ++q) {
                    const int i = lane + 32 * q;
                    if (i >= t && i < m) xn2 += cabs2(x[q]);
                }
                xn2 = wsum(xn2);
                const cf x0 = shfl_cf(x[0], t);
                float tau;
                cf alpha, v0;
                sb_reflector(xn2, x0, floor2, &tau, &alpha, &v0);
#pragma unroll
                for (int q = 0; q < SB1_RPL; ++q) {
                    const int i = lane + 32 * q;
                    cf v = mk(0.f, 0.f);
                    if (tau != 0.f && i >= t && i < m) v = i == t ? v0 : x[q];
                    if (i < m) Vc[t * vst + i] = v;
                    if (tau != 0.f && i >= t) x[q] = i == t ? alpha : mk(0.f, 0.f);
                }
                if (lane == 0) {
                    s_pt[t] = tau;
                    ttau[cw] = tau;
                }
            }
            __syncthreads();
            if (warp > t) {
                const float tau = s_pt[t];
                if (tau != 0.f) {
                    float dr = 0.f, di = 0.f;
#pragma unroll
                    for (int q = 0; q < SB1_RPL; ++q) {
                        const int i = lane + 32 * q;
                        if (i >= t && i < m) {
                            const cf v = vs[i];
                            dr += v.x * x[q].x + v.y * x[q].y;
                            di += v.x * x[q].y - v.y * x[q].x;
                        }
                    }
                    dr = tau * wsum(dr);
                    di = tau * wsum(di);
#pragma unroll
                    for (int q = 0; q < SB1_RPL; ++q) {
                        const int i = lane + 32 * q;
                        if (i >= t && i < m) {
                            const cf v = vs[i];
                            x[q].x -= v.x * dr - v.y * di;
                            x[q].y -= v.x * di + v.y * dr;
                        }
                    }
                }
            }
        }
        // ---- band of the panel's column: rows cw .. r0 - 1 from G, rows r0 .. r0 + w from R;
        // the reflector to the packed buffer (rows cw + b ..); columns without one get V = 0
        {
            const int dr0 = SB_B - warp;                   // first diagonal taken from R
            const cf xv = shfl_cf(x[0], (lane - dr0) & 31);
            if (lane <= SB_B) {
                cf val = mk(0.f, 0.f);
                if (cw + lane < n) val = lane < dr0 ? colw[cw + lane] : xv;
                band[(long long)cw * (SB_B + 1) + lane] = val;
            }
            if (warp < nr)
                for (int i = warp + lane; i < m; i += 32) Gglob[colstart(cw, n) + (r0 + i - cw)] = Vc[warp * vst + i];
        }
        __syncthreads();
        for (int idx = tid; idx < m * SB_B; idx += SB1_THREADS) {
            const int i = idx >> 4, t = idx & 15;
            Vd[idx] = t < nr ? Vc[t * vst + i] : mk(0.f, 0.f);
        }
        __syncthreads();
        // ---- S = V^H V (strict upper part; warp t: column t)
        if (warp > 0 && warp < nr) {                       // lanes (row parity r, column p)
            const int t = warp, r = lane >> 4, pc = lane & 15;
            float sr0 = 0.f, si0 = 0.f, sr1 = 0.f, si1 = 0.f;
            int i = t + r;
            for (; i + 2 < m; i += 4) {
                const cf vp = Vd[i * SB_B + pc], vt = Vd[i * SB_B + t];
                const cf wp = Vd[(i + 2) * SB_B + pc], wt = Vd[(i + 2) * SB_B + t];
                sr0 += vp.x * vt.x + vp.y * vt.y;
                si0 += vp.x * vt.y - vp.y * vt.x;
                sr1 += wp.x * wt.x + wp.y * wt.y;
                si1 += wp.x * wt.y - wp.y * wt.x;
            }
            if (i < m) {
                const cf vp = Vd[i * SB_B + pc], vt = Vd[i * SB_B + t];
                sr0 += vp.x * vt.x + vp.y * vt.y;
                si0 += vp.x * vt.y - vp.y * vt.x;
            }
            float sr = sr0 + sr1, si = si0 + si1;
            sr += __shfl_xor_sync(0xffffffffu, sr, 16);
            si += __shfl_xor_sync(0xffffffffu, si, 16);
            if (r == 0 && pc < t) Sm[pc * SB_B + t] = mk(sr, si);
        }
        __syncthreads();
        // ---- Y = V T without forming T: T^-1 = U = diag(1 / tau) + (strict upper part of S) (the
        // inverse of the forward recurrence for T), so each row of Y solves y U = v:
        //   y_t = tau_t (v_t - sum_{p < t} y_p S_pt)
        for (int i = tid; i < m; i += SB1_THREADS) {
            cf y[SB_B];
            const float4 *vr = (const float4 *)(Vd + i * SB_B);
#pragma unroll
            for (int q = 0; q < SB_B / 2; ++q) {
                const float4 v4 = vr[q];
                y[2 * q] = mk(v4.x, v4.y);
                y[2 * q + 1] = mk(v4.z, v4.w);
            }
#pragma unroll
            for (int t = 0; t < SB_B; ++t) {
                float ar = y[t].x, ai = y[t].y;
#pragma unroll
                for (int p = 0; p < t; ++p) {
                    const cf sv = Sm[p * SB_B + t];
                    ar -= y[p].x * sv.x - y[p].y * sv.y;
                    ai -= y[p].x * sv.y + y[p].y * sv.x;
                }
                const float tt = t < nr ? s_pt[t] : 0.f;
                y[t] = mk(tt * ar, tt * ai);
            }
            float4 *yw = (float4 *)(Ys + i * SB_B);
#pragma unroll
            for (int q = 0; q < SB_B / 2; ++q) yw[q] = make_float4(y[2 * q].x, y[2 * q].y, y[2 * q + 1].x, y[2 * q + 1].y);
        }
        __syncthreads();
        // ---- X = A Y over rows / columns r0 .. n - 1 (warp item: 32 rows x 8 columns of X)
        const int nrb = (m + 31) >> 5;
        for (int item = warp; item < 2 * nrb; item += EIG_WARPS) {
            const int rb = item >> 1, h = item & 1;
            const int il = 32 * rb + lane, i = r0 + il;
            const bool valid = il < m;
            float acc[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[u] = 0.f;
            const long long csi = valid ? colstart(i, n) : 0;
            long long csj = colstart(r0, n);
            for (int jl = 0; jl < m; ++jl) {
                const int j = r0 + jl;
                cf av = mk(0.f, 0.f);
                if (valid) {
                    const long long ix = j <= i ? csj + (i - j) : csi + (j - i);
                    av = Gs[ix];
                    if (j > i) av.y = -av.y;
                }
                const float4 *yr = (const float4 *)(Ys + jl * SB_B + 8 * h);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 y4 = yr[q];
                    acc[4 * q + 0] = fmaf(av.x, y4.x, acc[4 * q + 0]);
                    acc[4 * q + 0] = fmaf(-av.y, y4.y, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(av.x, y4.y, acc[4 * q + 1]);
                    acc[4 * q + 1] = fmaf(av.y, y4.x, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(av.x, y4.z, acc[4 * q + 2]);
                    acc[4 * q + 2] = fmaf(-av.y, y4.w, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(av.x, y4.w, acc[4 * q + 3]);
                    acc[4 * q + 3] = fmaf(av.y, y4.z, acc[4 * q + 3]);
                }
                csj += n - j;
            }
            if (valid) {
                float4 *xr = (float4 *)(Xs + il * SB_B + 8 * h);
#pragma unroll
                for (int q = 0; q < 4; ++q) xr[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            }
        }
        __syncthreads();
        // ---- M = Y^H X (warp p: row p)
        {                                                  // lanes (row parity r, column q)
            const int p = warp, r = lane >> 4, q = lane & 15;
            float mr0 = 0.f, mi0 = 0.f, mr1 = 0.f, mi1 = 0.f;
            int i = r;
            for (; i + 2 < m; i += 4) {
                const cf yp = Ys[i * SB_B + p], xq = Xs[i * SB_B + q];
                const cf zp = Ys[(i + 2) * SB_B + p], wq = Xs[(i + 2) * SB_B + q];
                mr0 += yp.x * xq.x + yp.y * xq.y;
                mi0 += yp.x * xq.y - yp.y * xq.x;
                mr1 += zp.x * wq.x + zp.y * wq.y;
                mi1 += zp.x * wq.y - zp.y * wq.x;
            }
            if (i < m) {
                const cf yp = Ys[i * SB_B + p], xq = Xs[i * SB_B + q];
                mr0 += yp.x * xq.x + yp.y * xq.y;
                mi0 += yp.x * xq.y - yp.y * xq.x;
            }
            float mr = mr0 + mr1, mi = mi0 + mi1;
            mr += __shfl_xor_sync(0xffffffffu, mr, 16);
            mi += __shfl_xor_sync(0xffffffffu, mi, 16);
            if (r == 0) Mm[p * SB_B + q] = mk(mr, mi);
        }
        __syncthreads();
        // ---- W = X - V M / 2, in place
        for (int idx = tid; idx < m * SB_B; idx += SB1_THREADS) {
            const int i = idx >> 4, q = idx & 15;
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int p = 0; p < SB_B; ++p) {
                const cf v = Vd[i * SB_B + p], mv = Mm[p * SB_B + q];
                ar += v.x * mv.x - v.y * mv.y;
                ai += v.x * mv.y + v.y * mv.x;
            }
            const cf xv = Xs[idx];
            Xs[idx] = mk(xv.x - 0.5f * ar, xv.y - 0.5f * ai);
        }
        __syncthreads();
        // ---- A <- A - W V^H - V W^H on the lower triangle (warp item: a 32 x 32 tile)
        const int ntiles = nrb * (nrb + 1) / 2;
        for (int tile = warp; tile < ntiles; tile += EIG_WARPS) {
            int rb = 0, cb = tile;
            while (cb > rb) {
                cb -= rb + 1;
                ++rb;
            }
            const int il = 32 * rb + lane;
            const bool valid = il < m;
            cf wi[SB_B], vi[SB_B];
#pragma unroll
            for (int p = 0; p < SB_B; ++p) {
                wi[p] = valid ? Xs[il * SB_B + p] : mk(0.f, 0.f);
                vi[p] = valid ? Vd[il * SB_B + p] : mk(0.f, 0.f);
            }
            const int jl1 = min(32 * cb + 32, m);
            long long csj = colstart(r0 + 32 * cb, n);
            for (int jl = 32 * cb; jl < jl1; csj += n - (r0 + jl), ++jl) {
                if (valid && jl <= il) {
                    cf *ap = Gs + csj + (il - jl);
                    float ar = ap->x, ai = ap->y;
                    const float4 *vr = (const float4 *)(Vd + jl * SB_B), *wr = (const float4 *)(Xs + jl * SB_B);
#pragma unroll
                    for (int q = 0; q < SB_B / 2; ++q) {
                        const float4 v4 = vr[q], w4 = wr[q];
                        // a -= w_i conj(v_j) + v_i conj(w_j), two columns per float4
                        ar = fmaf(-wi[2 * q].x, v4.x, ar); ar = fmaf(-wi[2 * q].y, v4.y, ar);
                        ai = fmaf(wi[2 * q].x, v4.y, ai);  ai = fmaf(-wi[2 * q].y, v4.x, ai);
                        ar = fmaf(-vi[2 * q].x, w4.x, ar); ar = fmaf(-vi[2 * q].y, w4.y, ar);
                        ai = fmaf(vi[2 * q].x, w4.y, ai);  ai = fmaf(-vi[2 * q].y, w4.x, ai);
                        ar = fmaf(-wi[2 * q + 1].x, v4.z, ar); ar = fmaf(-wi[2 * q + 1].y, v4.w, ar);
                        ai = fmaf(wi[2 * q + 1].x, v4.w, ai);  ai = fmaf(-wi[2 * q + 1].y, v4.z, ai);
                        ar = fmaf(-vi[2 * q + 1].x, w4.z, ar); ar = fmaf(-vi[2 * q + 1].y, w4.w, ar);
                        ai = fmaf(vi[2 * q + 1].x, w4.w, ai);  ai = fmaf(-vi[2 * q + 1].y, w4.z, ai);
                    }
                    *ap = mk(ar, ai);
                }
            }
        }
        __syncthreads();
    }
    // ---- band of the remaining columns (already within the band)
    for (int idx = tid; idx < (n - c0) * (SB_B + 1); idx += SB1_THREADS) {
        const int c = c0 + idx / (SB_B + 1), d = idx - (c - c0) * (SB_B + 1);
        band[(long long)c * (SB_B + 1) + d] = c + d < n ? Gs[colstart(c, n) + d] : mk(0.f, 0.f);
    }
    publish_flag(flag_of(a.bready, g, mat));
}

#define SB2_THREADS 256
#define SB2_WARPS (SB2_THREADS / 32)
#define SB2_LD (2 * SB_B)          // stored diagonals 0 .. 2 b - 1 (band and bulge)

__host__ __device__ inline size_t sb2_smem(int n) { return (size_t)n * SB2_LD * 8; }

// One bulge-chasing step (sweep j, step k) by a pair of warps on the band Ls
// (Ls[c LD + d] = A(c + d, c)).  Both warps form the reflector (the same arithmetic, so the
// same v and tau) from A[r0 .. r1, c]; after a pair barrier (both have read the column) warp 0
// writes the annihilated column and the reflector and applies it from both sides to the
// window's diagonal block (lane l: row l), while warp 1 applies it from the left to the
// columns between c and the window (lanes 0 .. 14) and from the right to the rows below the
// window (lanes 16 ..).  Every lane first loads the entries it updates, then computes, then
// stores.
__device__ __forceinline__ void sb2_step(cf *Ls, int n, int j, int k, float floor2, cf *rec, cf *sv, cf *sw,
                                         int role, int pair, int lane) {
    int c, r0, r1;
    if (k == 1) {
        c = j;
        r0 = j + 1;
        r1 = min(j + SB_B, n - 1);
    } else {
        c = j + 1 + (k - 2) * SB_B;
        r0 = j + 1 + (k - 1) * SB_B;
        r1 = min(j + k * SB_B, n - 1);
    }
    const int L = r1 - r0 + 1;                 // 2 .. SB_B
    const bool lo = lane < SB_B;
    const int l = lane & (SB_B - 1);
    cf x = mk(0.f, 0.f);
    if (lo && l < L) x = Ls[c * SB2_LD + (r0 - c) + l];
    float xn2 = cabs2(x);
#pragma unroll
    for (int o = SB_B / 2; o > 0; o >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, o);
    xn2 = __shfl_sync(0xffffffffu, xn2, 0);
    const cf x0 = shfl_cf(x, 0);
    float tau;
    cf alpha, v0;
    sb_reflector(xn2, x0, floor2, &tau, &alpha, &v0);
    cf v = mk(0.f, 0.f);
    if (tau != 0.f && lo && l < L) v = l == 0 ? v0 : x;
    if (role == 0 && lo) sv[l] = v;
    // pair barrier (ids 1 .. 4, compile-time so that only five barriers are reserved): column c
    // read by both warps, v in sv
    switch (pair) {
    case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    }
    if (role == 0) {
        if (lane == 0) rec[0] = mk(tau, __int_as_float(r0));
        if (lo) rec[1 + l] = v;
    }
    if (tau == 0.f) return;
    if (role == 0) {
        if (lo && l < L) Ls[c * SB2_LD + (r0 - c) + l] = l == 0 ? alpha : mk(0.f, 0.f);
        // diagonal block D = A[r0 .. r1, r0 .. r1]: p = tau D v, K = tau / 2 v^H p, w = p - K v,
        // D <- D - v w^H - w v^H (lower part, lane l: row l)
        float pr = 0.f, pi = 0.f;
#pragma unroll
        for (int i2 = 0; i2 < SB_B; ++i2) {
            if (lo && l < L && i2 < L) {
                const int ix = i2 <= l ? (r0 + i2) * SB2_LD + (l - i2) : (r0 + l) * SB2_LD + (i2 - l);
                cf dv = Ls[ix];
                if (i2 > l) dv.y = -dv.y;
                if (i2 == l) dv.y = 0.f;
                const cf vv = sv[i2];
                pr += dv.x * vv.x - dv.y * vv.y;
                pi += dv.x * vv.y + dv.y * vv.x;
            }
        }
        const cf p = mk(tau * pr, tau * pi);
        float kv = (lo && l < L) ? v.x * p.x + v.y * p.y : 0.f;
#pragma unroll
        for (int o = SB_B / 2; o > 0; o >>= 1) kv += __shfl_xor_sync(0xffffffffu, kv, o);
        kv = __shfl_sync(0xffffffffu, kv, 0);
        const float K = 0.5f * tau * kv;
        const cf w = mk(p.x - K * v.x, p.y - K * v.y);
        if (lo) sw[l] = w;
        __syncwarp();
        if (lo && l < L) {
#pragma unroll
            for (int i2 = 0; i2 < SB_B; ++i2) {
                if (i2 <= l) {
                    cf *dp = Ls + (r0 + i2) * SB2_LD + (l - i2);
                    const cf d0 = *dp, vj = sv[i2], wj = sw[i2];
                    float ur = d0.x, ui = d0.y;
                    ur -= v.x * wj.x + v.y * wj.y + w.x * vj.x + w.y * vj.y;
                    ui -= v.y * wj.x - v.x * wj.y + w.y * vj.x - w.x * vj.y;
                    if (i2 == l) ui = 0.f;
                    *dp = mk(ur, ui);
                }
            }
        }
    } else {
        cf *ep = nullptr;                      // lane's column (left of the window) or row (below)
        int stride = 0;
        bool act = false;
        if (lo) {
            if (k >= 2 && lane < r0 - c - 1) {
                const int cc = c + 1 + lane;
                ep = Ls + cc * SB2_LD + (r0 - cc);           // A[r0 + i, cc] = ep[i]
                stride = 1;
                act = true;
            }
        } else {
            const int row = r1 + 1 + (lane - SB_B);
            if (row < n && lane - SB_B < SB_B) {
                ep = Ls + r0 * SB2_LD + (row - r0);           // A[row, r0 + i] = ep[i (LD - 1)]
                stride = SB2_LD - 1;
                act = true;
            }
        }
        // conj(v) for a column (s = v^H col), v for a row (s = row v): one code path with
        // cs = -1 / +1 on the imaginary part of v
        const float cs = lo ? -1.f : 1.f;
        cf e[SB_B];
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int i = 0; i < SB_B; ++i) {
            e[i] = (act && i < L) ? ep[i * stride] : mk(0.f, 0.f);
            const cf vv = sv[i];
            const float vy = cs * vv.y;
            sr += e[i].x * vv.x - e[i].y * vy;
            si += e[i].x * vy + e[i].y * vv.x;
        }
        sr *= tau;
        si *= tau;
        if (act) {
#pragma unroll
            for (int i = 0; i < SB_B; ++i) {
                if (i < L) {
                    // column: col -= v s;  row: row -= s conj(v)
                    const cf vv = sv[i];
                    const float vy = -cs * vv.y;
                    cf u = e[i];
                    u.x -= vv.x * sr - vy * si;
                    u.y -= vv.x * si + vy * sr;
                    ep[i * stride] = u;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(SB2_THREADS, 4) k_sb2(GroupSet gs, int mat_begin, EigArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ float red[SB2_WARPS];
    __shared__ cf s_v[SB2_WARPS / 2][SB_B], s_w[SB2_WARPS / 2][SB_B];
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    pdl_release_dependents();
    if (is_frozen(g, mat, a.active)) return;
    wait_flag(flag_of(a.bready, g, mat), a.status, true);
    const int n = g.s;
    const cf *band = a.sb + g.sboff + (long long)mat * sb_stride(n);
    cf *rec = a.sb + g.sboff + (long long)mat * sb_stride(n) + (long long)n * (SB_B + 1);
    float *td = tri_d(a, g, mat);
    cf *te = (cf *)(td + 2 * n);
    cf *Ls = (cf *)bsm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float gm = 0.f;
    for (int idx = tid; idx < n * SB2_LD; idx += SB2_THREADS) {
        const int c = idx / SB2_LD, d = idx - c * SB2_LD;
        const cf v = d <= SB_B ? band[(long long)c * (SB_B + 1) + d] : mk(0.f, 0.f);
        Ls[idx] = v;
        if (d == 0) gm = fmaxf(gm, fabsf(v.x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if (lane == 0) red[warp] = gm;
    __syncthreads();
    for (int w = 0; w < SB2_WARPS; ++w) gm = fmaxf(gm, red[w]);
    const float floor2 = reflector_floor(gm);
    const int pair = warp >> 1, role = warp & 1;
    if (n >= 3) {
        const int kmax = sb_nsteps(n, 0);
        const int tlast = 3 * (n - 3) + sb_nsteps(n, n - 3);
        for (int tt = 1; tt <= tlast; ++tt) {
            // the steps of this time: k = tt mod 3 (1 .. 3), + 3, ...; pair q takes the q-th, the q+4-th, ...
            for (int k = (tt - 1) % 3 + 1 + 3 * pair; k <= kmax; k += 3 * (SB2_WARPS / 2)) {
                const int j = (tt - k) / 3;               // tt - k is a multiple of 3
                if (tt - k < 0 || j > n - 3 || k > sb_nsteps(n, j)) continue;
                sb2_step(Ls, n, j, k, floor2, rec + (sb_sweep_off(n, j) + k - 1) * (SB_B + 1), s_v[pair], s_w[pair],
                         role, pair, lane);
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += SB2_THREADS) {
        td[i] = Ls[i * SB2_LD].x;
        te[i] = i + 1 < n ? Ls[i * SB2_LD + 1] : mk(0.f, 0.f);
    }
    publish_flag(flag_of(a.ready, g, mat));
}

// ------------------------------------------------ real tridiagonal setup
// T = P T_r P^H with T_r real symmetric: f_k = |e_k| and phases ph_0 = 1,
// ph_{k+1} = ph_k e_k / |e_k| (warp 0 runs a product scan).  The caller
// synchronises before using the outputs.
__device__ __forceinline__ void tri_real_setup(const float *td, const float *ttau, const cf *te, int n, float *dd,
                                               float *taus, float *ff, float *f2, cf *ph, int tid, int lane,
                                               int warp, int nthreads = EIG_THREADS) {
    for (int k = tid; k < n; k += nthreads) {
        dd[k] = td[k];
        taus[k] = ttau[k];
        const float ae = k + 1 < n ? sqrtf(cabs2(te[k])) : 0.f;
        ff[k] = ae;
        f2[k] = ae * ae;
    }
    if (warp == 0) {
        const int per = (n + 31) / 32, k0 = lane * per, k1 = min(n, k0 + per);
        cf loc = mk(1.f, 0.f);
        for (int k = k0; k < k1; ++k) {
            const cf e = k + 1 < n ? te[k] : mk(0.f, 0.f);
            const float ae = sqrtf(cabs2(e));
            if (ae > 0.f) loc = cmul(loc, mk(e.x / ae, e.y / ae));
        }
        // exclusive product scan of the lane products
        cf incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const cf up = shfl_cf(incl, max(lane - o, 0));
            if (lane >= o) incl = cmul(up, incl);
        }
        cf cur = shfl_cf(incl, max(lane - 1, 0));
        if (lane == 0) cur = mk(1.f, 0.f);
        for (int k = k0; k < k1; ++k) {
            ph[k] = cur;
            const cf e = k + 1 < n ? te[k] : mk(0.f, 0.f);
            const float ae = sqrtf(cabs2(e));
            if (ae > 0.f) cur = cmul(cur, mk(e.x / ae, e.y / ae));
        }
    }
}

// Gershgorin interval [gl, gu] of T_r and the pivot floor of its Sturm counts.
__device__ __forceinline__ void gershgorin(const float *dd, const float *ff, const float *f2, int n, float *gl_,
                                           float *gu_, float *pivmin_) {
    float gl = FLT_MAX, gu = -FLT_MAX, fm2 = 0.f;
    for (int k = 0; k < n; ++k) {
        const float r0 = (k > 0 ? ff[k - 1] : 0.f) + (k + 1 < n ? ff[k] : 0.f);
        gl = fminf(gl, dd[k] - r0);
        gu = fmaxf(gu, dd[k] + r0);
        fm2 = fmaxf(fm2, f2[k]);
    }
    *gl_ = gl;
    *gu_ = gu;
    *pivmin_ = FLT_MIN * fmaxf(1.f, fm2);
}

// ---------------------------------------------------------------- eigvec
// Shared-memory layout of k_eigvec (16-byte aligned regions).
struct EvLayout {
    size_t ph, dd, ff, f2, taus, lam, clu, zv, lu0, lu1, lu2, llm, lpv, yc, total;
};
__host__ __device__ inline EvLayout ev_layout(int n, int chunk, int st) {
    EvLayout L;
    size_t o = 0;
    L.ph = o; o += al16((size_t)n * 8);
    L.dd = o; o += al16((size_t)n * 4);
    L.ff = o; o += al16((size_t)n * 4);
    L.f2 = o; o += al16((size_t)n * 4);
    L.taus = o; o += al16((size_t)n * 4);
    L.lam = o; o += al16((size_t)n * 4);
    L.clu = o; o += al16((size_t)n * 4);
    L.zv = o; o += al16((size_t)st * n * 4);
    L.lu0 = o; o += al16((size_t)st * n * 4);
    L.lu1 = o; o += al16((size_t)st * n * 4);
    L.lu2 = o; o += al16((size_t)st * n * 4);
    L.llm = o; o += al16((size_t)st * n * 4);
    L.lpv = o; o += al16((size_t)st * n);
    L.yc = o; o += al16((size_t)chunk * n * 8);
    L.total = o;
    return L;
}

// Eigenpairs of T above t^2 and their back-transformation (see file header).
// IV_CHUNK eigenvectors are solved per inverse-iteration pass; their arrays
// are interleaved with the odd stride IV_ST (> IV_CHUNK) so that both the
// thread-per-vector solves and the warp-per-vector reductions avoid bank
// conflicts.
template <int IV_CHUNK, int IV_ST, int NT>
__global__ void __launch_bounds__(NT, (NT >= 512 ? 2 : 3)) k_eigvec(GroupSet gs, int mat_begin, EigArgs a) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char vsm[];
    __shared__ float red[4];
    __shared__ int s_r, s_cst, s_wend;
    __shared__ cf s_cm[EV_HB * EV_HB];    // C_ji of the current batch of reflectors
    __shared__ float s_dv[16 * 2 * EV_HB];  // per warp: the batch's dot products u_j^H y
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    pdl_release_dependents();
    if (is_frozen(g, mat, a.active)) return;
    wait_flag(flag_of(a.ready, g, mat), a.status, true);
    const int n = g.s;
    float *zs = a.zsave ? a.zsave + g.off + (long long)mat * n * g.len : nullptr;
    const bool allp = a.allp != 0 && zs != nullptr;
    const long long pk = (long long)n * (n + 1) / 2;
    const cf *Gglob = a.Gp + g.poff + (long long)mat * pk;     // Householder vectors
    const EvLayout LY = ev_layout(n, IV_CHUNK, IV_ST);
    cf *ph = (cf *)(vsm + LY.ph);
    float *dd = (float *)(vsm + LY.dd), *ff = (float *)(vsm + LY.ff), *f2 = (float *)(vsm + LY.f2);
    float *taus = (float *)(vsm + LY.taus), *lamv = (float *)(vsm + LY.lam);
    int *clu = (int *)(vsm + LY.clu);
    float *zv = (float *)(vsm + LY.zv), *lu0 = (float *)(vsm + LY.lu0), *lu1 = (float *)(vsm + LY.lu1);
    float *lu2 = (float *)(vsm + LY.lu2), *llm = (float *)(vsm + LY.llm);
    unsigned char *lpv = vsm + LY.lpv;
    cf *Yc = (cf *)(vsm + LY.yc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float t2 = allp ? -FLT_MAX : g.thresh * g.thresh;
    const float *td = tri_d(a, g, mat), *ttau = td + n;
    const cf *te = (const cf *)(td + 2 * n);
    float *lam_out = a.lam + g.soff + (long long)mat * n;
    cf *V = a.V + g.off + (long long)mat * n * g.len;
    int *rank_out = a.rank + g.moff + mat;
    tri_real_setup(td, ttau, te, n, dd, taus, ff, f2, ph, tid, lane, warp, NT);
    __syncthreads();
    if (warp == 0) {
        float gl = 0.f, gu = 0.f, pivmin = 0.f;
        if (lane == 0) gershgorin(dd, ff, f2, n, &gl, &gu, &pivmin);
        gl = __shfl_sync(0xffffffffu, gl, 0);
        gu = __shfl_sync(0xffffffffu, gu, 0);
        pivmin = __shfl_sync(0xffffffffu, pivmin, 0);
        // near-degenerate at the threshold: t^2 below the FP32 resolution floor
        // F = 32 eps_32 max(|gl|, |gu|) of the Gram eigenvalues, with eigenvalues between t^2
        // and F, so the count above t^2 is not determined in FP32 -> FP64 re-solve.  Lane 0
        // counts the eigenvalues below t^2 and lane 1 those below F, side by side.
        const float F = 32.f * FLT_EPSILON * fmaxf(fabsf(gl), fabsf(gu));
        int c = 0;
        if (lane < 2) {
            const float x = lane == 0 ? t2 : F;
            c = (x >= gu) ? n : sturm_lt(dd, f2, n, x, pivmin);
        }
        const int ct = __shfl_sync(0xffffffffu, c, 0), cF = __shfl_sync(0xffffffffu, c, 1);
        if (lane == 0) {
            red[0] = gl; red[1] = gu; red[2] = pivmin;
            int rr = allp ? n : n - ct;
            if (!allp && a.fp64_fallback && rr > 0 && t2 < F && n - cF != rr) rr = -1;
            s_r = rr;
        }
    }
    __syncthreads();
    const float gl = red[0], gu = red[1], pivmin = red[2];
    const float tnorm = fmaxf(fabsf(gl), fabsf(gu));
    const int r = s_r;
    if (tid == 0) {
        *rank_out = r;
        if (a.rank_acc && r > 0) a.rank_acc[g.moff + mat] += (unsigned long long)r;   // one CTA per matrix
    }
    if (r <= 0) {               // nothing above t^2, or flagged for the FP64 re-solve (r = -1)
        publish_flag(flag_of(a.vready, g, mat));
        return;
    }
    for (int q = warp; q < r; q += NW) {
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
    if (tid == 0) {
        const float ortol = 1e-3f * tnorm;
        const float sep = 10.f * FLT_EPSILON * tnorm;
        for (int q = 0; q < r; ++q) {
            if (q > 0 && lamv[q - 1] - lamv[q] < sep) lamv[q] = lamv[q - 1] - sep;
            clu[q] = (q == 0) || (lamv[q - 1] - lamv[q] > ortol) ? 1 : 0;
        }
    }
    __syncthreads();
    for (int q = tid; q < r; q += NT) lam_out[q] = lamv[q];
    for (int q0 = 0; q0 < r; q0 += IV_CHUNK) {
        const int qc = min(IV_CHUNK, r - q0);
        for (int idx = tid; idx < qc * n; idx += NT) {
            const int q = idx / n, i = idx - q * n;
            zv[i * IV_ST + q] = 1.f + 0.25f * (float)(((i * 7919 + (q0 + q) * 104729) % 997) - 498) / 498.f;
        }
        __syncthreads();
        if (allp && tid == 0) {
            // the cluster of vector q0 may have started in an earlier chunk: its members
            // there are [s_cst, q0), its members here [q0, q0 + s_wend)
            int c = q0;
            while (c > 0 && !clu[c]) --c;
            int w = 1;
            while (w < qc && !clu[q0 + w]) ++w;
            s_cst = c;
            s_wend = w;
        }
        __syncthreads();
        for (int it = 0; it < INV_ITERS; ++it) {
            if (tid < qc)
                tri_solve<IV_ST>(dd, ff, n, lamv[q0 + tid], zv + tid, lu0 + tid, lu1 + tid, lu2 + tid, llm + tid,
                                 lpv + tid, FLT_EPSILON * tnorm + pivmin, it == 0);
            __syncthreads();
            if (allp && s_cst < q0) {
                for (int w = warp; w < s_wend; w += NW) {
                    for (int pass = 0; pass < 2; ++pass) {
                        for (int o = s_cst; o < q0; ++o) {
                            const float *zo = zs + (long long)o * n;
                            float dot = 0.f;
                            for (int i = lane; i < n; i += 32) dot += zv[i * IV_ST + w] * zo[i];
                            dot = wsum(dot);
                            for (int i = lane; i < n; i += 32) zv[i * IV_ST + w] -= dot * zo[i];
                            __syncwarp();
                        }
                    }
                }
                __syncthreads();
            }
            for (int w = warp; w < qc; w += NW) {
                if (!(w == 0 || clu[q0 + w])) continue;
                int end = w + 1;
                while (end < qc && !clu[q0 + end]) ++end;
                for (int mbr = w; mbr < end; ++mbr) {
                    for (int o = w; o < mbr; ++o) {
                        float dot = 0.f;
                        for (int i = lane; i < n; i += 32) dot += zv[i * IV_ST + o] * zv[i * IV_ST + mbr];
                        dot = wsum(dot);
                        for (int i = lane; i < n; i += 32) zv[i * IV_ST + mbr] -= dot * zv[i * IV_ST + o];
                        __syncwarp();
                    }
                    float nrm = 0.f;
                    for (int i = lane; i < n; i += 32) nrm += zv[i * IV_ST + mbr] * zv[i * IV_ST + mbr];
                    nrm = wsum(nrm);
                    const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
                    for (int i = lane; i < n; i += 32) zv[i * IV_ST + mbr] *= inv;
                    __syncwarp();
                }
            }
            __syncthreads();
        }
        if (zs) {
            for (int idx = tid; idx < qc * n; idx += NT) {
                const int w = idx / n, i = idx - w * n;
                zs[(long long)(q0 + w) * n + i] = zv[i * IV_ST + w];
            }
        }
        // back-transformation y = Q P z, reflectors applied for k = n-3 .. 0 in batches of EV_HB
        for (int idx = tid; idx < qc * n; idx += NT) {
            const int w = idx / n, i = idx - w * n;
            Yc[idx] = cscale(ph[i], zv[i * IV_ST + w]);
        }
        __syncthreads();
        if (a.band) {
            // two-stage reduction: y <- Q2 y = S_0 (S_1 (... S_{n-3} y)), the reflectors of one
            // sweep (disjoint windows of at most SB_B rows) two at a time, one per half-warp.  The
            // reflectors are staged by groups of sweeps (from the last) into two buffers in the
            // inverse-iteration arrays (free from here on), the next group while one is applied.
            const cf *rec = a.sb + g.sboff + (long long)mat * sb_stride(n) + (long long)n * (SB_B + 1);
            cf *qb = (cf *)(vsm + LY.zv);
            const long long cap = (long long)((LY.yc - LY.zv) / 8) / 2 / (SB_B + 1);   // reflectors per buffer
            auto group_lo = [&](int jh) {
                int jl = jh;
                while (jl > 0 && sb_sweep_off(n, jh + 1) - sb_sweep_off(n, jl - 1) <= cap) --jl;
                return jl;
            };
            auto stage = [&](int jh, int jl, int bi) {
                const long long o0 = sb_sweep_off(n, jl) * (SB_B + 1), o1 = sb_sweep_off(n, jh + 1) * (SB_B + 1);
                cf *dst = qb + (long long)bi * cap * (SB_B + 1);
                for (long long e = tid; e < o1 - o0; e += NT) cp_async8(dst + e, rec + o0 + e, 8);
                cp_async_commit();
            };
            const int hw = lane >> 4, l = lane & (SB_B - 1);
            int jhi = n - 3, jlo = group_lo(jhi), buf = 0;
            stage(jhi, jlo, 0);
            while (jhi >= 0) {
                const int nh = jlo - 1, nl = nh >= 0 ? group_lo(nh) : 0;
                if (nh >= 0) stage(nh, nl, buf ^ 1);
                else cp_async_commit();
                cp_async_wait_1();
                __syncthreads();
                const cf *gb = qb + (long long)buf * cap * (SB_B + 1);
                const long long ob = sb_sweep_off(n, jlo);
                for (int w = warp; w < qc; w += NW) {
                    cf *y = Yc + (long long)w * n;
                    for (int j = jhi; j >= jlo; --j) {
                        const int K = sb_nsteps(n, j);
                        const cf *rj = gb + (sb_sweep_off(n, j) - ob) * (SB_B + 1);
                        for (int k0 = 0; k0 < K; k0 += 2) {
                            const int k = k0 + hw;
                            float tau = 0.f;
                            int row = n;
                            cf v = mk(0.f, 0.f);
                            if (k < K) {
                                const cf hd = rj[k * (SB_B + 1)];
                                tau = hd.x;
                                row = __float_as_int(hd.y) + l;
                                v = rj[k * (SB_B + 1) + 1 + l];
                            }
                            const bool on = tau != 0.f && row < n;
                            const cf yy = on ? y[row] : mk(0.f, 0.f);
                            float dr = v.x * yy.x + v.y * yy.y, di = v.x * yy.y - v.y * yy.x;
#pragma unroll
                            for (int o = SB_B / 2; o > 0; o >>= 1) {
                                dr += __shfl_xor_sync(0xffffffffu, dr, o);
                                di += __shfl_xor_sync(0xffffffffu, di, o);
                            }
                            dr *= tau;
                            di *= tau;
                            if (on) y[row] = mk(yy.x - (v.x * dr - v.y * di), yy.y - (v.x * di + v.y * dr));
                        }
                        __syncwarp();
                    }
                }
                __syncthreads();                             // this buffer is staged into next-but-one
                jhi = nh;
                jlo = nl;
                buf ^= 1;
            }
            cp_async_wait_all();
            __syncthreads();
        }
        // Reflectors are applied in batches of EV_HB, u_j = v_{kb-j} (j = 0 .. EV_HB-1, in the order
        // of application), staged in shared memory by absolute row (zero above the reflector's
        // first row, and wholly zero past reflector 0).  With d_j = u_j^H y and C_ji = u_j^H u_i,
        // applying them one after the other is
        //   s_j = d_j - sum_{i<j} tau_i C_ji s_i,   y <- y - sum_j tau_j u_j s_j,
        // so each vector needs one round of reductions per batch instead of one per reflector:
        // its 2 EV_HB dot-product sums are reduced over the lanes by one transpose-reduce and
        // exchanged through shared memory.  C (independent of y) is formed by all warps after
        // staging, two entries per warp and round with one 4-value transpose-reduce.  Batches
        // are staged nbuf - 1 ahead (nbuf = 3 buffers where they fit, else 2) in the
        // inverse-iteration arrays (free from here on: zv was copied to Yc above) with cp.async,
        // one commit group per batch index.
        static_assert(EV_HB == 8, "the batch's 2 EV_HB dot products per vector are reduced by treduce16");
        const size_t hb_elems = (size_t)EV_HB * n;
        const int nbuf = 3 * hb_elems * 8 <= LY.yc - LY.zv ? 3 : 2;
        cf *hbuf0 = (cf *)(vsm + LY.zv);
        // reflector of column k: rows >= k + hoff (1; SB_B for the panel reflectors of the
        // two-stage reduction, the last of which belongs to column n - 2 - SB_B)
        const int hoff = a.band ? SB_B : 1;
        const int kfirst = n - 2 - hoff;
        const int nbatch = kfirst >= 0 ? kfirst / EV_HB + 1 : 0;   // batch b: kb = kfirst - b EV_HB
        auto issue_batch = [&](int b) {
            if (b < nbatch) {
                const int kb = kfirst - b * EV_HB;
                cf *buf = hbuf0 + (long long)(b % nbuf) * hb_elems;
                for (int j = 0; j < EV_HB; ++j) {
                    const int k = kb - j;
                    for (int row = tid; row < n; row += NT) {
                        const bool ok = k >= 0 && row >= k + hoff;
                        cp_async8(buf + (long long)j * n + row, ok ? Gglob + colstart(k, n) + (row - k) : Gglob,
                                  ok ? 8 : 0);
                    }
                }
            }
            cp_async_commit();
        };
        for (int b = 0; b + 1 < nbuf; ++b) issue_batch(b);
        for (int b = 0; b < nbatch; ++b) {
            const int kb = kfirst - b * EV_HB;
            const int nbat = min(EV_HB, kb + 1);
            const int r0 = kb - nbat + 1 + hoff;             // first row any u_j of the batch touches
            const cf *hb = hbuf0 + (long long)(b % nbuf) * hb_elems;
            if (nbuf == 3) cp_async_wait_1();                // every group but the newest (batch b + 1)
            else cp_async_wait_all();
            __syncthreads();                                 // batch b staged; the buffer of b - 1 is free
            issue_batch(b + nbuf - 1);
            // C_ji = u_j^H u_i, i < j, over the rows of u_i (rows > kb - i)
            for (int pq0 = 2 * warp; pq0 < EV_HB * (EV_HB - 1) / 2; pq0 += 2 * NW) {   // warp-uniform
                float cv[4];
                int jj[2], ii[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    int j = 1, i = pq0 + e;
                    while (i >= j) { i -= j; ++j; }
                    jj[e] = j;
                    ii[e] = i;
                    float cr = 0.f, ci = 0.f;
                    if (pq0 + e < EV_HB * (EV_HB - 1) / 2) {
                        const cf *uj = hb + (long long)j * n, *ui = hb + (long long)i * n;
                        for (int row = kb - i + hoff + lane; row < n; row += 32) {
                            const cf x = uj[row], z = ui[row];
                            cr += x.x * z.x + x.y * z.y;
                            ci += x.x * z.y - x.y * z.x;
                        }
                    }
                    cv[2 * e] = cr;
                    cv[2 * e + 1] = ci;
                }
                const float s = treduce4(cv, lane);          // lane L: total of value (L >> 3) & 3
                if ((lane & 7) == 0) {
                    const int v = (lane >> 3) & 3, e = v >> 1;
                    if (pq0 + e < EV_HB * (EV_HB - 1) / 2)
                        ((float *)s_cm)[2 * ((e ? jj[1] : jj[0]) * EV_HB + (e ? ii[1] : ii[0])) + (v & 1)] = s;
                }
            }
            __syncthreads();
            for (int w = warp; w < qc; w += NW) {
                cf *y = Yc + (long long)w * n;
                float dv[2 * EV_HB], dr[EV_HB], di[EV_HB], tj[EV_HB];
#pragma unroll
                for (int j = 0; j < 2 * EV_HB; ++j) dv[j] = 0.f;
                for (int row = r0 + lane; row < n; row += 32) {
                    const cf yy = y[row];
#pragma unroll
                    for (int j = 0; j < EV_HB; ++j) {
                        const cf u = hb[(long long)j * n + row];
                        dv[2 * j] += u.x * yy.x + u.y * yy.y;
                        dv[2 * j + 1] += u.x * yy.y - u.y * yy.x;
                    }
                }
                const float sred = treduce16(dv, lane);      // lane L: total of value (L >> 1) & 15
                float *sd = s_dv + warp * 2 * EV_HB;
                if ((lane & 1) == 0) sd[(lane >> 1) & 15] = sred;
                __syncwarp();
#pragma unroll
                for (int j = 0; j < EV_HB; ++j) {
                    dr[j] = sd[2 * j];
                    di[j] = sd[2 * j + 1];
                    tj[j] = j < nbat ? taus[kb - j] : 0.f;
                }
                __syncwarp();
                // forward substitution (every lane), then dr, di <- tau_j s_j
#pragma unroll
                for (int j = 0; j < EV_HB; ++j) {
                    float sr = dr[j], si = di[j];
#pragma unroll
                    for (int i = 0; i < j; ++i) {
                        const cf c = s_cm[j * EV_HB + i];
                        sr -= c.x * dr[i] - c.y * di[i];
                        si -= c.x * di[i] + c.y * dr[i];
                    }
                    dr[j] = tj[j] * sr;
                    di[j] = tj[j] * si;
                }
                for (int row = r0 + lane; row < n; row += 32) {
                    float ar = 0.f, ai = 0.f;
#pragma unroll
                    for (int j = 0; j < EV_HB; ++j) {
                        const cf u = hb[(long long)j * n + row];
                        ar += u.x * dr[j] - u.y * di[j];
                        ai += u.x * di[j] + u.y * dr[j];
                    }
                    y[row] = mk(y[row].x - ar, y[row].y - ai);
                }
            }
        }
        __syncthreads();
        for (int idx = tid; idx < qc * n; idx += NT) {
            const int w = idx / n, i = idx - w * n;
            const cf y = Yc[idx];
            if (!isfinite(y.x) || !isfinite(y.y)) atomicOr(a.status, (unsigned)ST_NONFINITE);
            V[(long long)(q0 + w) * n + i] = y;
        }
        __syncthreads();
    }
    publish_flag(flag_of(a.vready, g, mat));
}

// ------------------------------------------------------------- resolvent
// Shared-memory layout of k_resolvent (16-byte aligned regions); QC pairs per
// pass give 2 QC complex right-hand sides and 4 QC real solves.
struct RsLayout {
    size_t ph, dd, ff, f2, taus, zr, lu0, lu1, lu2, llm, lpv, wc, total;
};
__host__ __device__ inline RsLayout rs_layout(int n, int qc) {
    const size_t st = 4 * (size_t)qc + 1;
    RsLayout L;
    size_t o = 0;
    L.ph = o; o += al16((size_t)n * 8);
    L.dd = o; o += al16((size_t)n * 4);
    L.ff = o; o += al16((size_t)n * 4);
    L.f2 = o; o += al16((size_t)n * 4);
    L.taus = o; o += al16((size_t)n * 4);
    L.zr = o; o += al16(st * n * 4);
    L.lu0 = o; o += al16(st * n * 4);
    L.lu1 = o; o += al16(st * n * 4);
    L.lu2 = o; o += al16(st * n * 4);
    L.llm = o; o += al16(st * n * 4);
    L.lpv = o; o += al16(st * n);
    L.wc = o; o += al16(2 * (size_t)qc * n * 8);
    L.total = o;
    return L;
}

// One warp applies the reflectors H_k = I - tau_k v_k v_k^H (v_k: entries k+1..n-1,
// stored below the diagonal of packed column k) to its own vector y (length n,
// shared memory), reading each reflector from global memory into registers (lane
// holds entries lane, lane + 32, ...) with the next one prefetched; no block
// barrier.  forward: Q^H y = H_{n-3} ... H_0 y (k ascending); otherwise
// Q y = H_0 ... H_{n-3} y (k descending).  n <= 32 * RS_MAXJ.
#define RS_MAXJ 15
__device__ void warp_reflectors(cf *y, int n, const cf *Gglob, const float *taus, bool forward, int lane) {
    const int kmax = n - 3;
    if (kmax < 0) return;
    cf cur[RS_MAXJ], nxt[RS_MAXJ];
    int k = forward ? 0 : kmax;
    {
        const int m = n - k - 1;
        const cf *hv = Gglob + colstart(k, n) + 1;
#pragma unroll
        for (int j = 0; j < RS_MAXJ; ++j) {
            const int i = lane + 32 * j;
            cur[j] = i < m ? hv[i] : mk(0.f, 0.f);
        }
    }
    for (int step = 0; step <= kmax; ++step) {
        const int kn = forward ? k + 1 : k - 1;
        if (step < kmax) {
            const int m = n - kn - 1;
            const cf *hv = Gglob + colstart(kn, n) + 1;
#pragma unroll
            for (int j = 0; j < RS_MAXJ; ++j) {
                const int i = lane + 32 * j;
                nxt[j] = i < m ? hv[i] : mk(0.f, 0.f);
            }
        }
        const float tau = taus[k];
        if (tau != 0.f) {
            const int m = n - k - 1;
            cf *yk = y + k + 1;
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int j = 0; j < RS_MAXJ; ++j) {
                const int i = lane + 32 * j;
                if (i < m) {
                    const cf v = cur[j], yy = yk[i];
                    sr += v.x * yy.x + v.y * yy.y;
                    si += v.x * yy.y - v.y * yy.x;
                }
            }
            sr = wsum(sr) * tau;
            si = wsum(si) * tau;
#pragma unroll
            for (int j = 0; j < RS_MAXJ; ++j) {
                const int i = lane + 32 * j;
                if (i < m) {
                    const cf v = cur[j];
                    yk[i].x -= v.x * sr - v.y * si;
                    yk[i].y -= v.x * si + v.y * sr;
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < RS_MAXJ; ++j) cur[j] = nxt[j];
        k = kn;
    }
}

// Remove from the complex vector y (shared memory, one warp) its components
// along the r real orthonormal vectors zs (global, row stride n).
__device__ void project_one(cf *y, int n, const float *zs, int r, int lane) {
    for (int k = 0; k < r; ++k) {
        const float *z = zs + (long long)k * n;
        float cr = 0.f, ci = 0.f;
        for (int i = lane; i < n; i += 32) {
            cr = fmaf(z[i], y[i].x, cr);
            ci = fmaf(z[i], y[i].y, ci);
        }
        cr = wsum(cr);
        ci = wsum(ci);
        for (int i = lane; i < n; i += 32) {
            y[i].x -= cr * z[i];
            y[i].y -= ci * z[i];
        }
        __syncwarp();
    }
}

template <int QC>
__global__ void __launch_bounds__(EIG_THREADS) k_resolvent(GroupSet gs, EigArgs a, const cf *W, cf *Y) {
    extern __shared__ __align__(16) unsigned char rsm[];
    __shared__ float red[4];
    constexpr int ST = 4 * QC + 1;
    int mat;
    const int gi = find_group(gs, blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int n = g.s;
    const int r = a.rank[g.moff + mat];
    if (r == 0) return;
    const RsLayout LY = rs_layout(n, QC);
    cf *ph = (cf *)(rsm + LY.ph);
    float *dd = (float *)(rsm + LY.dd), *ff = (float *)(rsm + LY.ff), *f2 = (float *)(rsm + LY.f2);
    float *taus = (float *)(rsm + LY.taus), *zr = (float *)(rsm + LY.zr);
    float *lu0 = (float *)(rsm + LY.lu0), *lu1 = (float *)(rsm + LY.lu1), *lu2 = (float *)(rsm + LY.lu2);
    float *llm = (float *)(rsm + LY.llm);
    unsigned char *lpv = rsm + LY.lpv;
    cf *wc = (cf *)(rsm + LY.wc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long pk = (long long)n * (n + 1) / 2;
    const cf *Gglob = a.Gp + g.poff + (long long)mat * pk;
    const float *td = tri_d(a, g, mat), *ttau = td + n;
    const cf *te = (const cf *)(td + 2 * n);
    const float *lam = a.lam + g.soff + (long long)mat * n;
    const float *zs = a.zsave + g.off + (long long)mat * n * g.len;
    const long long wbase = 2 * (g.off + (long long)mat * n * g.len);
    tri_real_setup(td, ttau, te, n, dd, taus, ff, f2, ph, tid, lane, warp);
    __syncthreads();
    if (tid == 0) {
        float gl, gu, pivmin;
        gershgorin(dd, ff, f2, n, &gl, &gu, &pivmin);
        red[0] = FLT_EPSILON * fmaxf(fabsf(gl), fabsf(gu)) + pivmin;
    }
    __syncthreads();
    const float tiny = red[0];
    for (int q0 = 0; q0 < r; q0 += QC) {
        const int qc = min(QC, r - q0), nv = 2 * qc;
        for (int idx = tid; idx < nv * n; idx += EIG_THREADS) wc[idx] = W[wbase + (long long)2 * q0 * n + idx];
        __syncthreads();
        // each warp maps its own right-hand side to the tridiagonal basis: P^H Q^H w, projected
        for (int w = warp; w < nv; w += EIG_WARPS) {
            cf *y = wc + (long long)w * n;
            warp_reflectors(y, n, Gglob, taus, true, lane);
            for (int i = lane; i < n; i += 32) y[i] = cmulc(ph[i], y[i]);
            __syncwarp();
            project_one(y, n, zs, r, lane);
            for (int i = lane; i < n; i += 32) {
                zr[i * ST + 2 * w] = y[i].x;
                zr[i * ST + 2 * w + 1] = y[i].y;
            }
        }
        __syncthreads();
        if (tid < 2 * nv)       // real system tid: pair q0 + tid / 4, right-hand side (tid / 2) % 2, re / im
            tri_solve<ST>(dd, ff, n, lam[q0 + tid / 4], zr + tid, lu0 + tid, lu1 + tid, lu2 + tid, llm + tid,
                          lpv + tid, tiny, true);
        __syncthreads();
        for (int w = warp; w < nv; w += EIG_WARPS) {
            cf *y = wc + (long long)w * n;
            // (lambda I - T_r)^{-1} = -(T_r - lambda I)^{-1}
            for (int i = lane; i < n; i += 32) y[i] = mk(-zr[i * ST + 2 * w], -zr[i * ST + 2 * w + 1]);
            __syncwarp();
            project_one(y, n, zs, r, lane);
            for (int i = lane; i < n; i += 32) y[i] = cmul(ph[i], y[i]);
            __syncwarp();
            warp_reflectors(y, n, Gglob, taus, false, lane);
            bool bad = false;
            for (int i = lane; i < n; i += 32) {
                const cf v = y[i];
                if (!isfinite(v.x) || !isfinite(v.y)) bad = true;
                Y[wbase + (long long)(2 * q0 + w) * n + i] = v;
            }
            if (bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- apply
// k_apply_stream: the apply for matrices with r <= AS_CH pairs above t^2 (the
// usual case on the lifted matrices).  CTA = (matrix, tile of AS_ET rows of B);
// phase 1: Y[e][k] = h_k sum_c B[e][c] v_k[c], lane = e; for r <= AS_SMALL the warps
// split the rows c (partial sums reduced in a fixed order), otherwise they split the
// pairs k (one writer per entry), so the result is bitwise reproducible;
// phase 1 loads AS_P1B rows of B together (memory parallelism at 3 CTAs per SM);
// phase 2: Z[e][c] = sum_k Y[e][k] conj(v_k[c]) streamed over c with the
// epilogue (Z out, or D and E update) fused, B re-read from L1/L2.  No large
// per-thread arrays, so occupancy (and with it memory parallelism) is high.
#define AS_ET 32
#define AS_CH 64          // pairs handled by the streaming apply (variants for r <= 32 and 32 < r <= 64)
#define AS_SMALL 8        // up to this many pairs phase 1 splits the rows of B over the warps
#define AS_THREADS 256
#define AS_P1B 8          // rows of B loaded together in phase 1
// CH = 32: four CTAs per SM (at most 64 registers), more loads in flight per SM than the three
// that 80 registers allow (0.437 against 0.464 ms per apply stage on the 12-coil 256x256
// workload); CH = 64 keeps its registers (its eight accumulators per thread would spill)
template <int CH>
__global__ void __launch_bounds__(AS_THREADS, CH <= 32 ? 4 : 3)
    k_apply_stream(GroupSet gs, int mat_begin, EigArgs ea, SvtArgs a) {
    extern __shared__ cf ssm[];
    __shared__ float gcoef[CH];
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    pdl_release_dependents();
    if (is_frozen(g, mat, a.active)) return;
    const int n = g.s, len = g.len;
    const int e0 = blockIdx.y * AS_ET;
    if (e0 >= len) return;
    wait_flag(flag_of(ea.vready, g, mat), a.status, false);
    const int r = ea.rank[g.moff + mat];
    if (r < 0 || r > CH || (CH > 32 && r <= CH / 2)) return;   // FP64 re-solve / other variant / k_apply_eig
    const long long mb = g.off + (long long)mat * n * len;
    if (blockIdx.y == 0 && threadIdx.x == 0 && a.rank_out) a.rank_out[g.moff + mat] = r;
    const float t = g.thresh;
    cf *Ys = ssm;                          // [AS_ET][CH + 1]
    cf *P = Ys + AS_ET * (CH + 1);      // [warps][AS_ET][AS_SMALL + 1] partials (r <= AS_SMALL)
    const cf *__restrict__ Vs = ea.V + mb; // eigenvectors (rows), read through L1
    const float *lam = ea.lam + g.soff + (long long)mat * n;
    const int tid = threadIdx.x, e = tid & 31, w = tid >> 5;
    constexpr int NWS = AS_THREADS / 32;
    if (tid < r) {
        const float sg = sqrtf(fmaxf(lam[tid], 0.f));
        gcoef[tid] = sg > t ? 1.f - t / sg : 0.f;
    }
    const bool ein = e0 + e < len;
    const cf *Bcol = a.B0 + mb + e0 + e;
    if (r <= AS_SMALL) {
        // few pairs: warp w takes a slice of the rows c for every pair; fixed-order reduction
        const int c0 = (n * w) / NWS, c1 = (n * (w + 1)) / NWS;
        float yr[AS_SMALL], yi[AS_SMALL];
#pragma unroll
        for (int k = 0; k < AS_SMALL; ++k) yr[k] = yi[k] = 0.f;
        if (ein) {
            for (int cb = c0; cb < c1; cb += AS_P1B) {
                cf bb[AS_P1B];                     // AS_P1B rows of B in flight together
#pragma unroll
                for (int u = 0; u < AS_P1B; ++u) bb[u] = cb + u < c1 ? Bcol[(long long)(cb + u) * len] : mk(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < AS_P1B; ++u) {
                    if (cb + u < c1) {
                        const cf b = bb[u];
#pragma unroll
                        for (int k = 0; k < AS_SMALL; ++k) {
                            if (k < r) {
                                const cf v = Vs[(long long)k * n + cb + u];
                                yr[k] = fmaf(b.x, v.x, fmaf(-b.y, v.y, yr[k]));
                                yi[k] = fmaf(b.x, v.y, fmaf(b.y, v.x, yi[k]));
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < AS_SMALL; ++k)
            if (k < r) P[((long long)w * AS_ET + e) * (AS_SMALL + 1) + k] = mk(yr[k], yi[k]);
        __syncthreads();
        for (int idx = tid; idx < AS_ET * r; idx += AS_THREADS) {
            const int ee = idx / r, k = idx - ee * r;
            float sr = 0.f, si = 0.f;
            for (int ww = 0; ww < NWS; ++ww) {
                const cf pv = P[((long long)ww * AS_ET + ee) * (AS_SMALL + 1) + k];
                sr += pv.x;
                si += pv.y;
            }
            Ys[ee * (CH + 1) + k] = mk(gcoef[k] * sr, gcoef[k] * si);
        }
    } else {
        // more pairs: warp w takes pairs w, w + 8, ... over all rows; one writer per entry
        __syncthreads();                   // gcoef
        constexpr int KPW = CH / NWS;
        float yr[KPW], yi[KPW];
#pragma unroll
        for (int u = 0; u < KPW; ++u) yr[u] = yi[u] = 0.f;
        if (ein) {
            for (int cb = 0; cb < n; cb += AS_P1B) {
                cf bb[AS_P1B];
#pragma unroll
                for (int u = 0; u < AS_P1B; ++u) bb[u] = cb + u < n ? Bcol[(long long)(cb + u) * len] : mk(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < AS_P1B; ++u) {
                    if (cb + u < n) {
                        const cf b = bb[u];
#pragma unroll
                        for (int q = 0; q < KPW; ++q) {
                            const int k = w + NWS * q;
                            if (k < r) {
                                const cf v = Vs[(long long)k * n + cb + u];
                                yr[q] = fmaf(b.x, v.x, fmaf(-b.y, v.y, yr[q]));
                                yi[q] = fmaf(b.x, v.y, fmaf(b.y, v.x, yi[q]));
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < KPW; ++u) {
            const int k = w + NWS * u;
            if (k < r) Ys[e * (CH + 1) + k] = mk(gcoef[k] * yr[u], gcoef[k] * yi[u]);
        }
    }
    __syncthreads();
    if (!ein) return;
    const float ib = 1.f / a.beta;
    const cf *ye = Ys + e * (CH + 1);
    // Z columns c = w, w + 8, ...; batches of AS_B rows so that their loads are in flight together
    constexpr int AS_B = 4;
    const cf *__restrict__ B0 = a.B0;
    cf *__restrict__ Dp = a.D;
    cf *__restrict__ Ep = a.E;
    for (int cb = w; cb < n; cb += AS_B * NWS) {
        cf Av[AS_B], Dv[AS_B];
        float zr[AS_B], zi[AS_B];
#pragma unroll
        for (int u = 0; u < AS_B; ++u) {
            const int c = cb + u * NWS;
            const long long vi = mb + (long long)c * len + e0 + e;
            if (c < n && a.mode != 0) {
                Av[u] = B0[vi];
                Dv[u] = Dp[vi];
            }
            zr[u] = 0.f;
            zi[u] = 0.f;
        }
        for (int k = 0; k < r; ++k) {
            const cf y = ye[k];
#pragma unroll
            for (int u = 0; u < AS_B; ++u) {
                const int c = cb + u * NWS;
                if (c < n) {
                    const cf v = Vs[(long long)k * n + c];
                    zr[u] = fmaf(y.x, v.x, fmaf(y.y, v.y, zr[u]));
                    zi[u] = fmaf(y.y, v.x, fmaf(-y.x, v.y, zi[u]));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < AS_B; ++u) {
            const int c = cb + u * NWS;
            if (c >= n) continue;
            const long long vi = mb + (long long)c * len + e0 + e;
            if (a.mode == 0) {
                if (a.z_natural) {
                    const int rr = g.trans ? c : e0 + e, cc = g.trans ? e0 + e : c;
                    a.Zout[mb + (long long)rr * g.cols + cc] = mk(zr[u], zi[u]);
                } else {
                    a.Zout[vi] = mk(zr[u], zi[u]);
                }
            } else {
                const cf A = Av[u], D = Dv[u];
                const cf Dn = mk(D.x + a.tau * (A.x - D.x * ib - zr[u]), D.y + a.tau * (A.y - D.y * ib - zi[u]));
                // streaming stores: D and E are not read again in this launch, so they should not
                // evict B, whose rows the epilogue reads a second time
                __stcs(reinterpret_cast<float2 *>(Dp + vi), make_float2(Dn.x, Dn.y));
                __stcs(reinterpret_cast<float2 *>(Ep + vi), make_float2(zr[u] - Dn.x * ib, zi[u] - Dn.y * ib));
            }
        }
    }
}

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
    wait_flag(flag_of(ea.vready, g, mat), a.status, false);
    const int et = min(AP_ET, len - e0);
    const long long mb = g.off + (long long)mat * n * len;
    const int r = ea.rank[g.moff + mat];
    if (r <= AS_CH) return;                // k_apply_stream handled it
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
// The hand-off wait of the launch chain on a flag set (or never set) by the host.
__global__ void k_wait_selftest(unsigned *flag, unsigned *status, unsigned long long limit_ns) {
    wait_flag(flag, status, true, limit_ns);
}

cudaError_t launch_wait_selftest(unsigned *flag, unsigned *status, unsigned long long limit_ns, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(flag, status, limit_ns);
    return cudaGetLastError();
}

static int g_eig_smem_max = 0;

cudaError_t eig_init_attributes() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    g_eig_smem_max = optin - 2048;
    const int mx = g_eig_smem_max;
    e = cudaSuccess;
#define TRI_ATTR(R, H)                                                                                      \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tridiag<R, H, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tridiag<R, H, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    TRI_ATTR(1, false) TRI_ATTR(2, false) TRI_ATTR(4, false) TRI_ATTR(6, false) TRI_ATTR(7, false) TRI_ATTR(8, true)
#undef TRI_ATTR
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tridiag_g, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sb1, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sb2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb2_smem(SB_NMAX));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_eigvec<16, 17, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_eigvec<8, 9, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resolvent<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resolvent<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_apply_stream<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, g_eig_smem_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply_stream<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, g_eig_smem_max);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_apply_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, g_eig_smem_max);
}

static size_t tridiag_smem(int n) {
    return al16((size_t)n * (n + 1) / 2 * 8) + (size_t)(EIG_WARPS + 4) * n * 8 + (size_t)n * 4 + 16;
}
static size_t tridiag_g_smem(int n) { return 2 * (size_t)n * 8 + (size_t)n * 4 + 16; }
static int ev_chunk(int nmax) { return nmax <= 352 ? 16 : 8; }

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

template <int RPL, bool HYB>
static cudaError_t tridiag_launch(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, size_t smem,
                                  cudaStream_t st) {
    bool full = true;                  // every order equals 32 * RPL: no bound checks against n
    for (int k = 0; k < gs.n; ++k) full = full && gs.g[k].s == 32 * RPL;
    const bool pdl = ea.gready != nullptr;
    if (full)
        return launch_ex(pdl, k_tridiag<RPL, HYB, true>, dim3(mat_count), dim3(EIG_THREADS), smem, st, gs, mat_begin,
                         ea, (int)smem);
    return launch_ex(pdl, k_tridiag<RPL, HYB, false>, dim3(mat_count), dim3(EIG_THREADS), smem, st, gs, mat_begin, ea,
                     (int)smem);
}

cudaError_t launch_heig(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    if (g_eig_smem_max == 0) return cudaErrorNotReady;
    int nmax = 0;
    for (int k = 0; k < gs.n; ++k) nmax = max(nmax, gs.g[k].s);
    // shared memory of the eigenvector kernel, checked before anything is launched (a
    // reduction whose ready flags no k_eigvec consumes would leave them set)
    int chunk = ea.ev_chunk == 8 || ea.ev_chunk == 16 ? ea.ev_chunk : ev_chunk(nmax);
    if (chunk == 16 && nmax > 352) chunk = 8;         // the 16-vector layout exceeds shared memory
    size_t ev_smem = 0;
    for (int k = 0; k < gs.n; ++k) ev_smem = max(ev_smem, ev_layout(gs.g[k].s, chunk, chunk + 1).total);
    if (ev_smem > (size_t)g_eig_smem_max) return cudaErrorInvalidValue;
    // 1. tridiagonalisation (a programmatic dependent of k_gram_tc when ea.gready is set):
    // two-stage where every order allows it, scratch is given, the eigenpairs above t^2 are
    // all that is wanted (the reverse mode's resolvent solves use the one-stage reflectors)
    // and the flags of the launch chain are complete
    bool two = ea.sb != nullptr && ea.reduction != 1 && ea.zsave == nullptr && !ea.allp &&
               (ea.ready == nullptr || ea.bready != nullptr) && sb1_layout(nmax).total <= (size_t)g_eig_smem_max;
    int nmin = nmax;
    for (int k = 0; k < gs.n; ++k) {
        two = two && sb_eligible(gs.g[k].s) && gs.g[k].sboff >= 0;
        nmin = min(nmin, gs.g[k].s);
    }
    if (ea.reduction == 0) two = two && nmin >= SB_AUTO_MIN;
    EigArgs eb = ea;
    eb.band = two ? SB_B : 0;
    cudaError_t e;
    if (two) {
        e = launch_ex(ea.gready != nullptr, k_sb1, dim3(mat_count), dim3(SB1_THREADS), sb1_layout(nmax).total, st, gs,
                      mat_begin, eb);
        if (e == cudaSuccess)
            e = launch_ex(ea.ready != nullptr, k_sb2, dim3(mat_count), dim3(SB2_THREADS), sb2_smem(nmax), st, gs,
                          mat_begin, eb);
    } else if (nmax <= EIG_SMEM_MAX_N) {
        const size_t smem = tridiag_smem(nmax);
        if (smem > (size_t)g_eig_smem_max) return cudaErrorInvalidValue;
        if (nmax <= 32) e = tridiag_launch<1, false>(gs, mat_begin, mat_count, ea, smem, st);
        else if (nmax <= 64) e = tridiag_launch<2, false>(gs, mat_begin, mat_count, ea, smem, st);
        else if (nmax <= 128) e = tridiag_launch<4, false>(gs, mat_begin, mat_count, ea, smem, st);
        else if (nmax <= 192) e = tridiag_launch<6, false>(gs, mat_begin, mat_count, ea, smem, st);
        else e = tridiag_launch<7, false>(gs, mat_begin, mat_count, ea, smem, st);
    } else if (nmax <= 256) {
        // the first columns of the packed matrix stay in global memory (L2), the rest in smem
        e = tridiag_launch<8, true>(gs, mat_begin, mat_count, ea, (size_t)g_eig_smem_max, st);
    } else {
        e = launch_ex(ea.gready != nullptr, k_tridiag_g, dim3(mat_count), dim3(EIG_THREADS), tridiag_g_smem(nmax), st,
                      gs, mat_begin, ea);
    }
    if (e != cudaSuccess) return e;
    // 2. eigenpairs above t^2 and back-transformation; chunk 16: 512 threads; chunk 8: 256
    // threads (smaller CTAs, more matrices in flight per SM).  With ready flags the launch is
    // a programmatic dependent of the reduction.
    const bool pdl = ea.ready != nullptr;
    if (chunk == 16)
        return launch_ex(pdl, k_eigvec<16, 17, 512>, dim3(mat_count), dim3(512), ev_smem, st, gs, mat_begin, eb);
    return launch_ex(pdl, k_eigvec<8, 9, 256>, dim3(mat_count), dim3(256), ev_smem, st, gs, mat_begin, eb);
}

cudaError_t launch_apply_eig(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, const SvtArgs &a,
                             cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    if (g_eig_smem_max == 0) return cudaErrorNotReady;
    int maxlen = 0, maxn = 0;
    for (int k = 0; k < gs.n; ++k) { maxlen = max(maxlen, gs.g[k].len); maxn = max(maxn, gs.g[k].s); }
    if (maxn > 512) return cudaErrorInvalidValue;
    // matrices with at most AS_CH pairs above t^2: streaming kernel; the others: k_apply_eig
    const size_t smem32 = sizeof(cf) * ((size_t)AS_ET * (32 + 1) + (size_t)(AS_THREADS / 32) * AS_ET * (AS_SMALL + 1));
    const size_t smem64 = sizeof(cf) * ((size_t)AS_ET * (64 + 1) + (size_t)(AS_THREADS / 32) * AS_ET * (AS_SMALL + 1));
    dim3 grid_s(mat_count, (maxlen + AS_ET - 1) / AS_ET);
    // a programmatic dependent of k_eigvec when ea.vready is set
    cudaError_t e0 = launch_ex(ea.vready != nullptr, k_apply_stream<32>, grid_s, dim3(AS_THREADS), smem32, st, gs,
                               mat_begin, ea, a);
    if (e0 != cudaSuccess) return e0;
    k_apply_stream<64><<<grid_s, AS_THREADS, smem64, st>>>(gs, mat_begin, ea, a);
    e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    const size_t smem = sizeof(cf) * ((size_t)maxn * AP_ET + (size_t)AP_CH * maxn + AP_ET * AP_CH);
    dim3 grid(mat_count, (maxlen + AP_ET - 1) / AP_ET);
    k_apply_eig<<<grid, AP_THREADS, smem, st>>>(gs, mat_begin, ea, a);
    return cudaGetLastError();
}

cudaError_t launch_resolvent(const GroupSet &gs, int mat_count, const EigArgs &ea, const cf *W, cf *Y,
                             cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    if (g_eig_smem_max == 0) return cudaErrorNotReady;
    int nmax = 0;
    for (int k = 0; k < gs.n; ++k) nmax = max(nmax, gs.g[k].s);
    const int qc = nmax <= 256 ? 4 : 2;
    size_t smem = 0;
    for (int k = 0; k < gs.n; ++k) smem = max(smem, rs_layout(gs.g[k].s, qc).total);
    if (smem > (size_t)g_eig_smem_max) return cudaErrorInvalidValue;
    if (qc == 4) k_resolvent<4><<<mat_count, EIG_THREADS, smem, st>>>(gs, ea, W, Y);
    else k_resolvent<2><<<mat_count, EIG_THREADS, smem, st>>>(gs, ea, W, Y);
    return cudaGetLastError();
}
