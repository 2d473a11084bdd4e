// Internal declarations shared by the translation units of libselr.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/selr.h"

// NVTX range for the lifetime of a scope (host side: API calls and the issue of each ADMM
// stage, recorded once while a graph is captured); header-only NVTX, inert without a tool.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------- complex
struct __align__(8) cf {
    float x, y;
};

__host__ __device__ __forceinline__ cf mk(float a, float b) { cf r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ cf cadd(cf a, cf b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cf csub(cf a, cf b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cf cmul(cf a, cf b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__host__ __device__ __forceinline__ cf cmulc(cf a, cf b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__host__ __device__ __forceinline__ cf cconj(cf a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ cf cscale(cf a, float s) { return mk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float cabs2(cf a) { return a.x * a.x + a.y * a.y; }

// --------------------------------------------------------------- lift groups
enum { G_ROW = 0, G_COL = 1, G_PE = 2, G_PARAM = 3 };
#define SELR_MAX_INST 32                     // instances of one batched plan (2D models)
#define SELR_MAX_GROUPS (2 * SELR_MAX_INST)  // lift families: two per instance

// One family of lifted matrices (all rows, all columns, all PE or all
// parameter lifts).  A matrix is rows x cols = (nv - p + 1) x (C * p).
// Internal storage of lifted arrays is "vector-major": the s vectors of the
// shorter side, each of length len, contiguous.  trans = 0: vectors are the
// columns of A (cols <= rows); trans = 1: vectors are the rows of A.
struct Group {
    int kind;
    int nmat;
    int nv, p, J, C, vc;
    int rows, cols;
    int trans;
    int s, len;
    float thresh;          // SVT threshold of this family
    int dlen;              // Jacobi: inner products over the first dlen entries only (0: len)
    int M, N, L;           // array dims of the source / adjoint arrays
    long long off;         // element offset of matrix 0 in lifted workspaces
    long long soff;        // offset of matrix 0 in per-vector arrays (sigma)
    long long poff;        // offset of matrix 0 in packed Gram storage (s (s+1) / 2 per matrix)
    int moff;              // index of matrix 0 among all matrices (status words)
    long long sboff;       // offset of matrix 0 in the two-stage reduction scratch, -1: no
                           // scratch (order outside [SB_NMIN, SB_NMAX])
    int inst;              // instance of a batched plan the family belongs to
    int aoff;              // offset of the instance's FE positions in the activity flags
    const cf *w;           // weights (length nv) or nullptr (identity)
    const cf *src;         // lift source array
    cf *dst;               // adjoint destination array
};

struct GroupSet {
    int n;
    int total;                       // total matrices
    long long sb_total;              // elements of two-stage reduction scratch the set needs
    int start[SELR_MAX_GROUPS + 1];  // prefix sums of nmat
    Group g[SELR_MAX_GROUPS];
};

__device__ __forceinline__ int find_group(const GroupSet &gs, int mat_global, int *local) {
    int lo = 0, hi = gs.n - 1;           // last group whose start <= mat_global
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mat_global >= gs.start[mid]) lo = mid;
        else hi = mid - 1;
    }
    *local = mat_global - gs.start[lo];
    return lo;
}

// Address of element `pos` of the vector of coil j belonging to matrix `mat`.
__device__ __forceinline__ long long src_index(const Group &g, int mat, int j, int pos) {
    const long long M = g.M, N = g.N;
    switch (g.kind) {
        case G_ROW:   return ((long long)j * M + mat) * N + pos;                 // [J][M][N], row m = mat
        case G_COL:   return ((long long)j * M + pos) * N + mat;                 // column n = mat
        case G_PE: {  int m = mat / g.L, l = mat % g.L;                          // (m, l), along n
                      return (((long long)l * g.J + j) * M + m) * N + pos; }
        default: {    int m = mat / g.N, n = mat % g.N;                          // (m, n), along l
                      return (((long long)pos * g.J + j) * M + m) * N + n; }
    }
}

// Element (r, c) of matrix `mat` in vector-major storage (relative to group).
__device__ __forceinline__ long long vm_index(const Group &g, int mat, int r, int c) {
    const long long base = (long long)mat * g.s * g.len;
    return g.trans ? base + (long long)r * g.len + c : base + (long long)c * g.len + r;
}

// Lifted value lift(x)[mat][r][c] (Eq. 2 / Eq. 4 / Eq. 7).
__device__ __forceinline__ cf lift_value(const Group &g, int mat, int r, int c) {
    const int ch = c / g.p, q = c - ch * g.p, pos = r + q;
    cf v;
    if (ch < g.J) {
        v = g.src[src_index(g, mat, ch, pos)];
    } else {
        v = cconj(g.src[src_index(g, mat, ch - g.J, g.nv - 1 - pos)]);
    }
    if (g.w) v = cmul(g.w[pos], v);
    return v;
}

// ---------------------------------------------------------- status words
enum { ST_NOCONV = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

// --------------------------------------------------------------- launchers
// fft.cu
struct FftTable {
    int n;
    int nst;
    int radix[24];
    const cf *tw;   // tw[k] = exp(-2 pi i k / n), k < n
};
cudaError_t fft_table_build(int n, FftTable *t, cf **tw_dev);
cudaError_t fft_init_attributes();
// Transform along dim of [outer][n][inner] (element (o,k,i) at (o*n+k)*inner+i).
cudaError_t launch_fft(const cf *in, cf *out, const FftTable &t, long long outer, long long inner,
                       int inverse, cudaStream_t st);

// lift.cu
// mode 0: write natural layout [mat][rows][cols]; mode 1: vector-major (also copy to out2 if non-null)
cudaError_t launch_lift(const GroupSet &gs, int gfirst, int mat_begin, int mat_count, const cf *D,
                        int d_natural, float inv_beta, cf *out, cf *out2, int out_natural,
                        const int *active, cudaStream_t st);
cudaError_t launch_adjoint(const GroupSet &gs, int gfirst, int mat_begin, int mat_count,
                           const cf *E, int e_natural, cudaStream_t st);
cudaError_t launch_natural_to_vm(const GroupSet &gs, const cf *A, cf *out, cf *out2, cudaStream_t st);
cudaError_t launch_vm_to_natural(const GroupSet &gs, const cf *in, cf *A, cudaStream_t st);

// svt.cu
struct SvtArgs {
    cf *W;               // vector-major working copy (orthogonalised in place)
    const cf *B0;        // vector-major original matrices
    float *sigma;        // per-vector singular values
    int *mat_status;     // per-matrix sweeps used (negative = not converged)
    unsigned *status;    // plan status word (ST_* bits)
    int max_sweeps;
    float tol;
    // apply epilogue
    int mode;            // 0: write Z (natural if z_natural, else vector-major) ; 1: ADMM D/E update
    cf *Zout; int z_natural;
    cf *D; cf *E;        // vector-major
    float beta, tau;
    int *rank_out;
    const int *active;   // per-FE-position activity (parameter models) or nullptr
};
cudaError_t svt_init_attributes();
cudaError_t launch_jacobi(const GroupSet &gs, int mat_begin, int mat_count, const SvtArgs &a, cudaStream_t st);
cudaError_t launch_svt_apply(const GroupSet &gs, int mat_begin, int mat_count, const SvtArgs &a, cudaStream_t st);

// ----------------------------------------------------- kernel hand-offs
// The eigensolver's kernels run as a chain of programmatic dependent launches:
// k_gram_tc -> k_tridiag -> k_eigvec -> k_apply_stream.  Each kernel of the
// chain releases its dependents as soon as a CTA starts, so the next kernel's
// CTAs start on the SMs that the last, partial wave of the previous one leaves
// idle (512 matrices are 3.4 waves of k_tridiag on 152 SMs).  Per matrix and
// hand-off there is a ready flag: the producing CTA publishes it (release)
// after its last write, the consuming CTAs wait for it (acquire, bounded) before
// their first read.  The wait always ends, because dependents are only
// scheduled once every CTA of the producing kernel is resident.  Flags read by
// one CTA per matrix are cleared by that CTA as it consumes them.  The
// k_eigvec -> apply flags are read by every row tile of a matrix, so no
// consumer can clear them; k_tridiag clears them instead, and it does so
// BEFORE its griddepcontrol.launch_dependents (store, fence, block barrier,
// then the trigger).  k_eigvec is scheduled only after every k_tridiag CTA has
// triggered, and the apply only after every k_eigvec CTA has, so by the time
// any apply tile polls, the flag of the previous call is gone and only this
// call's k_eigvec can set it again.  (Clearing it after the trigger, as an
// earlier version did, let an apply tile see the previous call's flag while
// k_tridiag was still waiting for the tensor-core Gram, and use stale ranks
// and eigenvectors.)  k_tridiag itself starts after the previous call's apply
// kernels have completed: the chain's first kernel is an ordinary launch.
#define READY_WAIT_NS 2000000000ull

__device__ __forceinline__ unsigned long long eig_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void pdl_release_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// End of a producing CTA: every thread's writes, then the flag (if any).
__device__ __forceinline__ void publish_flag(unsigned *f) {
    if (!f) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(f), "r"(1u) : "memory");
    }
}

// Start of a CTA whose dependents poll `f`: clear it and make the store visible
// at GPU scope before any thread of the CTA executes the programmatic trigger.
__device__ __forceinline__ void clear_flag_before_release(unsigned *f) {
    if (f && threadIdx.x == 0) {
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(f), "r"(0u) : "memory");
        __threadfence();
    }
    __syncthreads();
}

// Start of a consuming CTA: wait (at most limit_ns, then ST_TIMEOUT) for the
// flag, optionally clear it.
__device__ __forceinline__ void wait_flag(unsigned *f, unsigned *status, bool clear,
                                          unsigned long long limit_ns = READY_WAIT_NS) {
    if (!f) return;
    if (threadIdx.x == 0) {
        const unsigned long long t0 = eig_globaltimer();
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
            if (v != 0u) break;
            if (eig_globaltimer() - t0 > limit_ns) {
                atomicOr(status, (unsigned)ST_TIMEOUT);
                break;
            }
            __nanosleep(256);
        }
        if (clear) *f = 0u;
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned *flag_of(unsigned *base, const Group &g, int mat) {
    return base ? base + g.moff + mat : nullptr;
}

// Launch with (pdl) or without programmatic stream serialization on the previous kernel.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_ex(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// One CTA of wait_flag on `flag` with the given limit (failure-handling self-test).
cudaError_t launch_wait_selftest(unsigned *flag, unsigned *status, unsigned long long limit_ns, cudaStream_t st);

// gram_tc.cu: G = B^H B on tcgen05 tensor cores, mode 1 = TF32, mode 3 = 3xTF32 (s <= 256)
bool gram_tc_fits(const Group &g);
// ready (or null): per-matrix flags published for a programmatically dependent k_tridiag.
cudaError_t launch_gram_tc(const GroupSet &gs, int mat_begin, int mat_count, const cf *B0, cf *Gp,
                           const int *active, int mode, unsigned *status, unsigned *ready, cudaStream_t st);

// svt_small.cu: warp-per-matrix Jacobi SVT for s <= 8, len <= 64 (same SvtArgs epilogue)
bool svt_small_fits(const Group &g);
cudaError_t launch_svt_small(const GroupSet &gs, int mat_begin, int mat_count, const SvtArgs &a, cudaStream_t st);

// svt_eig.cu
// Two-stage Householder reduction (svt_eig.cu): G -> Hermitian band of half-bandwidth SB_B
// (blocked panels, k_sb1) -> tridiagonal (bulge chasing, k_sb2), for orders in
// [SB_NMIN, SB_NMAX].  Per matrix the scratch holds the band ([n][SB_B + 1]) and the
// bulge-chasing reflectors, sweep-major: sweep j (j = 0 .. n-3) has sb_nsteps(n, j)
// reflectors, each stored as SB_B + 1 complex values (tau and its first row, then v).
#define SB_B 16
#define SB_NMIN 48
#define SB_NMAX 192
__host__ __device__ inline int sb_nsteps(int n, int j) { return (n - 3 - j) / SB_B + 1; }
// sum of floor(u / SB_B) over u = 0 .. U (0 for U < 0)
__host__ __device__ inline long long sb_fsum(long long U) {
    if (U < 0) return 0;
    const long long q = (U + 1) / SB_B, r = (U + 1) % SB_B;
    return (long long)SB_B * q * (q - 1) / 2 + q * r;
}
// reflectors of the sweeps before sweep j: sum of sb_nsteps(n, j') over j' < j
__host__ __device__ inline long long sb_sweep_off(int n, int j) {
    return j + sb_fsum(n - 3) - sb_fsum(n - 3 - j);
}
__host__ __device__ inline long long sb_stride(int n) {
    return (long long)n * (SB_B + 1) + sb_sweep_off(n, n - 2) * (SB_B + 1);
}
__host__ __device__ inline bool sb_eligible(int n) { return n >= SB_NMIN && n <= SB_NMAX; }

struct EigArgs {
    const cf *B0;
    cf *Gp;              // packed G in, Householder vectors out (offset g.poff per group)
    float *lam;          // [mat][s] eigenvalues above the threshold (descending)
    cf *V;               // [mat][s][s] eigenvectors (vector-major), first rank of them valid
    int *rank;           // [mat]
    float *tri;          // [mat][4 s]: tridiagonal d, reflector tau, complex sub-diagonal e
    const int *active;
    unsigned *status;
    float *zsave;        // non-null: keep the tridiagonal-basis eigenvectors of the computed
                         // pairs here ([mat] at g.off + mat s len, row q = pair q)
    int allp;            // compute every eigenpair, not only those above t^2 (needs zsave)
    int ev_chunk;        // inverse-iteration vectors per pass: 16 or 8 (0: by order)
    // per-matrix hand-off flags of the programmatic launch chain (or null: plain launches)
    unsigned *gready;    // k_gram_tc -> k_tridiag
    unsigned *ready;     // k_tridiag -> k_eigvec
    unsigned *vready;    // k_eigvec -> k_apply_stream / k_apply_eig
    unsigned long long *rank_acc;   // [mat] running sum of ranks over a solve, or null
    int fp64_fallback;   // flag near-degenerate matrices (rank -1) for the FP64 re-solve
    // two-stage reduction: scratch of GroupSet::sb_total elements (Group::sboff), or null;
    // reduction 0 = by order, 1 = one-stage only, 2 = two-stage wherever the order allows
    cf *sb;
    int reduction;
    unsigned *bready;    // k_sb1 -> k_sb2 (with gready / ready; null with plain launches)
    int band;            // set by launch_heig: k_eigvec back-transforms through the two stages
};
cudaError_t eig_init_attributes();
cudaError_t launch_gram(const GroupSet &gs, int mat_begin, int mat_count, const cf *B0, cf *Gp,
                        const int *active, cudaStream_t st);
cudaError_t launch_heig(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, cudaStream_t st);
cudaError_t launch_apply_eig(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, const SvtArgs &a,
                             cudaStream_t st);
// Resolvent solves of the reverse mode: for every computed pair q of every matrix,
// Y[2q + c] = Q P Pi (lambda_q I - T_r)^{-1} Pi P^H Q^H W[2q + c] (c = 0, 1), with
// Pi = I - sum_k z_k z_k^T over the computed pairs (zsave).  W, Y: per matrix at
// 2 (g.off + mat s len), 2 rank vectors of length s.
cudaError_t launch_resolvent(const GroupSet &gs, int mat_count, const EigArgs &ea, const cf *W, cf *Y,
                             cudaStream_t st);

// svt_fp64.cu: FP64 one-sided Jacobi S_t of the matrices k_eigvec flagged (rank -1), with the
// outputs of the FP32 apply; `slots` CTAs, each with slot_elems double2 of `work`.
#define SELR_FP64_SLOTS 8
cudaError_t launch_svt_fp64(const GroupSet &gs, int mat_begin, int mat_count, const EigArgs &ea, const SvtArgs &a,
                            void *work, long long slot_elems, int slots, cudaStream_t st);

// grad.cu
cudaError_t launch_cgemm(int batch, int m, int n, int k, cf alpha, const cf *A, int opa, long long lda, long long sa,
                         const cf *B, int opb, long long ldb, long long sb, cf beta, cf *C, long long ldc,
                         long long sc, cudaStream_t st);
cudaError_t launch_gamma(int batch, int s, const float *lam, float t, cf *M, long long sm, long long sl,
                         cudaStream_t st);
cudaError_t launch_scale_vecs(int batch, int s, const float *lam, float t, const cf *V, cf *Vs, long long sv,
                              long long sl, int mode, cudaStream_t st);
cudaError_t launch_tbar(int batch, int s, const float *lam, float t, const cf *Ct, long long sm, long long sl,
                        float *tbar, cudaStream_t st);
cudaError_t launch_herm_sum(int batch, int s, cf *M, long long sm, cudaStream_t st);
cudaError_t launch_axpbypcz(long long n, float a, const cf *x, float b, const cf *y, float c, const cf *z, cf *out,
                            cudaStream_t st);
cudaError_t launch_dot_re(long long n, const cf *x, const cf *y, double *part, float *out, cudaStream_t st);
cudaError_t launch_augment(int batch, int s, int len, const cf *Bt, cf *aug, cudaStream_t st);
struct LrBuffers {
    cf *U, *Gv, *W, *Y, *C11, *M2, *X, *Ab;   // see k_lr_front in grad.cu for the slots
    double *tpart;                           // per-matrix threshold-cotangent partials
};
cudaError_t launch_lowrank_vjp(const GroupSet &gs, int nmat, const cf *Bt, const cf *Zt, const cf *V, const float *lam,
                               const int *rank, float t, const LrBuffers &b, float *tbar, cf *Bbart, cf *Zout_t,
                               const EigArgs &ea, cudaStream_t st);
cudaError_t launch_split_aug(int batch, int s, int len, const cf *aug, cf *Vt, float *lam, cudaStream_t st);
cudaError_t launch_add_diag(int batch, int s, cf *M, long long sm, float v, cudaStream_t st);

// dc.cu
struct DcArgs {
    int model2d;
    int L, J, M, N;
    const cf *Y; const uint8_t *mask;
    const cf *a; const cf *b;     // already in k-space
    cf *K;
    const float *da;              // 2D: d_r(k_n) [N]; param: d_pe(k_n) [N]
    const float *db;              // 2D: d_c(k_m) [M]; param: c_p(l) [L]
    float lambda, beta;
    double *partial;              // [M][2]
    const int *active;            // per m or nullptr
    unsigned *status;
};
cudaError_t launch_dc(const DcArgs &a, cudaStream_t st);
cudaError_t launch_dc_vjp(const DcArgs &a, const cf *Kbar, cf *out, cf *ybar, cudaStream_t st);
cudaError_t launch_rel_finalize(const double *partial, int M, int per_m, float tol, float *rel,
                                int *active_next, cudaStream_t st);
cudaError_t launch_fill(cf *p, long long n, cf v, cudaStream_t st);

// spirit.cu: SPIRiT calibration and the CG X-update of SHLR-S / SHLR-SV
#define SP_NB 304                 // CTAs of the CG kernels (fixed: deterministic partial sums)
#define SELR_SPIRIT_SLOTS 16      // coil systems solved concurrently in the calibration
struct SpiritArgs {
    int J, M, N, ks, acs, cg_iters;
    long long nK;
    float lambda, beta, lambda1, reg;
    const float *da, *db;         // lift normal diagonals d_r(k_n), d_c(k_m)
    const uint8_t *mask;          // [M][N]
    const cf *Y;                  // [J][M][N] data
    cf *K;                        // iterate, overwritten by the X-update
    const cf *adjA, *adjB;        // transformed lift adjoints (k-space)
    cf *Gm;                       // [J][J][M][N] image-domain G - I
    cf *Hm;                       // [J (J + 1) / 2][M][N] (G - I)^H (G - I), upper triangle per pixel
    cf *g;                        // [J][J][ks][ks] kernel
    float *cj;                    // [J] preconditioner constants
    cf *x, *r, *z, *p, *q, *t;    // CG vectors [J][M][N]
    float *dv, *pdv;              // [J][M][N] diagonal of the operator and the preconditioner
    double *part;                 // [3][SP_NB]
    double *partial;              // [M][2] stopping-ratio partials
    unsigned *status;
    double2 *cal_C, *cal_work;    // calibration: C = A^H A, SELR_SPIRIT_SLOTS Cholesky slots
    FftTable ftM, ftN;
};
cudaError_t launch_spirit_calibrate(const SpiritArgs &s, const cf *Y, cudaStream_t st);
cudaError_t launch_spirit_x_update(const SpiritArgs &s, cudaStream_t st);
cudaError_t launch_fill_i(int *p, long long n, int v, cudaStream_t st);
cudaError_t launch_copy_active(const int *src, int *dst, int n, cudaStream_t st);
