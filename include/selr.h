/*
 * selr.h - C ABI of libselr, a GB300 (sm_103a) implementation of the
 * separable low-rank Hankel reconstruction of Zhang et al., "Accelerated MRI
 * Reconstruction with Separable and Enhanced Low-Rank Hankel Regularization"
 * (SHLR, SHLR-V, SHLR-P, SHLR-VP).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex data is complex64: interleaved (re, im) float pairs, C-contiguous.
 * - 2D models (SHLR, SHLR-V) use arrays [J][M][N] (coil j, row m, column n).
 *   Parameter models (SHLR-P, SHLR-VP) use [L][J][M][N] (echo l outermost,
 *   m = frequency encoding (FE), n = phase encoding (PE)).  For 2D models
 *   L = 1 and the two layouts coincide.
 * - The Fourier transform is the centred unitary DFT
 *   F x = fftshift(fft(ifftshift(x))) / sqrt(n), DC at index n/2; every
 *   transformed length must be even and factor into 2, 3 and 5.
 * - A lifted matrix ("A") has rows = nv - p + 1 window positions and
 *   cols = C * p, channel-major (column c = channel * p + tap), where nv is
 *   the lifted vector length, p the window, C = J or 2J (virtual coils).
 *   Its entries are A[i][ch*p + q] = w[i+q] * v_ch[i+q] for the plain
 *   channels and w[i+q] * conj(v_j[nv-1-(i+q)]) for virtual coil ch = J + j.
 *   Lifted arrays passed across this ABI are [nmat][rows][cols] row-major.
 * - All array pointers are DEVICE pointers owned by the caller unless a
 *   comment says "host".  Nothing is freed or retained by the library.
 * - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *   default stream).  Host-detectable errors (bad arguments, shapes, CUDA
 *   launch failures) are returned immediately and nothing is launched.
 *   Device-detected conditions (Jacobi non-convergence, non-finite values)
 *   are recorded in the plan and reported by selr_sync_status().
 * - No call prints, throws, or aborts.  A plan is not thread-safe; distinct
 *   plans may be used concurrently from different host threads.
 */
#ifndef SELR_H
#define SELR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *selr_stream;   /* == cudaStream_t */

typedef enum {
    SELR_OK = 0,
    SELR_ERR_INVALID_ARG = 1,     /* null pointer, bad enum, non-positive size, bad parameter */
    SELR_ERR_SHAPE = 2,           /* sizes inconsistent with the plan or unsupported length */
    SELR_ERR_CUDA = 3,            /* a CUDA runtime call failed */
    SELR_ERR_NO_CONVERGENCE = 4,  /* a Jacobi SVD hit its sweep cap (device-detected) */
    SELR_ERR_NONFINITE = 5,       /* NaN/Inf met in data or in the iterate (device-detected) */
    SELR_ERR_TIMEOUT = 6,         /* a bounded device wait ran out (device-detected) */
    SELR_ERR_UNSUPPORTED = 7,     /* feature not built */
    SELR_ERR_ALLOC = 8            /* device allocation failed */
} selr_status;

typedef enum {
    SELR_SHLR = 0,     /* Eq. 2: row + column lifts, H~ W~ F~                         */
    SELR_SHLR_V = 1,   /* Eq. 5: as SHLR with virtual coils H~_vc (Eq. 4)               */
    SELR_SHLR_P = 2,   /* Eq. 7: per FE position, PE lifts + parameter-dimension lifts  */
    SELR_SHLR_VP = 3,  /* Eq. 8: SHLR-P with virtual coils on the PE lifts              */
    SELR_SHLR_S = 4,   /* Eq. 3: SHLR + lambda1/2 ||X - G X||^2 (SPIRiT operator G)      */
    SELR_SHLR_SV = 5   /* Eq. 6: SHLR-S with virtual coils                              */
} selr_model;

/* Lift families.  Each names the vectors that are lifted and their source array. */
typedef enum {
    SELR_AXIS_ROW = 0,   /* 2D: row m, vectors over n, source = F^1D along n of the image   */
    SELR_AXIS_COL = 1,   /* 2D: column n, vectors over m, source = F^1D along m             */
    SELR_AXIS_PE = 2,    /* param: (m, l), vectors over PE n, source = PE k-space [L][J][M][N] */
    SELR_AXIS_PARAM = 3  /* param: (m, n), vectors over echoes l, source = image [L][J][M][N] */
} selr_axis;

typedef enum {
    SELR_EXEC_BATCHED = 0, /* every matrix of an iteration in one launch per step; the whole
                              iteration captured once as a CUDA graph                      */
    SELR_EXEC_PLAIN = 1    /* one launch per matrix for lift/SVT/adjoint, no graph           */
} selr_exec;

/* How S_t is computed (both give the exact SVT up to FP32 rounding). */
typedef enum {
    SELR_SVD_EIG = 0,     /* Gram matrix + Hermitian eigensolver for the eigenpairs above t^2 only
                             (Householder tridiagonal, bisection, inverse iteration); default  */
    SELR_SVD_JACOBI = 1   /* one-sided Jacobi on the lifted matrix (all singular pairs)          */
} selr_svd_method;

/* Arithmetic of the Gram matrices G = B^H B that feed the eigensolver
 * (SELR_SVD_EIG; precision option of the SVT, not in the paper).  The
 * tensor-core modes run on tcgen05 (TF32 operands, FP32 accumulation) for
 * families with min(rows, cols) <= 256 and fall back to FP32 otherwise. */
typedef enum {
    SELR_GRAM_FP32 = 0,    /* FP32 FMA (default)                                              */
    SELR_GRAM_TF32 = 1,    /* one TF32 product per term: ~1e-3 relative error in G             */
    SELR_GRAM_3XTF32 = 3,  /* x = x_hi + x_lo split, three TF32 products: about FP32 accuracy  */
    SELR_GRAM_BF16X3 = 4,  /* x = x_hi + x_lo in bf16, three BF16 products (kind::f16):
                              ~2^-16 relative error in G                                        */
    SELR_GRAM_BF16X6 = 6   /* x = x_hi + x_mid + x_lo in bf16, the six products of order <= 4:
                              about FP32 accuracy                                               */
} selr_gram_precision;
/* Measured against the FP64 oracle: reconstructions with 3XTF32 stay at FP32 level
 * (SHLR 12-coil 256x256: 1.8e-7 after 30 iterations; SHLR-P / SHLR-VP 2 coils 8x48x8
 * echoes: below 1e-4 after 10 iterations, as with FP32). */

/* Problem description (Sec. III; Algorithms S1 and S2). */
typedef struct {
    int32_t model;            /* selr_model                                               */
    int32_t J, M, N, L;       /* coils, rows (FE), columns (PE), echoes (1 for 2D models) */
    int32_t window;           /* Hankel window p of row / column / PE lifts               */
    int32_t window_param;     /* Hankel window of the parameter-dimension lift            */
    int32_t weight;           /* W: 0 = identity, 1 = circular first-difference filter    */
    float lambda;             /* data weight (Eq. 2); <= 0 selects hard data consistency  */
    float lambda2;            /* parameter-lift weight (Eq. 7/8); SVT threshold lambda2/beta */
    float beta;               /* ADMM penalty; SVT threshold of row/col/PE lifts is 1/beta */
    float tau;                /* multiplier step (Eqs. 13-14)                             */
    float d_init;             /* initial multiplier value (the paper uses 1)              */
    int32_t max_iter;         /* iteration cap (paper: 50 for S1, 100 for S2)             */
    float tol;                /* stop when ||X+ - X||^2/||X||^2 < tol; < 0 = run max_iter */
    int32_t jacobi_max_sweeps;/* sweep cap of the one-sided Jacobi SVD                    */
    float jacobi_tol;         /* rotate a pair while |x^H y| > tol * ||x|| ||y||          */
    int32_t exec;             /* selr_exec                                                */
    int32_t svd_method;       /* selr_svd_method                                          */
    int32_t gram_precision;   /* selr_gram_precision (SELR_SVD_EIG path)                   */
    float lambda1;            /* SHLR-S / SHLR-SV: SPIRiT weight lambda_1 (Eq. 3; default 1e3)   */
    int32_t spirit_ksize;     /* SPIRiT kernel size: 3, 5 (default) or 7                      */
    int32_t spirit_acs;       /* ACS rows for the calibration: the spirit_acs centre rows of
                                 k-space (all columns), which must be fully sampled (default 24) */
    float spirit_reg;         /* Tikhonov weight of the calibration, relative to the mean
                                 diagonal of the normal matrix (default 1e-3)                   */
    int32_t cg_iters;         /* preconditioned CG iterations of the SHLR-S / SHLR-SV X-update
                                 (default 30)                                                   */
    int32_t fp64_fallback;    /* SELR_SVD_EIG: 1 (default) = re-solve in FP64 every matrix whose
                                 thresholding is not determined in FP32 (t^2 below the FP32
                                 resolution 64 eps_32 lambda_max of its Gram eigenvalues, with
                                 eigenvalues between them); 0 = FP32 only.  A re-solved matrix
                                 costs ~0.1 s (FP64 one-sided Jacobi); the plan holds 8 FP64
                                 work slots of min(rows, cols) x max(rows, cols) elements. */
} selr_desc;

typedef struct selr_plan selr_plan;   /* opaque; owns its device workspace */

/* Fill *desc with defaults (SHLR, weight 1, beta = tau = 20, lambda = 1e4,
 * lambda2 = 2, d_init = 1, max_iter = 30, tol = -1, 30 sweeps, tol 2e-6,
 * batched, SELR_SVD_EIG, SELR_GRAM_FP32, lambda1 = 1e3, SPIRiT kernel 5 x 5 on 24
 * ACS rows with relative Tikhonov weight 1e-3, 30 CG iterations, fp64_fallback = 1). */
void selr_desc_default(selr_desc *desc);

/* Validate *desc and allocate the plan's device workspace on the current
 * device (multipliers D, Jacobi work copies, FFT twiddles, weights).
 * Errors: SELR_ERR_INVALID_ARG, SELR_ERR_SHAPE (odd or non-2/3/5 FFT length,
 * window larger than the vector), SELR_ERR_ALLOC, SELR_ERR_CUDA.
 * *out is set to NULL on failure. */
selr_status selr_plan_create(const selr_desc *desc, selr_plan **out);

/* One plan for n_inst independent reconstructions of uneven size, batched:
 * every step of an iteration runs for all instances at once, and all lifted
 * matrices of one SVT size class (tiny / tridiagonal buckets n <= 32, 64,
 * 128, 208, larger) across all instances go to one launch per kernel (the
 * paper solves one problem at a time; batching is an engineering extension).
 * descs[i] may differ in J, M, N, L, window, window_param, lambda and lambda2;
 * every other field must equal descs[0] (SELR_ERR_INVALID_ARG otherwise).
 * 1 <= n_inst <= 32.  selr_solve then takes packed arrays: instance i's
 * Y / X [L][J][M][N] at element offset k_offset(i) and its mask [L][M][N] at
 * mask_offset(i) (selr_plan_instance_layout).  With tol >= 0 a 2D batch runs
 * until every instance meets the stopping rule (rel_out: the largest change);
 * a parameter-model batch freezes each FE position of each instance on its own
 * criterion (Algorithm S2) and stops when none is left.  The
 * single-operator entry points (selr_lift_shape, selr_transform, selr_lift,
 * selr_adjoint, selr_dc, selr_dc_vjp) return SELR_ERR_UNSUPPORTED on a plan
 * with more than one instance; selr_svt / selr_svt_vjp work on any plan.
 * SHLR-S / SHLR-SV plans hold one instance (SELR_ERR_UNSUPPORTED for a batch
 * of them). */
selr_status selr_plan_create_batch(const selr_desc *descs, int32_t n_inst, selr_plan **out);

/* Element offsets of instance inst in the packed k-space / image arrays and in
 * the packed mask array of a plan (host outputs; either may be NULL). */
selr_status selr_plan_instance_layout(const selr_plan *plan, int32_t inst, int64_t *k_offset,
                                      int64_t *mask_offset);

/* Free the plan and its workspace.  NULL is accepted. */
selr_status selr_plan_destroy(selr_plan *plan);

/* Bytes of device workspace held by the plan (host value). */
size_t selr_plan_workspace_bytes(const selr_plan *plan);

/* Number of matrices, rows and columns of the plan's lift family `axis`
 * (host outputs; any may be NULL).  SELR_ERR_INVALID_ARG if the model has no
 * such family (rows/cols for 2D models, PE/PARAM for parameter models). */
selr_status selr_lift_shape(const selr_plan *plan, int32_t axis, int32_t *nmat,
                            int32_t *rows, int32_t *cols);

/* Centred unitary 1D DFT of an array [L][J][M][N] along dim M (dim = 0) or
 * dim N (dim = 1); inverse != 0 selects F*.  in and out may alias.
 * (Sec. III-A, F^1D; hybrid transforms feeding the row / column lifts.) */
selr_status selr_transform(selr_plan *plan, int32_t dim, int32_t inverse,
                           const void *in, void *out, selr_stream stream);

/* Hankel lift (Eq. 2, Eq. 4, Eq. 7/8): A_out[mat] = lift(x)[mat] + D[mat] / beta.
 * x  : the family's source array (see selr_axis) [L][J][M][N] complex64.
 * D  : [nmat][rows][cols] complex64 or NULL (treated as zero).
 * A_out: [nmat][rows][cols] complex64, fully overwritten. */
selr_status selr_lift(selr_plan *plan, int32_t axis, const void *x, const void *D,
                      void *A_out, selr_stream stream);

/* Singular value thresholding S_t (Eqs. 16-17, S8-S9) of nmat complex64
 * matrices [nmat][rows][cols], in place: A <- U diag(max(sigma - t, 0)) V^H.
 * Computed as the plan's svd_method says: SELR_SVD_EIG (default) forms
 * G = B^H B (B the matrix with its shorter side as columns) in the plan's Gram
 * precision, finds the eigenpairs of G above t^2 by Householder
 * tridiagonalisation, multisection and inverse iteration in FP32 (matrices that
 * FP32 cannot resolve at the threshold are re-solved in FP64, see
 * selr_desc.fp64_fallback), and writes sum (1 - t / sigma_i) (B v_i) v_i^H;
 * SELR_SVD_JACOBI runs one-sided Jacobi on B in FP32.
 * thresh: one t for all nmat matrices.  The paper's thresholds are per lift
 * family (1/beta for row / column / PE lifts, lambda2/beta for the
 * parameter-dimension lifts, Eqs. 16-17 and S8-S9), so a scalar per call is
 * the reading; matrices with different thresholds take separate calls.
 * rank_out: device int32[nmat] receiving #{sigma > t}, or NULL.
 * Requires nmat*rows*cols within the plan's workspace capacity
 * (SELR_ERR_SHAPE otherwise) and t >= 0. */
selr_status selr_svt(selr_plan *plan, void *A, int32_t nmat, int32_t rows, int32_t cols,
                     float thresh, int32_t *rank_out, selr_stream stream);

/* Allocation-free variant of selr_svt (the paper has no counterpart; this is
 * an engineering entry point).  For callers that cannot allocate device
 * memory while they run: code issuing work during a CUDA stream capture,
 * where cudaMalloc is not allowed; services that reserve their whole memory
 * budget up front; hosts whose framework owns every device allocation.
 * It computes the same S_t as selr_svt, in place on A [nmat][rows][cols]
 * complex64 (device), with the Jacobi sweep cap `max_sweeps` and rotation
 * tolerance `tol` of selr_desc, without a plan and without allocating:
 * its scratch is a fixed area of the library (about 17 MB per device, held
 * until the process exits).  Limits: nmat * rows * cols <=
 * SELR_SVT_NOALLOC_MAX_ELEMS, nmat <= SELR_SVT_NOALLOC_MAX_MATS,
 * max(rows, cols) <= 512; larger sizes return SELR_ERR_SHAPE.  The first
 * call on each device looks up the scratch address (and sets kernel
 * attributes) for that device, so make it before any stream capture.  All
 * calls on one device share the scratch: calls that may overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Device-side conditions (sweep cap reached, non-finite input) are
 * read back with selr_svt_noalloc_status.
 * rank_out: device int32[nmat] receiving #{sigma > t}, or NULL. */
#define SELR_SVT_NOALLOC_MAX_ELEMS (1 << 20)
#define SELR_SVT_NOALLOC_MAX_MATS 65536
selr_status selr_svt_noalloc(void *A, int32_t nmat, int32_t rows, int32_t cols, float thresh,
                             int32_t max_sweeps, float tol, int32_t *rank_out, selr_stream stream);

/* Condition recorded by the last selr_svt_noalloc call on the current device
 * (no counterpart in the paper): synchronises `stream` (use the stream of that
 * call), reads the fixed status word of the allocation-free scratch and
 * returns SELR_ERR_NONFINITE (NaN/Inf met), SELR_ERR_NO_CONVERGENCE (a matrix
 * reached max_sweeps) or SELR_OK; SELR_ERR_CUDA if a CUDA call fails.  The
 * word is cleared by the next selr_svt_noalloc call, not by this read.
 * Allocates nothing. */
selr_status selr_svt_noalloc_status(selr_stream stream);

/* SPIRiT calibration (Eq. 3 / Eq. 6; SHLR-S and SHLR-SV plans): the kernel g
 * [J][J][ks][ks] that predicts each k-space sample of coil j from the ks x ks
 * neighbourhoods of all coils (the sample itself excluded, circular in
 * k-space), fitted on every kernel position inside the spirit_acs centre rows
 * of Y [J][M][N] by Tikhonov-regularised least squares per target coil in
 * FP64 (the paper gives neither kernel size nor calibration: these are
 * readings), and from it the image-domain operator G - I, a J x J matrix per
 * pixel, kept in the plan.  selr_solve calibrates from its own Y before the
 * first iteration; selr_dc on such a plan needs this call first.
 * SELR_ERR_UNSUPPORTED for other models. */
selr_status selr_spirit_calibrate(selr_plan *plan, const void *Y, selr_stream stream);

/* Copy of the calibrated kernel g [J][J][ks][ks] complex64 into g_out (device),
 * row j = target coil; g[j][j][ks/2][ks/2] = 0.  SELR_ERR_UNSUPPORTED before a
 * calibration or on other models. */
selr_status selr_spirit_kernel(selr_plan *plan, void *g_out, selr_stream stream);

/* Real adjoint of the lift (the transpose appearing in Eq. 15 / S7):
 * x_out = L^T E for the family `axis`.  Plain channel j contributes
 * conj(w) * H*(E_j); virtual coil J+j contributes flip(w * conj(H*(E_{J+j}))),
 * where H* sums anti-diagonals.  E: [nmat][rows][cols]; x_out: [L][J][M][N],
 * fully overwritten, in the family's source domain. */
selr_status selr_adjoint(selr_plan *plan, int32_t axis, const void *E, void *x_out,
                         selr_stream stream);

/* X-update of Eq. 15 (2D) / Eq. S7 (parameter models).  Without the SPIRiT
 * term a pointwise divide in k-space:
 *   K = (lambda U Y + beta (F a + F' b)) / (lambda U + beta (d_a + d_b)).
 * SHLR-S / SHLR-SV: (lambda U + beta (d_a + d_b) + lambda_1 F (G - I)^H (G - I) F*) K
 * = lambda U Y + beta (F a + F' b), by cg_iters conjugate-gradient iterations
 * preconditioned with the k-space diagonal, from the K passed in.
 * 2D: adj_a = row-lift adjoint (F along M applied here), adj_b = column-lift
 *     adjoint (F along N applied here).
 * Parameter: adj_a = PE-lift adjoint (already in PE k-space), adj_b =
 *     parameter-lift adjoint (F along N applied here).
 * adj_a and adj_b are overwritten (transformed in place).  K is read as the
 * previous iterate and overwritten.  Y: zero-filled data [L][J][M][N];
 * mask: [L][M][N] uint8 0/1.  rel_out: device float receiving
 * ||K_new - K||^2 / ||K||^2, or NULL. */
selr_status selr_dc(selr_plan *plan, const void *Y, const uint8_t *mask, void *adj_a,
                    void *adj_b, void *K, float *rel_out, selr_stream stream);

/* Full reconstruction: Algorithm S1 (SHLR, SHLR-V) or S2 (SHLR-P, SHLR-VP,
 * all FE positions batched, each stopping on its own criterion).
 * Init: K = Y, Z = 0, D = d_init.  Per iteration: X-update (Eq. 15 / S7),
 * Z = SVT (Eqs. 16-17 / S8-S9), D update (Eqs. 13-14 / S5-S6).
 * Y: [L][J][M][N] zero-filled k-space (parameter models: after the inverse
 * DFT along FE, i.e. hybrid (m, k_n) data).  mask: [L][M][N] uint8.
 * X_out: [L][J][M][N] complex64 image.  iters_out (host, may be NULL):
 * iterations run (max over FE positions for parameter models).
 * rel_out (host, may be NULL): last relative change.
 * state_inout (device, may be NULL): a checkpoint of the iteration of
 * selr_state_bytes() bytes holding K, the multipliers D, E = Z - D / beta
 * and the per-FE activity flags (the state between two passes of the loop
 * body of Algorithm S1 / S2).  When non-NULL the final state is written to
 * it.  resume = 1 (state_inout required) starts from that state instead of
 * the initialisation above and runs max_iter further iterations; the state
 * must come from a plan of the same description.  The kernels are
 * deterministic, so k1 iterations, a checkpoint and k2 resumed iterations
 * give bitwise the result of k1 + k2 iterations in one call.
 * With tol >= 0 the call synchronises `stream` once per iteration.
 * Errors: SELR_ERR_INVALID_ARG (NULL arrays, resume not 0/1, resume without
 * a state), SELR_ERR_CUDA. */
selr_status selr_solve(selr_plan *plan, const void *Y, const uint8_t *mask, void *X_out,
                       void *state_inout, int32_t resume, int32_t *iters_out, float *rel_out,
                       selr_stream stream);

/* Forward pass of an unrolled reconstruction (differentiation through
 * Algorithm S1; the paper fixes t and tau): n_iter iterations on the plan's
 * instances (2D models without the SPIRiT term; any number of instances),
 * iteration k with SVT threshold ts[k] (Eqs. 16-17) and multiplier step taus[k]
 * (Eqs. 13-14) instead of 1/beta and tau.  ts, taus: HOST float [n_iter]
 * (ts[k] >= 0).  X_out: the image of the last X-update ([L][J][M][N], packed as
 * for selr_solve).  ckpt_K (device, may be NULL): [n_iter][nK] complex64, the
 * k-space iterate after the X-update of each iteration; ckpt_D (device, may be
 * NULL): [n_iter][selr_lifted_elems] complex64, the multipliers entering that
 * iteration's Z / D steps, in the plan's internal layout (selr_lifted_unpack).
 * On a non-default stream in batched execution the whole pass is one CUDA
 * graph, captured on every call (the parameters change) and updated in place
 * of the previous call's executable graph.  Errors: SELR_ERR_INVALID_ARG,
 * SELR_ERR_UNSUPPORTED (parameter or SPIRiT models), SELR_ERR_CUDA. */
selr_status selr_solve_unrolled(selr_plan *plan, const void *Y, const uint8_t *mask, void *X_out, const float *ts,
                                const float *taus, int32_t n_iter, void *ckpt_K, void *ckpt_D, selr_stream stream);

/* Number of complex64 elements of all lifted matrices of the plan (one
 * multiplier array; host output). */
selr_status selr_lifted_elems(const selr_plan *plan, int64_t *elems);

/* The lifted matrices of family `axis` (selr_axis) of instance `inst` out of a
 * multiplier array in the plan's internal layout (packed: selr_lifted_elems
 * elements, e.g. one checkpoint of selr_solve_unrolled), written to `out` as
 * [nmat][rows][cols] complex64 (device). */
selr_status selr_lifted_unpack(const selr_plan *plan, const void *packed, int32_t inst, int32_t axis, void *out,
                               selr_stream stream);

/* Bytes of a solver state buffer for selr_solve's state_inout (host output). */
selr_status selr_state_bytes(const selr_plan *plan, size_t *bytes);

/* Per-matrix sums of the number of singular values above t found by the
 * eigensolver (SELR_SVD_EIG families) over the iterations of the last
 * selr_solve call (instrumentation: the rank histogram that sets the
 * eigensolver's work, Eqs. 16-17).  out: host int64[n], n = the plan's total
 * number of lifted matrices (every family, in family order); iterations
 * (host, may be NULL): iterations of that call.  Matrices of the
 * warp-per-matrix Jacobi family read 0.  Synchronises `stream`.
 * SELR_ERR_UNSUPPORTED for a SELR_SVD_JACOBI plan. */
selr_status selr_plan_rank_sums(selr_plan *plan, int64_t *out, int32_t n, int32_t *iterations,
                                selr_stream stream);

/* Autotuner (engineering extension, not in the paper): runs short solves
 * (2 iterations each) of the caller's problem Y / mask (as for selr_solve;
 * X_scratch receives throw-away images) and keeps the fastest settings in the
 * plan: with SELR_SVD_EIG the Gram precision among the modes of FP32-level
 * accuracy (SELR_GRAM_FP32, SELR_GRAM_3XTF32, SELR_GRAM_BF16X6; also SELR_GRAM_TF32 and
 * SELR_GRAM_BF16X3 when flags & 1) and the number of eigenvectors refined per inverse-iteration
 * pass (8 or 16), then, on a plan whose reduction mode is 0 and that has two-stage scratch
 * (orders 48 .. 192), whether the two-stage reduction is faster (mode 2 if so); with
 * SELR_SVD_JACOBI the sweep cap (twice the largest
 * number of sweeps a matrix needed, + 2, if below the current cap and no
 * matrix reached it).
 * max_iter, tol and profiling are restored afterwards; cached CUDA graphs are
 * dropped.  Synchronises the stream. */
selr_status selr_plan_autotune(selr_plan *plan, const void *Y, const uint8_t *mask, void *X_scratch,
                               int32_t flags, selr_stream stream);

/* Settings in force (host outputs, any may be NULL): Gram precision, inverse-
 * iteration chunk (0 = chosen by order), Jacobi sweep cap. */
selr_status selr_plan_tuning(const selr_plan *plan, int32_t *gram_precision, int32_t *ev_chunk,
                             int32_t *jacobi_max_sweeps);

/* Sets what the autotuner would: the Gram precision (any SELR_GRAM_* mode) and the number
 * of eigenvectors refined per inverse-iteration pass (8 or 16; 0 = chosen by order; 16 falls
 * back to 8 for orders whose 16-vector layout exceeds shared memory).  Cached CUDA graphs
 * are dropped.  SELR_ERR_INVALID_ARG for other values. */
selr_status selr_plan_set_tuning(selr_plan *plan, int32_t gram_precision, int32_t ev_chunk);

/* Householder reduction of the Gram matrices (SELR_SVD_EIG): 0 = chosen by order, 1 = the
 * one-stage reduction to tridiagonal form for every order, 2 = the two-stage reduction
 * (Hermitian band of half-bandwidth 16 by blocked reflectors, then bulge chasing to
 * tridiagonal form) wherever the order is within 48 .. 192.  Both compute the same
 * eigenpairs to FP32 accuracy; the reverse-mode SVT derivative always uses the one-stage
 * reduction.  Cached CUDA graphs are dropped.  SELR_ERR_INVALID_ARG for other modes. */
selr_status selr_plan_set_reduction(selr_plan *plan, int32_t mode);

/* The reduction mode in force (as set above, or 2 when selr_plan_autotune found the two-stage
 * reduction faster on a plan left at 0). */
selr_status selr_plan_get_reduction(const selr_plan *plan, int32_t *mode);

/* Change the iteration cap and stopping tolerance of an existing plan
 * (same meaning as selr_desc.max_iter / tol).  SELR_ERR_INVALID_ARG if
 * max_iter < 1. */
selr_status selr_set_iterations(selr_plan *plan, int32_t max_iter, float tol);

/* Stage timing of selr_solve (instrumentation, not part of the method).
 * Stages: 0 lift adjoints, 1 data consistency (FFTs of the adjoints, the
 * pointwise solve and its reduction), 2 hybrid transforms, 3 lifts,
 * 4 Gram matrices (SELR_SVD_EIG), 5 eigensolver or Jacobi SVD, 6 SVT apply
 * + multiplier update.  In plain mode stage 3 holds lift, SVD and apply.
 * selr_profile_enable(plan, on): when on, the following selr_solve calls
 * record CUDA events on `stream` around every stage of every iteration (in
 * batched mode each stage is captured as its own CUDA graph and the events
 * are recorded between graph launches).
 * selr_profile_read(plan, stage, total_ms, count): host outputs with the
 * summed duration of `stage` over the last profiled solve and the number of
 * iterations timed; synchronises on the recorded events. */
selr_status selr_profile_enable(selr_plan *plan, int32_t on);
selr_status selr_profile_read(selr_plan *plan, int32_t stage, float *total_ms, int32_t *count);

/* Synchronise `stream` and return the first device-side condition recorded
 * since the last call (SELR_ERR_TIMEOUT, SELR_ERR_NONFINITE,
 * SELR_ERR_NO_CONVERGENCE, in that order of precedence), or SELR_ERR_CUDA if
 * the stream reports an error; clears the record.  SELR_ERR_TIMEOUT means a
 * bounded device wait ran out (an mbarrier of the tensor-core Gram, or the
 * per-matrix hand-off between the eigensolver's kernels, 2 s each): the
 * results of that call are not valid, the context stays usable. */
selr_status selr_sync_status(selr_plan *plan, selr_stream stream);

/* Failure-handling self-test (no counterpart in the paper): one CTA runs the
 * bounded hand-off wait of the eigensolver's kernels on a device flag that the
 * host sets to `set_flag` (0 or 1) beforehand and nothing sets afterwards,
 * with a limit of limit_us microseconds (1 .. 2 000 000).  Returns SELR_OK
 * when the flag was set (and the wait consumed it), SELR_ERR_TIMEOUT when the
 * wait ran out, SELR_ERR_INVALID_ARG for arguments out of range (checked
 * before any CUDA call), SELR_ERR_ALLOC / SELR_ERR_CUDA otherwise.
 * Allocates and frees 8 bytes of device memory; synchronises the device. */
selr_status selr_selftest_wait(int32_t set_flag, int32_t limit_us);

/* ---------------------------------------------------------------------
 * Reverse mode, for unrolled reconstructions whose per-iteration SVT
 * thresholds and multiplier steps are learned (differentiating through the
 * iteration of Algorithm S1; the paper fixes these scalars and has no
 * reverse pass).  Cotangents use the real inner product Re tr(X^H Y) of
 * complex arrays, so the VJP of a complex-linear map is its conjugate
 * transpose.
 * --------------------------------------------------------------------- */

/* VJP of Z = S_t(A) (Eqs. 16-17) for nmat matrices A [nmat][rows][cols]
 * (complex64, device, natural row-major layout, not modified) and the
 * cotangent Zbar of the same shape.  With B = A (cols <= rows) or A^T and
 * G = B^H B = V diag(lambda) V^H, S_t(B) = B h(G) with
 * h(lambda) = max(1 - t / sqrt(lambda), 0), and
 *   Bbar = Zbar h(G) + B (Gbar + Gbar^H),
 *   Gbar = V [Gamma o (V^H B^H Zbar V)] V^H,
 *   Gamma_ij = (h(lambda_i) - h(lambda_j)) / (lambda_i - lambda_j)
 *              (h'(lambda) at ties; evaluated as t / (s_i s_j (s_i + s_j)),
 *              s = sqrt(lambda), when both exceed t, which has no cancellation),
 *   tbar = -Re sum_{lambda_i > t^2} (V^H B^H Zbar V)_ii / sqrt(lambda_i).
 * svd_method = SELR_SVD_EIG (default): only the r pairs above t^2 are computed
 * (the eigensolver of selr_svt); the blocks of Gamma that involve the other
 * pairs are applied as resolvents R_q = sum_{lambda_j <= t^2} v_j v_j^H /
 * (lambda_q - lambda_j), one tridiagonal solve per right-hand side, so the
 * rest costs O(r s len).  SELR_SVD_JACOBI: every pair by one-sided Jacobi on
 * [B; I] (the plan's jacobi_max_sweeps / jacobi_tol; a matrix reaching the
 * cap is reported by selr_sync_status as SELR_ERR_NO_CONVERGENCE), one
 * Newton-Schulz orthonormalisation step and dense s x s products.
 * Abar: [nmat][rows][cols] device output (may not alias A or Zbar).  tbar:
 * device float receiving the threshold cotangent summed over the nmat
 * matrices.  Z_out: NULL, or [nmat][rows][cols] device output receiving
 * S_t(A) itself (computed on the way).  Shapes as for selr_svt plus
 * min(rows, cols) <= 480; the first call allocates the plan's reverse-mode
 * workspace (about 16 lifted arrays). */
selr_status selr_svt_vjp(selr_plan *plan, const void *A, const void *Zbar, int32_t nmat, int32_t rows,
                         int32_t cols, float thresh, void *Abar, float *tbar, void *Z_out, selr_stream stream);

/* VJP of the X-update of Eq. 15 / S7 as computed by selr_dc:
 * K = (lambda U Y + beta S) / den, den = lambda U + beta (d_a + d_b), S the
 * sum of the transformed lift adjoints.  Given Kbar [L][J][M][N] (device),
 * writes Sbar = beta Kbar / den into adj_out and, if Ybar is not NULL,
 * Ybar = lambda U Kbar / den; with lambda <= 0 (hard consistency, K = Y on
 * sampled points) Sbar = Kbar / (d_a + d_b) off the mask, 0 on it, and
 * Ybar = Kbar on it.  Where den is 0 both are 0 (the forward writes 0
 * there).  The caller applies the inverse transforms of the two adjoint
 * families to Sbar.  mask: [L][M][N] uint8, device. */
selr_status selr_dc_vjp(selr_plan *plan, const uint8_t *mask, const void *Kbar, void *adj_out, void *Ybar,
                        selr_stream stream);

/* out = a x + b y + c z over n complex64 elements (device; y or z NULL drops
 * its term; out may alias any input). */
selr_status selr_axpby(int64_t n, float a, const void *x, float b, const void *y, float c, const void *z,
                       void *out, selr_stream stream);

/* *out = Re sum_i conj(x_i) y_i over n complex64 elements (device), reduced
 * in a fixed order in double precision; out is a device float. */
selr_status selr_dot_re(selr_plan *plan, int64_t n, const void *x, const void *y, float *out, selr_stream stream);

/* ---------------------------------------------------------------------
 * Evaluation of reconstructions (Sec. IV; Supplement S3).  Plan-free; every
 * pointer is a device pointer unless marked host; nothing is allocated;
 * reductions run in a fixed order (deterministic).
 * --------------------------------------------------------------------- */

/* SSOS coil combination: out[b][p] = sqrt(sum_j |X[b][j][p]|^2) for X
 * [nb][J][npix] complex64 (nb = 1 for a 2D image [J][M][N] with npix = M N;
 * nb = L echoes for parameter data [L][J][M][N]).  out: float [nb][npix]. */
selr_status selr_ssos(const void *X, int32_t nb, int32_t J, int64_t npix, float *out, selr_stream stream);

/* RLNE = ||x - xhat||_2 / ||x||_2 (Supplement S3) over n floats; *out
 * (device float) receives it (0 when x = 0).  FP64 accumulation. */
selr_status selr_rlne(const float *x, const float *xhat, int64_t n, float *out, selr_stream stream);

/* MSSIM of reference A and image B (real [M][N], Supplement S3): the mean over
 * every window position that fits in the image of
 *   (2 mu_a mu_b + C1)(2 sigma_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(sigma_a^2 + sigma_b^2 + C2)),
 * with Gaussian-weighted local statistics.  The paper fixes neither window nor
 * constants: an 11 x 11 Gaussian window (sigma 1.5, weights summing to 1) and
 * C1 = (0.01 L)^2, C2 = (0.03 L)^2 are taken, L = dynamic range (host value,
 * > 0; usually max A, see selr_max).  ssim_map: caller-owned float
 * [(M - 10)(N - 10)] receiving the per-window values; *out (device float) the
 * mean.  M, N >= 11. */
selr_status selr_mssim(const float *A, const float *B, int32_t M, int32_t N, float L, float *ssim_map, float *out,
                       selr_stream stream);

/* *out (device float) = max of v[0..n). */
selr_status selr_max(const float *v, int64_t n, float *out, selr_stream stream);

/* Pixel-by-pixel nonlinear least-squares T2 fit (Sec. IV, T2 mapping): for
 * every pixel p of S [L][npix] (magnitudes, e.g. SSOS per echo) fits
 * S_l = M0 exp(-TE_l / T2) by Levenberg-Marquardt in FP64 on (M0, 1/T2)
 * from the log-linear fit.  te_ms: HOST float [L] echo times, 2 <= L <= 32.
 * T2_out [npix] (ms) and M0_out [npix] (may be NULL) are NaN where a sample
 * is not positive or T2 falls outside [t2_min, t2_max] (the paper excludes
 * T2 values outside a reasonable range without stating it). */
selr_status selr_t2_fit(const float *S, const float *te_ms, int32_t L, int64_t npix, float t2_min, float t2_max,
                        float *T2_out, float *M0_out, selr_stream stream);

/* Measurement utility (no counterpart in the paper): the FP32 FMA rate of the
 * current device, the denominator of the eigensolver's roofline.  Runs
 * independent FMA chains (x <- x a + b; scalar FFMA when packed = 0, packed
 * two-lane FFMA2 when packed = 1) in 8 CTAs of 256 threads per SM for
 * `iters` (1 .. 2^20) iterations, twice, and reports the second launch:
 * *tflops_out (host) = 2 x FMAs / seconds / 1e12, *ms_out (host, may be
 * NULL) its duration.  Allocates 4 bytes of device memory; synchronises
 * the device. */
selr_status selr_probe_fp32_peak(int32_t packed, int32_t iters, float *tflops_out, float *ms_out);

/* Name of the last CUDA runtime error behind a SELR_ERR_CUDA returned on
 * the calling host thread (diagnostics; static storage). */
const char *selr_last_error_string(void);

/* Static, human-readable name of a status code. */
const char *selr_status_string(selr_status status);

#ifdef __cplusplus
}
#endif
#endif /* SELR_H */
