// C ABI of libselr: plan management, the five operator entry points and the
// ADMM driver (Algorithm S1 for SHLR / SHLR-V, Algorithm S2 for SHLR-P /
// SHLR-VP with every FE position batched).
#include "selr_internal.cuh"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <new>

// One reconstruction problem of a plan: its sizes, its slices of the k-space
// sized arrays and the mask, and its transform tables, weights and normal
// diagonals (the lifted state of all instances shares the plan's arrays).
struct Inst {
    int J, M, N, L, p;
    float lambda;
    long long nK, koff, mkoff;   // k-space elements; offsets in K-sized arrays and in the mask
    int poff;                    // offset of its [M][2] partial sums
    int aoff;                    // offset of its FE positions in the activity flags (parameter models)
    int roff;                    // offset of its block in `rel` (1 value, or 1 + M for parameter models)
    FftTable ftM, ftN;
    cf *twM, *twN, *wM, *wN;
    float *da, *db;
};

struct selr_plan {
    selr_desc d;
    int model2d, vc;
    int L, J, M, N;              // instance 0 (the only one unless created by selr_plan_create_batch)
    long long nK;                // k-space elements of all instances
    int n_inst;
    Inst inst[SELR_MAX_INST];
    GroupSet gs;
    long long lift_elems, vec_elems;
    cf *K, *hybA, *hybB, *adjA, *adjB;
    cf *D, *E, *W, *B0;
    cf *Gp, *V;              // packed Gram matrices / Householder vectors; eigenvectors
    float *lam, *tri;
    int *rank;
    int spirit;                          // SHLR-S / SHLR-SV: SPIRiT term and CG X-update
    int spirit_ready;                    // the kernel has been calibrated (host flag)
    cf *sp_Gm, *sp_g, *sp_vec;           // image-domain G - I, kernel, six CG vectors
    cf *sp_Hm;                           // per pixel (G - I)^H (G - I), packed upper triangle
    float *sp_cj;
    float *sp_diag;                      // diagonal of the X-update operator and preconditioner
    double *sp_part;
    double2 *sp_C, *sp_work;
    unsigned *gready, *ready, *vready;   // kernel hand-off flags, one per matrix (see EigArgs)
    unsigned *bready;                    // k_sb1 -> k_sb2 hand-off flags (two-stage reduction)
    cf *sb;                              // two-stage reduction scratch (gs.sb_total elements)
    long long sb_elems;
    int reduction;                       // 0 by order, 1 one-stage, 2 two-stage (EigArgs)
    unsigned long long *rank_acc;        // per-matrix sum of eigensolver ranks over the last solve
    void *f64work;                       // FP64 re-solve slots (SELR_FP64_SLOTS x f64slot double2)
    long long f64slot;
    int rank_iters;                      // iterations accumulated in rank_acc
    long long packed_elems;
    float *sigma;
    int *mat_status;
    double *partial;
    float *rel;
    int *active, *active_next;
    int Mact;                    // length of the activity flags: FE positions of all instances
    int nrel;                    // length of `rel`
    unsigned *status;
    size_t bytes;
    float *h_rel;          // pinned host mirror
    int *h_active;         // pinned host mirror
    cudaGraphExec_t graph;
    const void *graph_Y;
    const uint8_t *graph_mask;
    cudaStream_t graph_stream;
    int graph_iters;          // 1: `graph` holds one iteration; 0: per-stage graphs (profiling)
    cudaGraphExec_t ugraph;   // the last unrolled forward (selr_solve_unrolled), updated in place
    cudaStream_t ugraph_stream;
    int ovr_on;               // per-iteration threshold / step override (unrolled forward)
    float ovr_tau;
    GroupSet ovr_gs;          // gs with the overriding threshold
    // stage profiling
    int prof_on;
    int prof_cap;             // iterations with events allocated
    cudaEvent_t *ev;          // [prof_cap][NSTAGE][2]
    int prof_count;           // iterations timed by the last solve
    cudaGraphExec_t stage_graph[8];   // profiling: one graph per stage (NSTAGE <= 8)
    // reverse-mode workspaces (allocated on the first VJP call)
    cf *gw_Z, *gw_Bbar, *gw_S1, *gw_S2, *gw_S3, *gw_S4, *gw_V, *gw_aug, *gw_aug2, *gw_Gp;
    cf *gw_U, *gw_Gv, *gw_W, *gw_Yv, *gw_C11, *gw_M2, *gw_X, *gw_Ab, *gw_Zo;
    float *gw_lam, *gw_tri, *gw_zs;
    int *gw_rank;
    double *gw_tpart;
    int ev_chunk;              // tuned inverse-iteration chunk (0: by order)
    int tuned;                 // selr_plan_autotune ran
    double *gw_part;
};

#define NSTAGE 7

static void drop_graphs(selr_plan *p);

// Last CUDA error seen by an entry point on this host thread (diagnostics).
static thread_local cudaError_t g_last_error = cudaSuccess;

#define CK(x)                                          \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) {                       \
            g_last_error = e_;                         \
            return SELR_ERR_CUDA;                      \
        }                                              \
    } while (0)

static bool smooth_even(int n) {
    if (n < 2 || (n & 1)) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    while (n % 5 == 0) n /= 5;
    return n == 1;
}

extern "C" void selr_desc_default(selr_desc *d) {
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->model = SELR_SHLR;
    d->J = 4; d->M = 64; d->N = 64; d->L = 1;
    d->window = 8;
    d->window_param = 4;
    d->weight = 1;
    d->lambda = 1.0e4f;
    d->lambda2 = 2.0f;
    d->beta = 20.0f;
    d->tau = 20.0f;
    d->d_init = 1.0f;
    d->max_iter = 30;
    d->tol = -1.0f;
    d->jacobi_max_sweeps = 30;
    d->jacobi_tol = 2.0e-6f;
    d->exec = SELR_EXEC_BATCHED;
    d->svd_method = SELR_SVD_EIG;
    d->gram_precision = SELR_GRAM_FP32;
    d->fp64_fallback = 1;
    d->lambda1 = 1.0e3f;
    d->spirit_ksize = 5;
    d->spirit_acs = 24;
    d->spirit_reg = 1.0e-3f;
    d->cg_iters = 30;
}

extern "C" const char *selr_status_string(selr_status s) {
    switch (s) {
        case SELR_OK: return "SELR_OK";
        case SELR_ERR_INVALID_ARG: return "SELR_ERR_INVALID_ARG";
        case SELR_ERR_SHAPE: return "SELR_ERR_SHAPE";
        case SELR_ERR_CUDA: return "SELR_ERR_CUDA";
        case SELR_ERR_NO_CONVERGENCE: return "SELR_ERR_NO_CONVERGENCE";
        case SELR_ERR_NONFINITE: return "SELR_ERR_NONFINITE";
        case SELR_ERR_TIMEOUT: return "SELR_ERR_TIMEOUT";
        case SELR_ERR_UNSUPPORTED: return "SELR_ERR_UNSUPPORTED";
        case SELR_ERR_ALLOC: return "SELR_ERR_ALLOC";
    }
    return "SELR_ERR_UNKNOWN";
}

// Host-side description of one lift family (see Group in selr_internal.cuh).
static Group make_group(int kind, int nmat, int nv, int p, int J, int vc, int M, int N, int L, float thresh) {
    Group g;
    memset(&g, 0, sizeof(g));
    g.kind = kind;
    g.nmat = nmat;
    g.nv = nv;
    g.p = p;
    g.J = J;
    g.vc = vc;
    g.C = vc ? 2 * J : J;
    g.rows = nv - p + 1;
    g.cols = g.C * p;
    g.trans = g.cols > g.rows ? 1 : 0;
    g.s = g.trans ? g.rows : g.cols;
    g.len = g.trans ? g.cols : g.rows;
    g.thresh = thresh;
    g.M = M;
    g.N = N;
    g.L = L;
    return g;
}

static void finish_set(GroupSet *gs) {
    long long off = 0, soff = 0, poff = 0, sboff = 0;
    int moff = 0;
    gs->start[0] = 0;
    for (int k = 0; k < gs->n; ++k) {
        gs->g[k].off = off;
        gs->g[k].soff = soff;
        gs->g[k].poff = poff;
        gs->g[k].moff = moff;
        gs->g[k].sboff = -1;
        if (sb_eligible(gs->g[k].s)) {
            gs->g[k].sboff = sboff;
            sboff += (long long)gs->g[k].nmat * sb_stride(gs->g[k].s);
        }
        poff += (long long)gs->g[k].nmat * gs->g[k].s * (gs->g[k].s + 1) / 2;
        off += (long long)gs->g[k].nmat * gs->g[k].rows * gs->g[k].cols;
        soff += (long long)gs->g[k].nmat * gs->g[k].s;
        moff += gs->g[k].nmat;
        gs->start[k + 1] = moff;
    }
    gs->total = moff;
    gs->sb_total = sboff;
}

static selr_status validate(const selr_desc *d) {
    if (!d) return SELR_ERR_INVALID_ARG;
    if (d->model < SELR_SHLR || d->model > SELR_SHLR_SV) return SELR_ERR_INVALID_ARG;
    if (d->J < 1 || d->M < 1 || d->N < 1 || d->L < 1 || d->window < 1) return SELR_ERR_INVALID_ARG;
    if (!(d->beta > 0.f) || !(d->tau > 0.f) || d->max_iter < 1 || d->jacobi_max_sweeps < 1 ||
        !(d->jacobi_tol > 0.f) || !isfinite(d->lambda) || !isfinite(d->beta) || !isfinite(d->tau) ||
        !isfinite(d->d_init) || !(d->lambda2 >= 0.f))
        return SELR_ERR_INVALID_ARG;
    if (d->weight != 0 && d->weight != 1) return SELR_ERR_INVALID_ARG;
    if (d->fp64_fallback != 0 && d->fp64_fallback != 1) return SELR_ERR_INVALID_ARG;
    if (d->exec != SELR_EXEC_BATCHED && d->exec != SELR_EXEC_PLAIN) return SELR_ERR_INVALID_ARG;
    if (d->svd_method != SELR_SVD_EIG && d->svd_method != SELR_SVD_JACOBI) return SELR_ERR_INVALID_ARG;
    if (d->gram_precision != SELR_GRAM_FP32 && d->gram_precision != SELR_GRAM_TF32 &&
        d->gram_precision != SELR_GRAM_3XTF32 && d->gram_precision != SELR_GRAM_BF16X3 &&
        d->gram_precision != SELR_GRAM_BF16X6)
        return SELR_ERR_INVALID_ARG;
    const bool two_d = d->model <= SELR_SHLR_V || d->model >= SELR_SHLR_S;
    if (d->model >= SELR_SHLR_S) {
        if (!(d->lambda > 0.f) || !(d->lambda1 >= 0.f) || !isfinite(d->lambda1) || !(d->spirit_reg > 0.f) ||
            d->cg_iters < 1 || d->cg_iters > 200)
            return SELR_ERR_INVALID_ARG;
        if ((d->spirit_ksize != 3 && d->spirit_ksize != 5 && d->spirit_ksize != 7) || d->J > 32)
            return SELR_ERR_INVALID_ARG;
        if (d->spirit_acs < d->spirit_ksize || d->spirit_acs > d->M || d->spirit_ksize > d->N) return SELR_ERR_SHAPE;
    }
    if (two_d) {
        if (d->L != 1) return SELR_ERR_SHAPE;
        if (!smooth_even(d->M) || !smooth_even(d->N) || d->M > 1024 || d->N > 1024) return SELR_ERR_SHAPE;
        if (d->window > d->M || d->window > d->N) return SELR_ERR_SHAPE;
    } else {
        if (d->window_param < 1 || d->window_param > d->L) return SELR_ERR_SHAPE;
        if (!smooth_even(d->N) || d->N > 1024) return SELR_ERR_SHAPE;
        if (d->window > d->N) return SELR_ERR_SHAPE;
    }
    return SELR_OK;
}

static selr_status alloc(selr_plan *p, void **ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return SELR_ERR_ALLOC;
    }
    p->bytes += bytes;
    return SELR_OK;
}

static void host_weights(int n, int kind, cf *out) {
    for (int k = 0; k < n; ++k) {
        if (kind == 0) { out[k] = mk(1.f, 0.f); continue; }
        const double a = -2.0 * M_PI * ((double)k - n / 2.0) / (double)n;
        out[k] = mk((float)(1.0 - cos(a)), (float)(-sin(a)));
    }
}

// d(k) = c(k)|w(k)|^2 [+ c(n-1-k)|w(n-1-k)|^2], c = Hankel multiplicities.
static void host_normal(int n, int p, int kind, int vc, float *out) {
    cf *w = (cf *)malloc(sizeof(cf) * n);
    for (int k = 0; k < n; ++k) out[k] = 0.f;
    host_weights(n, kind, w);
    const int l = n - p + 1;
    double *acc = (double *)calloc(n, sizeof(double));
    for (int k = 0; k < n; ++k) {
        int c = k + 1;
        if (p < c) c = p;
        if (n - k < c) c = n - k;
        if (l < c) c = l;
        const double w2 = (double)w[k].x * w[k].x + (double)w[k].y * w[k].y;
        acc[k] += c * w2;
        if (vc) acc[n - 1 - k] += c * w2;
    }
    for (int k = 0; k < n; ++k) out[k] = (float)acc[k];
    free(acc);
    free(w);
}

static void host_multiplicity(int n, int p, float *out) {
    const int l = n - p + 1;
    for (int k = 0; k < n; ++k) {
        int c = k + 1;
        if (p < c) c = p;
        if (n - k < c) c = n - k;
        if (l < c) c = l;
        out[k] = (float)c;
    }
}

static selr_status upload(void *dst, const void *src, size_t bytes) {
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess ? SELR_OK : SELR_ERR_CUDA;
}

extern "C" selr_status selr_plan_destroy(selr_plan *p) {
    if (!p) return SELR_OK;
    drop_graphs(p);
    void *gbufs[] = {p->gw_Z, p->gw_Bbar, p->gw_S1, p->gw_S2, p->gw_S3, p->gw_S4, p->gw_V, p->gw_aug, p->gw_aug2,
                     p->gw_Gp, p->gw_U, p->gw_Gv, p->gw_W, p->gw_Yv, p->gw_C11, p->gw_M2, p->gw_X, p->gw_Ab,
                     p->gw_Zo, p->gw_lam, p->gw_tri, p->gw_zs, p->gw_rank, p->gw_tpart, p->gw_part};
    for (void *b : gbufs)
        if (b) cudaFree(b);
    void *bufs[] = {p->K, p->hybA, p->hybB, p->adjA, p->adjB, p->D, p->E, p->W, p->B0, p->Gp, p->V, p->lam, p->tri,
                    p->rank, p->gready, p->ready, p->vready, p->bready, p->sb, p->rank_acc, p->f64work, p->sp_Gm, p->sp_g,
                    p->sp_vec, p->sp_Hm, p->sp_cj, p->sp_diag, p->sp_part, p->sp_C, p->sp_work, p->sigma,
                    p->mat_status, p->partial, p->rel, p->active, p->active_next, p->status};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (int i = 0; i < p->n_inst; ++i) {
        Inst &I = p->inst[i];
        void *ib[] = {I.twM, I.twN, I.wM, I.wN, I.da, I.db};
        for (void *b : ib)
            if (b) cudaFree(b);
    }
    if (p->ev) {
        for (size_t i = 0; i < (size_t)p->prof_cap * NSTAGE * 2; ++i) cudaEventDestroy(p->ev[i]);
        free(p->ev);
    }
    if (p->h_rel) cudaFreeHost(p->h_rel);
    if (p->h_active) cudaFreeHost(p->h_active);
    delete p;
    return SELR_OK;
}

// SVT kernel class of a lift family: families of one class share one launch
// sequence (0: warp-per-matrix SVT; eigensolver: tridiagonal template buckets).
static int svt_class(const Group &g, int svd) {
    if (svt_small_fits(g)) return 0;
    if (svd == SELR_SVD_JACOBI) return 1;
    if (g.s <= 32) return 1;
    if (g.s <= 64) return 2;
    if (g.s <= 128) return 3;
    if (g.s <= 192) return 4;
    if (g.s <= 208) return 5;
    if (g.s <= 256) return 6;
    return 7;
}

// Descriptions of a batch must agree on everything but the problem sizes and lambda.
static selr_status check_batch(const selr_desc *ds, int n) {
    for (int i = 0; i < n; ++i) {
        const selr_status s = validate(&ds[i]);
        if (s != SELR_OK) return s;
    }
    if (n == 1) return SELR_OK;
    for (int i = 0; i < n; ++i) {
        const selr_desc &a = ds[0], &b = ds[i];
        if (b.model >= SELR_SHLR_S) return SELR_ERR_UNSUPPORTED;    // SPIRiT plans hold one instance
        if (b.model != a.model || b.weight != a.weight || b.beta != a.beta || b.tau != a.tau ||
            b.d_init != a.d_init || b.max_iter != a.max_iter || b.tol != a.tol || b.exec != a.exec ||
            b.svd_method != a.svd_method || b.gram_precision != a.gram_precision ||
            b.jacobi_max_sweeps != a.jacobi_max_sweeps || b.jacobi_tol != a.jacobi_tol ||
            b.fp64_fallback != a.fp64_fallback)
            return SELR_ERR_INVALID_ARG;
    }
    return SELR_OK;
}

static selr_status create_plan(const selr_desc *ds, int n_inst, selr_plan **out) {
    if (!out) return SELR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ds || n_inst < 1 || n_inst > SELR_MAX_INST) return SELR_ERR_INVALID_ARG;
    selr_status s = check_batch(ds, n_inst);
    if (s != SELR_OK) return s;
    selr_plan *p = new (std::nothrow) selr_plan;
    if (!p) return SELR_ERR_ALLOC;
    memset(p, 0, sizeof(*p));
    const selr_desc *d = &ds[0];
    p->d = *d;
    p->n_inst = n_inst;
    p->model2d = d->model <= SELR_SHLR_V || d->model >= SELR_SHLR_S;
    p->vc = d->model == SELR_SHLR_V || d->model == SELR_SHLR_VP || d->model == SELR_SHLR_SV;
    p->spirit = d->model >= SELR_SHLR_S;
    p->L = d->L; p->J = d->J; p->M = d->M; p->N = d->N;
    const float t1 = 1.0f / d->beta;
    GroupSet &gs = p->gs;
    gs.n = 0;
    long long koff = 0, mkoff = 0;
    int poff = 0, aoff = 0, roff = 0;
    for (int i = 0; i < n_inst; ++i) {
        const selr_desc &di = ds[i];
        Inst &I = p->inst[i];
        I.J = di.J; I.M = di.M; I.N = di.N; I.L = di.L; I.p = di.window; I.lambda = di.lambda;
        I.nK = (long long)di.L * di.J * di.M * di.N;
        I.koff = koff; I.mkoff = mkoff; I.poff = poff; I.aoff = aoff; I.roff = roff;
        koff += I.nK;
        mkoff += (long long)di.L * di.M * di.N;
        poff += 2 * di.M;
        aoff += p->model2d ? 0 : di.M;
        roff += p->model2d ? 1 : 1 + di.M;
        if (p->model2d) {
            gs.g[gs.n] = make_group(G_ROW, di.M, di.N, di.window, di.J, p->vc, di.M, di.N, 1, t1);
            gs.g[gs.n++].inst = i;
            gs.g[gs.n] = make_group(G_COL, di.N, di.M, di.window, di.J, p->vc, di.M, di.N, 1, t1);
            gs.g[gs.n++].inst = i;
        } else {
            gs.g[gs.n] = make_group(G_PE, di.M * di.L, di.N, di.window, di.J, p->vc, di.M, di.N, di.L, t1);
            gs.g[gs.n].inst = i;
            gs.g[gs.n++].aoff = I.aoff;
            gs.g[gs.n] = make_group(G_PARAM, di.M * di.N, di.L, di.window_param, di.J, 0, di.M, di.N, di.L,
                                    di.lambda2 / di.beta);
            gs.g[gs.n].inst = i;
            gs.g[gs.n++].aoff = I.aoff;
        }
    }
    p->nK = koff;
    p->Mact = p->model2d ? d->M : aoff;
    p->nrel = roff;
    for (int k = 0; k < gs.n; ++k) {
        if (gs.g[k].len > 512 || gs.g[k].s > 1024) { delete p; return SELR_ERR_SHAPE; }
        if (d->svd_method == SELR_SVD_EIG && gs.g[k].s > 480) { delete p; return SELR_ERR_SHAPE; }
    }
    if (n_inst > 1) {
        // order the families by SVT class so that each class is one contiguous launch
        for (int a = 1; a < gs.n; ++a) {
            const Group g = gs.g[a];
            const int c = svt_class(g, d->svd_method);
            int b = a - 1;
            while (b >= 0 && svt_class(gs.g[b], d->svd_method) > c) { gs.g[b + 1] = gs.g[b]; --b; }
            gs.g[b + 1] = g;
        }
    }
    finish_set(&gs);
    p->lift_elems = 0;
    p->vec_elems = 0;
    p->packed_elems = 0;
    for (int k = 0; k < gs.n; ++k) {
        p->lift_elems += (long long)gs.g[k].nmat * gs.g[k].rows * gs.g[k].cols;
        p->vec_elems += (long long)gs.g[k].nmat * gs.g[k].s;
        p->packed_elems += (long long)gs.g[k].nmat * gs.g[k].s * (gs.g[k].s + 1) / 2;
    }
    if (fft_init_attributes() != cudaSuccess || svt_init_attributes() != cudaSuccess ||
        eig_init_attributes() != cudaSuccess) {
        delete p;
        return SELR_ERR_CUDA;
    }
#define AL(ptr, bytes)                                                      \
    do {                                                                    \
        selr_status s_ = alloc(p, (void **)&(ptr), (bytes));                \
        if (s_ != SELR_OK) { selr_plan_destroy(p); return s_; }             \
    } while (0)
    const size_t kb = sizeof(cf) * (size_t)p->nK;
    AL(p->K, kb); AL(p->hybA, kb); AL(p->hybB, kb); AL(p->adjA, kb); AL(p->adjB, kb);
    const size_t lb = sizeof(cf) * (size_t)p->lift_elems;
    AL(p->D, lb); AL(p->E, lb); AL(p->B0, lb);
    if (d->svd_method == SELR_SVD_JACOBI) {
        AL(p->W, lb);
    } else {
        AL(p->V, lb);
        AL(p->Gp, sizeof(cf) * (size_t)p->packed_elems);
        AL(p->lam, sizeof(float) * (size_t)p->vec_elems);
        AL(p->tri, 4 * sizeof(float) * (size_t)p->vec_elems);
        AL(p->rank, sizeof(int) * (size_t)gs.total);
        AL(p->gready, sizeof(unsigned) * (size_t)gs.total);
        AL(p->ready, sizeof(unsigned) * (size_t)gs.total);
        AL(p->vready, sizeof(unsigned) * (size_t)gs.total);
        if (gs.sb_total > 0) {
            AL(p->bready, sizeof(unsigned) * (size_t)gs.total);
            AL(p->sb, sizeof(cf) * (size_t)gs.sb_total);
            p->sb_elems = gs.sb_total;
        }
        AL(p->rank_acc, sizeof(unsigned long long) * (size_t)gs.total);
        if (d->fp64_fallback) {
            long long mx = 0;
            for (int k = 0; k < gs.n; ++k) mx = mx > (long long)gs.g[k].s * gs.g[k].len ? mx : (long long)gs.g[k].s * gs.g[k].len;
            p->f64slot = mx;
            AL(p->f64work, 16 * (size_t)mx * SELR_FP64_SLOTS);
        }
    }
    const size_t nrel = (size_t)p->nrel;
    AL(p->sigma, sizeof(float) * (size_t)p->vec_elems);
    AL(p->mat_status, sizeof(int) * (size_t)gs.total);
    AL(p->partial, sizeof(double) * (size_t)poff);
    AL(p->rel, sizeof(float) * nrel);
    AL(p->active, sizeof(int) * (size_t)p->Mact);
    AL(p->active_next, sizeof(int) * (size_t)p->Mact);
    AL(p->status, sizeof(unsigned));
    if (p->spirit) {
        const long long J = d->J, ks = d->spirit_ksize, nu = J * ks * ks, ns = nu - 1;
        AL(p->sp_Gm, sizeof(cf) * (size_t)(J * J * d->M * d->N));
        AL(p->sp_Hm, sizeof(cf) * (size_t)(J * (J + 1) / 2 * d->M * d->N));
        AL(p->sp_g, sizeof(cf) * (size_t)(J * J * ks * ks));
        AL(p->sp_vec, 6 * sizeof(cf) * (size_t)p->nK);
        AL(p->sp_diag, 2 * sizeof(float) * (size_t)p->nK);
        AL(p->sp_cj, sizeof(float) * (size_t)J);
        AL(p->sp_part, 3 * sizeof(double) * SP_NB);
        AL(p->sp_C, sizeof(double2) * (size_t)(nu * nu));
        AL(p->sp_work, sizeof(double2) * (size_t)(SELR_SPIRIT_SLOTS * (ns * ns + ns)));
    }
    for (int i = 0; i < n_inst; ++i) {
        Inst &I = p->inst[i];
        AL(I.wN, sizeof(cf) * I.N);
        AL(I.wM, sizeof(cf) * I.M);
        AL(I.da, sizeof(float) * I.N);
        AL(I.db, sizeof(float) * (p->model2d ? I.M : I.L));
    }
#undef AL
    if (cudaMemset(p->status, 0, sizeof(unsigned)) != cudaSuccess ||
        (p->ready && (cudaMemset(p->gready, 0, sizeof(unsigned) * (size_t)gs.total) != cudaSuccess ||
                      cudaMemset(p->ready, 0, sizeof(unsigned) * (size_t)gs.total) != cudaSuccess ||
                      cudaMemset(p->vready, 0, sizeof(unsigned) * (size_t)gs.total) != cudaSuccess ||
                      (p->bready && cudaMemset(p->bready, 0, sizeof(unsigned) * (size_t)gs.total) != cudaSuccess)))) {
        selr_plan_destroy(p);
        return SELR_ERR_CUDA;
    }
    for (int i = 0; i < n_inst; ++i) {
        Inst &I = p->inst[i];
        const selr_desc &di = ds[i];
        // FFT tables (N always; M for the 2D models)
        if (fft_table_build(I.N, &I.ftN, &I.twN) != cudaSuccess) { selr_plan_destroy(p); return SELR_ERR_SHAPE; }
        if (p->model2d && fft_table_build(I.M, &I.ftM, &I.twM) != cudaSuccess) {
            selr_plan_destroy(p);
            return SELR_ERR_SHAPE;
        }
        // weights and normal diagonals
        const int nmax = I.M > I.N ? I.M : I.N;
        cf *hw = (cf *)malloc(sizeof(cf) * nmax);
        float *hd = (float *)malloc(sizeof(float) * (nmax > I.L ? nmax : I.L));
        selr_status e = (hw && hd) ? SELR_OK : SELR_ERR_ALLOC;
        if (e == SELR_OK) {
            host_weights(I.N, di.weight, hw);
            e = upload(I.wN, hw, sizeof(cf) * I.N);
            host_weights(I.M, di.weight, hw);
            if (e == SELR_OK) e = upload(I.wM, hw, sizeof(cf) * I.M);
            host_normal(I.N, di.window, di.weight, p->vc, hd);
            if (e == SELR_OK) e = upload(I.da, hd, sizeof(float) * I.N);
            if (p->model2d) {
                host_normal(I.M, di.window, di.weight, p->vc, hd);
                if (e == SELR_OK) e = upload(I.db, hd, sizeof(float) * I.M);
            } else {
                host_multiplicity(I.L, di.window_param, hd);
                if (e == SELR_OK) e = upload(I.db, hd, sizeof(float) * I.L);
            }
        }
        free(hw);
        free(hd);
        if (e != SELR_OK) { selr_plan_destroy(p); return e; }
    }
    // sources and destinations of every family
    for (int k = 0; k < gs.n; ++k) {
        Group &g = gs.g[k];
        const Inst &I = p->inst[g.inst];
        switch (g.kind) {
            case G_ROW: g.w = d->weight ? I.wN : nullptr; g.src = p->hybA + I.koff; g.dst = p->adjA + I.koff; break;
            case G_COL: g.w = d->weight ? I.wM : nullptr; g.src = p->hybB + I.koff; g.dst = p->adjB + I.koff; break;
            case G_PE: g.w = d->weight ? I.wN : nullptr; g.src = p->K + I.koff; g.dst = p->adjA + I.koff; break;
            default: g.w = nullptr; g.src = p->hybB + I.koff; g.dst = p->adjB + I.koff; break;
        }
    }
    if (cudaMallocHost((void **)&p->h_rel, sizeof(float) * nrel) != cudaSuccess ||
        cudaMallocHost((void **)&p->h_active, sizeof(int) * (size_t)p->Mact) != cudaSuccess) {
        cudaGetLastError();
        selr_plan_destroy(p);
        return SELR_ERR_ALLOC;
    }
    *out = p;
    return SELR_OK;
}

extern "C" selr_status selr_plan_create(const selr_desc *d, selr_plan **out) { return create_plan(d, 1, out); }

extern "C" selr_status selr_plan_create_batch(const selr_desc *descs, int32_t n_inst, selr_plan **out) {
    return create_plan(descs, n_inst, out);
}

extern "C" selr_status selr_plan_instance_layout(const selr_plan *p, int32_t inst, int64_t *k_offset,
                                                 int64_t *mask_offset) {
    if (!p || inst < 0 || inst >= p->n_inst) return SELR_ERR_INVALID_ARG;
    if (k_offset) *k_offset = p->inst[inst].koff;
    if (mask_offset) *mask_offset = p->inst[inst].mkoff;
    return SELR_OK;
}

extern "C" size_t selr_plan_workspace_bytes(const selr_plan *p) { return p ? p->bytes : 0; }

static int group_index(const selr_plan *p, int axis) {
    if (p->model2d) {
        if (axis == SELR_AXIS_ROW) return 0;
        if (axis == SELR_AXIS_COL) return 1;
    } else {
        if (axis == SELR_AXIS_PE) return 0;
        if (axis == SELR_AXIS_PARAM) return 1;
    }
    return -1;
}

extern "C" selr_status selr_lift_shape(const selr_plan *p, int32_t axis, int32_t *nmat, int32_t *rows,
                                       int32_t *cols) {
    if (!p) return SELR_ERR_INVALID_ARG;
    if (p->n_inst != 1) return SELR_ERR_UNSUPPORTED;
    const int gi = group_index(p, axis);
    if (gi < 0) return SELR_ERR_INVALID_ARG;
    if (nmat) *nmat = p->gs.g[gi].nmat;
    if (rows) *rows = p->gs.g[gi].rows;
    if (cols) *cols = p->gs.g[gi].cols;
    return SELR_OK;
}

// Transform along M (dim 0) or N (dim 1) of instance i's [L][J][M][N] array.
static cudaError_t transform(selr_plan *p, int i, int dim, int inverse, const cf *in, cf *out, cudaStream_t st) {
    const Inst &I = p->inst[i];
    if (dim == 0) return launch_fft(in, out, I.ftM, (long long)I.L * I.J, I.N, inverse, st);
    return launch_fft(in, out, I.ftN, (long long)I.L * I.J * I.M, 1, inverse, st);
}

extern "C" selr_status selr_transform(selr_plan *p, int32_t dim, int32_t inverse, const void *in, void *out,
                                      selr_stream stream) {
    if (!p || !in || !out || (dim != 0 && dim != 1)) return SELR_ERR_INVALID_ARG;
    if (p->n_inst != 1) return SELR_ERR_UNSUPPORTED;
    if (dim == 0 && !p->model2d) return SELR_ERR_SHAPE;
    CK(transform(p, 0, dim, inverse ? 1 : 0, (const cf *)in, (cf *)out, (cudaStream_t)stream));
    return SELR_OK;
}

static GroupSet single_group(const selr_plan *p, int gi) {
    GroupSet s;
    memset(&s, 0, sizeof(s));
    s.n = 1;
    s.g[0] = p->gs.g[gi];
    finish_set(&s);
    return s;
}

extern "C" selr_status selr_lift(selr_plan *p, int32_t axis, const void *x, const void *D, void *A_out,
                                 selr_stream stream) {
    NvtxRange nvtx_range("selr_lift");
    if (!p || !x || !A_out) return SELR_ERR_INVALID_ARG;
    if (p->n_inst != 1) return SELR_ERR_UNSUPPORTED;
    const int gi = group_index(p, axis);
    if (gi < 0) return SELR_ERR_INVALID_ARG;
    GroupSet s = single_group(p, gi);
    s.g[0].src = (const cf *)x;
    CK(launch_lift(s, 0, 0, s.total, (const cf *)D, 1, 1.0f / p->d.beta, (cf *)A_out, nullptr, 1, nullptr,
                   (cudaStream_t)stream));
    return SELR_OK;
}

extern "C" selr_status selr_adjoint(selr_plan *p, int32_t axis, const void *E, void *x_out, selr_stream stream) {
    NvtxRange nvtx_range("selr_adjoint");
    if (!p || !E || !x_out) return SELR_ERR_INVALID_ARG;
    if (p->n_inst != 1) return SELR_ERR_UNSUPPORTED;
    const int gi = group_index(p, axis);
    if (gi < 0) return SELR_ERR_INVALID_ARG;
    GroupSet s = single_group(p, gi);
    s.g[0].dst = (cf *)x_out;
    CK(launch_adjoint(s, 0, 0, s.total, (const cf *)E, 1, (cudaStream_t)stream));
    return SELR_OK;
}

static SvtArgs svt_args(selr_plan *p) {
    SvtArgs a;
    memset(&a, 0, sizeof(a));
    a.W = p->W;
    a.B0 = p->B0;
    a.sigma = p->sigma;
    a.mat_status = p->mat_status;
    a.status = p->status;
    a.max_sweeps = p->d.jacobi_max_sweeps;
    a.tol = p->d.jacobi_tol;
    a.beta = p->d.beta;
    a.tau = p->d.tau;
    return a;
}

static EigArgs eig_args(selr_plan *p, const int *active) {
    EigArgs e;
    memset(&e, 0, sizeof(e));
    e.B0 = p->B0;
    e.Gp = p->Gp;
    e.lam = p->lam;
    e.V = p->V;
    e.rank = p->rank;
    e.tri = p->tri;
    e.active = active;
    e.status = p->status;
    e.ev_chunk = p->ev_chunk;
    e.ready = p->ready;
    e.vready = p->vready;
    e.bready = p->bready;
    e.sb = p->sb;
    e.reduction = p->reduction;
    return e;
}

// S_t of every matrix of `gs` in [m0, m0 + mc): B0 (and W for Jacobi) already filled.
static cudaError_t svd_apply(selr_plan *p, const GroupSet &gs, int m0, int mc, const SvtArgs &a, int part,
                             cudaStream_t st) {
    // one launch sequence per run of consecutive families of the same SVT class (the
    // families of a batched plan are ordered by class): kernels are sized for their
    // class, tiny matrices go to the warp-per-matrix kernel
    const int svd = p->d.svd_method;
    for (int k = 0; k < gs.n;) {
        const int c = svt_class(gs.g[k], svd);
        int k1 = k + 1;
        while (k1 < gs.n && svt_class(gs.g[k1], svd) == c) ++k1;
        const int b = m0 > gs.start[k] ? m0 : gs.start[k];
        const int e_ = (m0 + mc) < gs.start[k1] ? (m0 + mc) : gs.start[k1];
        if (b < e_) {
            GroupSet v;
            memset(&v, 0, sizeof(v));
            v.n = k1 - k;
            bool tc = p->d.gram_precision != SELR_GRAM_FP32;
            for (int i = 0; i < v.n; ++i) {
                v.g[i] = gs.g[k + i];
                v.start[i] = gs.start[k + i] - gs.start[k];
                tc = tc && gram_tc_fits(v.g[i]);
            }
            v.start[v.n] = gs.start[k1] - gs.start[k];
            v.total = v.start[v.n];
            const int lb = b - gs.start[k], lc = e_ - b;
            cudaError_t e = cudaSuccess;
            if (c == 0) {
                if (part & 4) e = launch_svt_small(v, lb, lc, a, st);
            } else if (svd == SELR_SVD_JACOBI) {
                if (part & 2) e = launch_jacobi(v, lb, lc, a, st);
                if (e == cudaSuccess && (part & 4)) e = launch_svt_apply(v, lb, lc, a, st);
            } else {
                // the tensor-core Gram (one CTA per matrix) hands each matrix to k_tridiag by flag
                EigArgs ea = eig_args(p, a.active);
                ea.gready = tc ? p->gready : nullptr;
                ea.rank_acc = a.mode == 1 ? p->rank_acc : nullptr;    // ADMM iterations only
                ea.fp64_fallback = p->f64work != nullptr;
                if (gs.sb_total > p->sb_elems) ea.sb = nullptr;         // scratch too small: one-stage
                if (part & 1)
                    e = tc ? launch_gram_tc(v, lb, lc, p->B0, p->Gp, a.active, (int)p->d.gram_precision, p->status,
                                            p->gready, st)
                           : launch_gram(v, lb, lc, p->B0, p->Gp, a.active, st);
                if (e == cudaSuccess && (part & 2)) e = launch_heig(v, lb, lc, ea, st);
                if (e == cudaSuccess && (part & 4)) e = launch_apply_eig(v, lb, lc, ea, a, st);
                if (e == cudaSuccess && (part & 4) && p->f64work)
                    e = launch_svt_fp64(v, lb, lc, ea, a, p->f64work, p->f64slot, SELR_FP64_SLOTS, st);
            }
            if (e != cudaSuccess) return e;
        }
        k = k1;
    }
    return cudaSuccess;
}

extern "C" selr_status selr_svt(selr_plan *p, void *A, int32_t nmat, int32_t rows, int32_t cols, float thresh,
                                int32_t *rank_out, selr_stream stream) {
    NvtxRange nvtx_range("selr_svt");
    if (!p || !A || nmat < 1 || rows < 1 || cols < 1 || !(thresh >= 0.f) || !isfinite(thresh))
        return SELR_ERR_INVALID_ARG;
    GroupSet s;
    memset(&s, 0, sizeof(s));
    s.n = 1;
    Group &g = s.g[0];
    g.kind = G_ROW;
    g.nmat = nmat;
    g.rows = rows;
    g.cols = cols;
    g.trans = cols > rows ? 1 : 0;
    g.s = g.trans ? rows : cols;
    g.len = g.trans ? cols : rows;
    g.thresh = thresh;
    finish_set(&s);
    if (g.len > 512 || g.s > 1024) return SELR_ERR_SHAPE;
    if ((long long)nmat * rows * cols > p->lift_elems || (long long)nmat * g.s > p->vec_elems || nmat > p->gs.total ||
        (p->d.svd_method == SELR_SVD_EIG && ((long long)nmat * g.s * (g.s + 1) / 2 > p->packed_elems || g.s > 480)))
        return SELR_ERR_SHAPE;
    cudaStream_t st = (cudaStream_t)stream;
    const bool jac = p->d.svd_method == SELR_SVD_JACOBI;
    CK(launch_natural_to_vm(s, (const cf *)A, jac ? p->W : p->B0, jac ? p->B0 : nullptr, st));
    SvtArgs a = svt_args(p);
    a.mode = 0;
    a.Zout = (cf *)A;
    a.z_natural = 1;
    a.rank_out = rank_out;
    CK(svd_apply(p, s, 0, nmat, a, 7, st));
    return SELR_OK;
}

// Arguments of the SPIRiT kernels of a single-instance SHLR-S / SHLR-SV plan.
static SpiritArgs spirit_args(selr_plan *p, const cf *Y, const uint8_t *mask, const cf *adj_a, const cf *adj_b,
                              cf *K) {
    SpiritArgs s;
    memset(&s, 0, sizeof(s));
    const Inst &I = p->inst[0];
    s.J = I.J; s.M = I.M; s.N = I.N;
    s.ks = p->d.spirit_ksize; s.acs = p->d.spirit_acs; s.cg_iters = p->d.cg_iters;
    s.nK = I.nK;
    s.lambda = I.lambda; s.beta = p->d.beta; s.lambda1 = p->d.lambda1; s.reg = p->d.spirit_reg;
    s.da = I.da; s.db = I.db; s.mask = mask; s.Y = Y; s.K = K; s.adjA = adj_a; s.adjB = adj_b;
    s.Gm = p->sp_Gm; s.Hm = p->sp_Hm; s.g = p->sp_g; s.cj = p->sp_cj;
    s.x = p->sp_vec; s.r = s.x + I.nK; s.z = s.r + I.nK; s.p = s.z + I.nK; s.q = s.p + I.nK; s.t = s.q + I.nK;
    s.dv = p->sp_diag; s.pdv = s.dv + I.nK;
    s.part = p->sp_part; s.partial = p->partial + I.poff; s.status = p->status;
    s.cal_C = p->sp_C; s.cal_work = p->sp_work;
    s.ftM = I.ftM; s.ftN = I.ftN;
    return s;
}

// FFTs of the adjoints to k-space, the pointwise solve (or, with the SPIRiT
// term, the CG solve) and the reduction, per instance (arrays are the packed
// ones; each instance works on its slices).
static cudaError_t dc_step(selr_plan *p, const cf *Y, const uint8_t *mask, cf *adj_a, cf *adj_b, cf *K,
                           const int *active, int *active_next, cudaStream_t st) {
    cudaError_t e;
    for (int i = 0; i < p->n_inst; ++i) {
        const Inst &I = p->inst[i];
        cf *aa = adj_a + I.koff, *ab = adj_b + I.koff;
        if (p->model2d) {
            if ((e = transform(p, i, 0, 0, aa, aa, st)) != cudaSuccess) return e;
            if ((e = transform(p, i, 1, 0, ab, ab, st)) != cudaSuccess) return e;
        } else {
            if ((e = transform(p, i, 1, 0, ab, ab, st)) != cudaSuccess) return e;
        }
        DcArgs a;
        memset(&a, 0, sizeof(a));
        a.model2d = p->model2d;
        a.L = I.L; a.J = I.J; a.M = I.M; a.N = I.N;
        a.Y = Y + I.koff; a.mask = mask + I.mkoff; a.a = aa; a.b = ab; a.K = K + I.koff;
        a.da = I.da; a.db = I.db;
        a.lambda = I.lambda;
        a.beta = p->d.beta;
        a.partial = p->partial + I.poff;
        a.active = active ? active + I.aoff : nullptr;
        a.status = p->status;
        if (p->spirit) e = launch_spirit_x_update(spirit_args(p, Y, mask, aa, ab, K), st);
        else e = launch_dc(a, st);
        if (e != cudaSuccess) return e;
        if ((e = launch_rel_finalize(p->partial + I.poff, I.M, !p->model2d, p->d.tol, p->rel + I.roff,
                                     active_next ? active_next + I.aoff : nullptr, st)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

extern "C" selr_status selr_spirit_calibrate(selr_plan *p, const void *Y, selr_stream stream) {
    NvtxRange nvtx_range("selr_spirit_calibrate");
    if (!p || !Y) return SELR_ERR_INVALID_ARG;
    if (!p->spirit) return SELR_ERR_UNSUPPORTED;
    CK(launch_spirit_calibrate(spirit_args(p, (const cf *)Y, nullptr, nullptr, nullptr, nullptr), (const cf *)Y,
                               (cudaStream_t)stream));
    p->spirit_ready = 1;
    return SELR_OK;
}

extern "C" selr_status selr_spirit_kernel(selr_plan *p, void *g_out, selr_stream stream) {
    if (!p || !g_out) return SELR_ERR_INVALID_ARG;
    if (!p->spirit || !p->spirit_ready) return SELR_ERR_UNSUPPORTED;
    const size_t bytes = sizeof(cf) * (size_t)p->d.J * p->d.J * p->d.spirit_ksize * p->d.spirit_ksize;
    CK(cudaMemcpyAsync(g_out, p->sp_g, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SELR_OK;
}

extern "C" selr_status selr_dc(selr_plan *p, const void *Y, const uint8_t *mask, void *adj_a, void *adj_b,
                               void *K, float *rel_out, selr_stream stream) {
    NvtxRange nvtx_range("selr_dc");
    if (!p || !Y || !mask || !adj_a || !adj_b || !K) return SELR_ERR_INVALID_ARG;
    if (p->n_inst != 1) return SELR_ERR_UNSUPPORTED;
    if (p->spirit && !p->spirit_ready) return SELR_ERR_UNSUPPORTED;    // selr_spirit_calibrate first
    cudaStream_t st = (cudaStream_t)stream;
    CK(dc_step(p, (const cf *)Y, mask, (cf *)adj_a, (cf *)adj_b, (cf *)K, nullptr, nullptr, st));
    if (rel_out) CK(cudaMemcpyAsync(rel_out, p->rel, sizeof(float), cudaMemcpyDeviceToDevice, st));
    return SELR_OK;
}

// The seven stages of one ADMM iteration (X, then Z and D) on the plan's state:
//   0 adjoint of (Z - D/beta), 1 X-update (Eq. 15 / S7), 2 lift sources
//   (hybrid transforms), 3 lifts, 4 Gram matrices, 5 eigensolver / Jacobi SVD,
//   6 SVT apply + D update.  In plain mode stage 3 runs lift and the whole SVT
//   one matrix at a time and stages 4-6 are empty.
static cudaError_t admm_stage_body(selr_plan *p, int stage, const cf *Y, const uint8_t *mask, cudaStream_t st);

// One ADMM stage (0 adjoint, 1 X-update, 2 hybrid transforms, 3 lift, 4 Gram, 5 eigensolver,
// 6 apply and multiplier update) inside an NVTX range named after it.
static cudaError_t admm_stage(selr_plan *p, int stage, const cf *Y, const uint8_t *mask, cudaStream_t st) {
    static const char *const names[] = {"adjoint", "dc", "hybrid_fft", "lift", "gram", "svd", "apply"};
    NvtxRange r(stage >= 0 && stage < 7 ? names[stage] : "stage");
    return admm_stage_body(p, stage, Y, mask, st);
}

static cudaError_t admm_stage_body(selr_plan *p, int stage, const cf *Y, const uint8_t *mask, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    const bool plain = p->d.exec == SELR_EXEC_PLAIN;
    const bool jac = p->d.svd_method == SELR_SVD_JACOBI;
    const int *act = p->model2d ? nullptr : p->active;
    int *act_next = p->model2d ? nullptr : p->active_next;
    const int total = p->gs.total;
    SvtArgs a = svt_args(p);
    a.mode = 1;
    a.D = p->D;
    a.E = p->E;
    a.active = act;
    if (p->ovr_on) a.tau = p->ovr_tau;
    const GroupSet &G = p->ovr_on ? p->ovr_gs : p->gs;    // thresholds of this iteration
    const float ib = 1.0f / p->d.beta;
    cf *lift_out = jac ? p->W : p->B0;
    cf *lift_out2 = jac ? p->B0 : nullptr;
    switch (stage) {
        case 0:
            if (plain) {
                for (int m = 0; m < total && e == cudaSuccess; ++m) e = launch_adjoint(p->gs, 0, m, 1, p->E, 0, st);
                return e;
            }
            return launch_adjoint(p->gs, 0, 0, total, p->E, 0, st);
        case 1:
            return dc_step(p, Y, mask, p->adjA, p->adjB, p->K, act, act_next, st);
        case 2:
            for (int i = 0; i < p->n_inst; ++i) {
                const long long o = p->inst[i].koff;
                if (p->model2d && (e = transform(p, i, 0, 1, p->K + o, p->hybA + o, st)) != cudaSuccess) return e;
                if ((e = transform(p, i, 1, 1, p->K + o, p->hybB + o, st)) != cudaSuccess) return e;
            }
            return cudaSuccess;
        case 3:
            if (plain) {
                for (int m = 0; m < total; ++m) {
                    if ((e = launch_lift(p->gs, 0, m, 1, p->D, 0, ib, lift_out, lift_out2, 0, act, st)) != cudaSuccess)
                        return e;
                    if ((e = svd_apply(p, G, m, 1, a, 7, st)) != cudaSuccess) return e;
                }
                if (!p->model2d) return launch_copy_active(p->active_next, p->active, p->Mact, st);
                return cudaSuccess;
            }
            return launch_lift(p->gs, 0, 0, total, p->D, 0, ib, lift_out, lift_out2, 0, act, st);
        case 4:
            return plain ? cudaSuccess : svd_apply(p, G, 0, total, a, 1, st);
        case 5:
            return plain ? cudaSuccess : svd_apply(p, G, 0, total, a, 2, st);
        default:
            if (plain) return cudaSuccess;
            if ((e = svd_apply(p, G, 0, total, a, 4, st)) != cudaSuccess) return e;
            if (!p->model2d) return launch_copy_active(p->active_next, p->active, p->Mact, st);
            return cudaSuccess;
    }
}

static cudaError_t admm_iteration(selr_plan *p, const cf *Y, const uint8_t *mask, cudaStream_t st) {
    for (int s = 0; s < NSTAGE; ++s) {
        cudaError_t e = admm_stage(p, s, Y, mask, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t prof_reserve(selr_plan *p, int iters) {
    if (iters <= p->prof_cap) return cudaSuccess;
    cudaEvent_t *ev = (cudaEvent_t *)calloc((size_t)iters * NSTAGE * 2, sizeof(cudaEvent_t));
    if (!ev) return cudaErrorMemoryAllocation;
    for (size_t i = 0; i < (size_t)p->prof_cap * NSTAGE * 2; ++i) ev[i] = p->ev[i];
    for (size_t i = (size_t)p->prof_cap * NSTAGE * 2; i < (size_t)iters * NSTAGE * 2; ++i) {
        cudaError_t e = cudaEventCreate(&ev[i]);
        if (e != cudaSuccess) {
            for (size_t k = (size_t)p->prof_cap * NSTAGE * 2; k < i; ++k) cudaEventDestroy(ev[k]);
            free(ev);
            return e;
        }
    }
    free(p->ev);
    p->ev = ev;
    p->prof_cap = iters;
    return cudaSuccess;
}

static void drop_graphs(selr_plan *p) {
    if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
    if (p->ugraph) { cudaGraphExecDestroy(p->ugraph); p->ugraph = nullptr; }
    for (int s = 0; s < 8; ++s)
        if (p->stage_graph[s]) { cudaGraphExecDestroy(p->stage_graph[s]); p->stage_graph[s] = nullptr; }
}

// Capture [s0, s1) stages (or a whole iteration) into an executable graph.
static cudaError_t capture(selr_plan *p, int s0, int s1, const cf *Y, const uint8_t *mask, cudaStream_t st,
                           cudaGraphExec_t *out) {
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int s = s0; s < s1 && e == cudaSuccess; ++s) e = admm_stage(p, s, Y, mask, st);
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(g);
        return e != cudaSuccess ? e : e2;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// Layout of a solver state (checkpoint) buffer: the iterate K, the multipliers D,
// E = Z - D / beta (the Z of Eqs. 16-17 is never stored on its own) and the per-FE
// activity flags, each region starting on a 256-byte boundary.
struct StateLayout {
    size_t k, d, e, act, act_next, total;
};
static StateLayout state_layout(const selr_plan *p) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    StateLayout L;
    L.k = 0;
    L.d = al(L.k + sizeof(cf) * (size_t)p->nK);
    L.e = al(L.d + sizeof(cf) * (size_t)p->lift_elems);
    L.act = al(L.e + sizeof(cf) * (size_t)p->lift_elems);
    L.act_next = al(L.act + sizeof(int) * (size_t)p->Mact);
    L.total = al(L.act_next + sizeof(int) * (size_t)p->Mact);
    return L;
}

extern "C" selr_status selr_state_bytes(const selr_plan *p, size_t *bytes) {
    if (!p || !bytes) return SELR_ERR_INVALID_ARG;
    *bytes = state_layout(p).total;
    return SELR_OK;
}

static cudaError_t state_copy(selr_plan *p, unsigned char *state, int save, cudaStream_t st) {
    const StateLayout L = state_layout(p);
    struct { void *plan; size_t off, bytes; } r[] = {
        {p->K, L.k, sizeof(cf) * (size_t)p->nK}, {p->D, L.d, sizeof(cf) * (size_t)p->lift_elems},
        {p->E, L.e, sizeof(cf) * (size_t)p->lift_elems}, {p->active, L.act, sizeof(int) * (size_t)p->Mact},
        {p->active_next, L.act_next, sizeof(int) * (size_t)p->Mact}};
    for (auto &x : r) {
        cudaError_t e = save ? cudaMemcpyAsync(state + x.off, x.plan, x.bytes, cudaMemcpyDeviceToDevice, st)
                             : cudaMemcpyAsync(x.plan, state + x.off, x.bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t admm_init(selr_plan *p, const cf *Y, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(p->K, Y, sizeof(cf) * p->nK, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = launch_fill(p->D, p->lift_elems, mk(p->d.d_init, 0.f), st)) != cudaSuccess) return e;
    if ((e = launch_fill(p->E, p->lift_elems, mk(-p->d.d_init / p->d.beta, 0.f), st)) != cudaSuccess) return e;
    if ((e = launch_fill_i(p->active, p->Mact, 1, st)) != cudaSuccess) return e;
    return launch_fill_i(p->active_next, p->Mact, 1, st);
}

static cudaError_t output_image(selr_plan *p, cf *X, cudaStream_t st) {
    cudaError_t e;
    for (int i = 0; i < p->n_inst; ++i) {
        const long long o = p->inst[i].koff;
        if ((e = transform(p, i, 1, 1, p->K + o, X + o, st)) != cudaSuccess) return e;
        if (p->model2d && (e = transform(p, i, 0, 1, X + o, X + o, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

extern "C" selr_status selr_solve(selr_plan *p, const void *Yv, const uint8_t *mask, void *X_out,
                                  void *state_inout, int32_t resume, int32_t *iters_out, float *rel_out,
                                  selr_stream stream) {
    NvtxRange nvtx_range("selr_solve");
    if (!p || !Yv || !mask || !X_out || (resume != 0 && resume != 1) || (resume && !state_inout))
        return SELR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const cf *Y = (const cf *)Yv;
    if (p->spirit) {       // SPIRiT kernel from this data's ACS rows (before the iteration graph)
        CK(launch_spirit_calibrate(spirit_args(p, Y, mask, nullptr, nullptr, nullptr), Y, st));
        p->spirit_ready = 1;
    }
    if (resume) CK(state_copy(p, (unsigned char *)state_inout, 0, st));
    else CK(admm_init(p, Y, st));
    if (p->rank_acc) CK(cudaMemsetAsync(p->rank_acc, 0, sizeof(unsigned long long) * (size_t)p->gs.total, st));
    int iters = 0;
    float last_rel = -1.f;
    const bool fixed = p->d.tol < 0.f;
    const bool use_graph = fixed && p->d.exec == SELR_EXEC_BATCHED && st != 0;
    if (p->prof_on) CK(prof_reserve(p, p->d.max_iter));
    const int prof = p->prof_on;
    if (use_graph) {
        if (p->graph_Y != Yv || p->graph_mask != mask || p->graph_stream != st || p->graph_iters != (prof ? 0 : 1) ||
            (prof ? !p->stage_graph[0] : !p->graph)) {
            drop_graphs(p);
            if (prof) {
                for (int s = 0; s < NSTAGE; ++s) CK(capture(p, s, s + 1, Y, mask, st, &p->stage_graph[s]));
            } else {
                CK(capture(p, 0, NSTAGE, Y, mask, st, &p->graph));
            }
            p->graph_Y = Yv;
            p->graph_mask = mask;
            p->graph_stream = st;
            p->graph_iters = prof ? 0 : 1;
        }
        for (int k = 0; k < p->d.max_iter; ++k) {
            if (!prof) {
                CK(cudaGraphLaunch(p->graph, st));
                continue;
            }
            for (int s = 0; s < NSTAGE; ++s) {
                CK(cudaEventRecord(p->ev[((size_t)k * NSTAGE + s) * 2], st));
                CK(cudaGraphLaunch(p->stage_graph[s], st));
                CK(cudaEventRecord(p->ev[((size_t)k * NSTAGE + s) * 2 + 1], st));
            }
        }
        iters = p->d.max_iter;
    } else {
        for (int k = 0; k < p->d.max_iter; ++k) {
            if (prof) {
                for (int s = 0; s < NSTAGE; ++s) {
                    CK(cudaEventRecord(p->ev[((size_t)k * NSTAGE + s) * 2], st));
                    CK(admm_stage(p, s, Y, mask, st));
                    CK(cudaEventRecord(p->ev[((size_t)k * NSTAGE + s) * 2 + 1], st));
                }
            } else {
                CK(admm_iteration(p, Y, mask, st));
            }
            ++iters;
            if (!fixed) {
                CK(cudaMemcpyAsync(p->h_rel, p->rel, sizeof(float) * p->nrel, cudaMemcpyDeviceToHost, st));
                if (!p->model2d)
                    CK(cudaMemcpyAsync(p->h_active, p->active, sizeof(int) * p->Mact, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                last_rel = p->h_rel[p->inst[0].roff];
                for (int i = 1; i < p->n_inst; ++i) last_rel = fmaxf(last_rel, p->h_rel[p->inst[i].roff]);
                if (p->model2d) {
                    if (last_rel < p->d.tol) break;      // every instance meets the criterion
                } else {
                    int any = 0;
                    for (int m = 0; m < p->Mact; ++m) any |= p->h_active[m];
                    if (!any) break;
                }
            }
        }
    }
    p->prof_count = p->prof_on ? (iters < p->prof_cap ? iters : p->prof_cap) : 0;
    p->rank_iters = iters;
    if (state_inout) CK(state_copy(p, (unsigned char *)state_inout, 1, st));
    CK(output_image(p, (cf *)X_out, st));
    if (rel_out || iters_out) {
        if (rel_out && fixed) {
            CK(cudaMemcpyAsync(p->h_rel, p->rel, sizeof(float) * p->nrel, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            last_rel = p->h_rel[p->inst[0].roff];
            for (int i = 1; i < p->n_inst; ++i) last_rel = fmaxf(last_rel, p->h_rel[p->inst[i].roff]);
        }
        if (rel_out) *rel_out = last_rel;
        if (iters_out) *iters_out = iters;
    }
    return SELR_OK;
}

extern "C" const char *selr_last_error_string(void) { return cudaGetErrorString(g_last_error); }

// ------------------------------------------------------ unrolled forward
// n iterations of Algorithm S1 with threshold ts[k] and step taus[k] in iteration k;
// checkpoint k = (K after the X-update of iteration k, D entering its Z / D steps).
static cudaError_t unrolled_forward(selr_plan *p, const cf *Y, const uint8_t *mask, const float *ts,
                                    const float *taus, int n, cf *ckK, cf *ckD, cf *X, cudaStream_t st) {
    cudaError_t e = admm_init(p, Y, st);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        p->ovr_on = 0;
        if ((e = admm_stage(p, 0, Y, mask, st)) != cudaSuccess) break;
        if ((e = admm_stage(p, 1, Y, mask, st)) != cudaSuccess) break;
        if (ckK && (e = cudaMemcpyAsync(ckK + (long long)k * p->nK, p->K, sizeof(cf) * p->nK, cudaMemcpyDeviceToDevice,
                                        st)) != cudaSuccess)
            break;
        if (ckD && (e = cudaMemcpyAsync(ckD + (long long)k * p->lift_elems, p->D, sizeof(cf) * p->lift_elems,
                                        cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            break;
        if (k == n - 1) break;
        p->ovr_gs = p->gs;
        for (int g = 0; g < p->ovr_gs.n; ++g) p->ovr_gs.g[g].thresh = ts[k];
        p->ovr_tau = taus[k];
        p->ovr_on = 1;
        for (int s = 2; s < NSTAGE && e == cudaSuccess; ++s) e = admm_stage(p, s, Y, mask, st);
    }
    p->ovr_on = 0;
    if (e != cudaSuccess) return e;
    return output_image(p, X, st);
}

extern "C" selr_status selr_solve_unrolled(selr_plan *p, const void *Y, const uint8_t *mask, void *X_out,
                                           const float *ts, const float *taus, int32_t n_iter, void *ckpt_K,
                                           void *ckpt_D, selr_stream stream) {
    NvtxRange nvtx_range("selr_solve_unrolled");
    if (!p || !Y || !mask || !X_out || !ts || !taus || n_iter < 1) return SELR_ERR_INVALID_ARG;
    if (!p->model2d || p->spirit) return SELR_ERR_UNSUPPORTED;
    for (int k = 0; k < n_iter; ++k)
        if (!(ts[k] >= 0.f) || !isfinite(ts[k]) || !isfinite(taus[k])) return SELR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const cf *Yc = (const cf *)Y;
    cf *ckK = (cf *)ckpt_K, *ckD = (cf *)ckpt_D, *X = (cf *)X_out;
    if (st == 0 || p->d.exec != SELR_EXEC_BATCHED) {
        CK(unrolled_forward(p, Yc, mask, ts, taus, n_iter, ckK, ckD, X, st));
        return SELR_OK;
    }
    // the whole forward as one CUDA graph; the parameters change every call, so it is captured
    // each time and the executable graph of the previous call updated in place when possible
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = unrolled_forward(p, Yc, mask, ts, taus, n_iter, ckK, ckD, X, st);
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(g);
        g_last_error = e != cudaSuccess ? e : e2;
        return SELR_ERR_CUDA;
    }
    bool updated = false;
    if (p->ugraph && p->ugraph_stream == st) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(p->ugraph, g, &info) == cudaSuccess;
        if (!updated) cudaGetLastError();
    }
    if (!updated) {
        if (p->ugraph) { cudaGraphExecDestroy(p->ugraph); p->ugraph = nullptr; }
        e = cudaGraphInstantiate(&p->ugraph, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            p->ugraph = nullptr;
            g_last_error = e;
            return SELR_ERR_CUDA;
        }
        p->ugraph_stream = st;
    }
    cudaGraphDestroy(g);
    CK(cudaGraphLaunch(p->ugraph, st));
    return SELR_OK;
}

extern "C" selr_status selr_lifted_unpack(const selr_plan *p, const void *packed, int32_t inst, int32_t axis,
                                          void *out, selr_stream stream) {
    if (!p || !packed || !out || inst < 0 || inst >= p->n_inst) return SELR_ERR_INVALID_ARG;
    const int kind = axis == SELR_AXIS_ROW ? G_ROW : axis == SELR_AXIS_COL ? G_COL : axis == SELR_AXIS_PE ? G_PE
                   : axis == SELR_AXIS_PARAM ? G_PARAM : -1;
    if (kind < 0) return SELR_ERR_INVALID_ARG;
    for (int k = 0; k < p->gs.n; ++k) {
        const Group &g = p->gs.g[k];
        if (g.inst != inst || g.kind != kind) continue;
        GroupSet s;
        memset(&s, 0, sizeof(s));
        s.n = 1;
        s.g[0] = g;
        finish_set(&s);
        CK(launch_vm_to_natural(s, (const cf *)packed + g.off, (cf *)out, (cudaStream_t)stream));
        return SELR_OK;
    }
    return SELR_ERR_INVALID_ARG;
}

extern "C" selr_status selr_lifted_elems(const selr_plan *p, int64_t *elems) {
    if (!p || !elems) return SELR_ERR_INVALID_ARG;
    *elems = p->lift_elems;
    return SELR_OK;
}

extern "C" selr_status selr_plan_rank_sums(selr_plan *p, int64_t *out, int32_t n, int32_t *iterations,
                                           selr_stream stream) {
    if (!p || !out || n != p->gs.total) return SELR_ERR_INVALID_ARG;
    if (!p->rank_acc) return SELR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(out, p->rank_acc, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (iterations) *iterations = p->rank_iters;
    return SELR_OK;
}

// ------------------------------------------------------------ reverse mode
static selr_status grad_workspace(selr_plan *p) {
    if (p->gw_Z) return SELR_OK;
    const size_t lb = sizeof(cf) * (size_t)p->lift_elems;
    const bool jac = p->d.svd_method == SELR_SVD_JACOBI;
    // s x s scratch fits in s x len (s <= len).  Jacobi path: [B; I] needs s (len + s) <= 2 s len.
    // Eigensolver path: packed Gram / Householder storage, tridiagonals, and the
    // tridiagonal-basis eigenvectors (s x s floats per matrix).
    // Buffers already allocated by an earlier, partly failed call are kept.
    struct { void **ptr; size_t bytes; bool need; } req[] = {
        {(void **)&p->gw_Bbar, lb, true}, {(void **)&p->gw_S1, lb, true}, {(void **)&p->gw_V, lb, true},
        {(void **)&p->gw_Zo, lb, true},
        {(void **)&p->gw_lam, sizeof(float) * (size_t)p->vec_elems, true},
        {(void **)&p->gw_part, sizeof(double) * 512, true},
        // Jacobi path: batched s x s products and [B; I]
        {(void **)&p->gw_S2, lb, jac}, {(void **)&p->gw_S3, lb, jac}, {(void **)&p->gw_S4, lb, jac},
        {(void **)&p->gw_aug, 2 * lb, jac}, {(void **)&p->gw_aug2, 2 * lb, jac},
        // eigensolver path: eigen data and the low-rank slots
        {(void **)&p->gw_Gp, sizeof(cf) * (size_t)p->packed_elems, !jac},
        {(void **)&p->gw_tri, 4 * sizeof(float) * (size_t)p->vec_elems, !jac},
        {(void **)&p->gw_rank, sizeof(int) * (size_t)p->gs.total, !jac},
        {(void **)&p->gw_zs, sizeof(float) * (size_t)p->lift_elems, !jac},
        {(void **)&p->gw_U, lb, !jac}, {(void **)&p->gw_Gv, lb, !jac}, {(void **)&p->gw_W, 2 * lb, !jac},
        {(void **)&p->gw_Yv, 2 * lb, !jac}, {(void **)&p->gw_C11, lb, !jac}, {(void **)&p->gw_M2, lb, !jac},
        {(void **)&p->gw_X, lb, !jac}, {(void **)&p->gw_Ab, lb, !jac},
        {(void **)&p->gw_tpart, sizeof(double) * (size_t)p->gs.total, !jac},
        {(void **)&p->gw_Z, lb, true},     // last: marks the workspace as complete
    };
    for (auto &r : req) {
        if (!r.need || *r.ptr) continue;
        const selr_status s = alloc(p, r.ptr, r.bytes);
        if (s != SELR_OK) return s;
    }
    return SELR_OK;
}

extern "C" selr_status selr_svt_vjp(selr_plan *p, const void *A, const void *Zbar, int32_t nmat, int32_t rows,
                                    int32_t cols, float thresh, void *Abar, float *tbar, void *Z_out,
                                    selr_stream stream) {
    NvtxRange nvtx_range("selr_svt_vjp");
    if (!p || !A || !Zbar || !Abar || !tbar || nmat < 1 || rows < 1 || cols < 1 || !(thresh >= 0.f) ||
        !isfinite(thresh))
        return SELR_ERR_INVALID_ARG;
    GroupSet gs;
    memset(&gs, 0, sizeof(gs));
    gs.n = 1;
    Group &g = gs.g[0];
    g.kind = G_ROW;
    g.nmat = nmat;
    g.rows = rows;
    g.cols = cols;
    g.trans = cols > rows ? 1 : 0;
    g.s = g.trans ? rows : cols;
    g.len = g.trans ? cols : rows;
    g.thresh = thresh;
    finish_set(&gs);
    const int n = g.s, len = g.len;
    if (len > 512 || n > 480) return SELR_ERR_SHAPE;
    if ((long long)nmat * rows * cols > p->lift_elems || (long long)nmat * n > p->vec_elems || nmat > p->gs.total)
        return SELR_ERR_SHAPE;
    selr_status ws = grad_workspace(p);
    if (ws != SELR_OK) return ws;
    cudaStream_t st = (cudaStream_t)stream;
    // Bt (vector-major: row q of Bt is column q of B) and Zbar in the same layout
    CK(launch_natural_to_vm(gs, (const cf *)A, p->gw_S1, nullptr, st));
    CK(launch_natural_to_vm(gs, (const cf *)Zbar, p->gw_Z, nullptr, st));
    const long long sbl = (long long)n * len, ss = (long long)n * n;
    const cf one = mk(1.f, 0.f), zero = mk(0.f, 0.f);
    cf *Vt = p->gw_V;
    if (p->d.svd_method == SELR_SVD_JACOBI) {
        const long long sv = ss;        // batch stride of the compact Vt (row stride n)
        // every eigenpair of G = B^H B by one-sided Jacobi on [B; I]
        GroupSet ga = gs;
        ga.g[0].len = len + n;
        ga.g[0].dlen = len;
        CK(launch_augment(nmat, n, len, p->gw_S1, p->gw_aug, st));
        SvtArgs ja;
        memset(&ja, 0, sizeof(ja));
        ja.W = p->gw_aug;
        ja.sigma = p->sigma;
        ja.mat_status = p->mat_status;
        ja.status = p->status;
        ja.max_sweeps = p->d.jacobi_max_sweeps;
        ja.tol = p->d.jacobi_tol;
        CK(launch_jacobi(ga, 0, nmat, ja, st));
        const long long La = (long long)len + n, sa = (long long)n * La;
        // one polar step: Aug2^T = (1.5 I - 0.5 Q^H Q)^T Aug^T (rows of Aug^T are the columns)
        CK(launch_cgemm(nmat, n, n, n, mk(-0.5f, 0.f), p->gw_aug + len, 3, La, sa, p->gw_aug + len, 1, La, sa,
                        zero, p->gw_S2, n, ss, st));
        CK(launch_add_diag(nmat, n, p->gw_S2, ss, 1.5f, st));
        CK(launch_cgemm(nmat, n, (int)La, n, one, p->gw_S2, 1, n, ss, p->gw_aug, 0, La, sa, zero, p->gw_aug2, La,
                        sa, st));
        CK(launch_split_aug(nmat, n, len, p->gw_aug2, Vt, p->gw_lam, st));
        cf *Bt = p->gw_S1;
        // C = B^H Zbar = conj(Bt) Zt^T
        CK(launch_cgemm(nmat, n, n, len, one, Bt, 3, len, sbl, p->gw_Z, 1, len, sbl, zero, p->gw_S2, n, ss, st));
        // Ct = V^H C V = conj(Vt) C Vt^T
        CK(launch_cgemm(nmat, n, n, n, one, Vt, 3, n, sv, p->gw_S2, 0, n, ss, zero, p->gw_S3, n, ss, st));
        CK(launch_cgemm(nmat, n, n, n, one, p->gw_S3, 0, n, ss, Vt, 1, n, sv, zero, p->gw_S4, n, ss, st));
        CK(launch_tbar(nmat, n, p->gw_lam, thresh, p->gw_S4, ss, n, tbar, st));
        CK(launch_gamma(nmat, n, p->gw_lam, thresh, p->gw_S4, ss, n, st));
        // Gbar = V (Gamma o Ct) V^H = Vt^T S4 conj(Vt); then Gbar + Gbar^H
        CK(launch_cgemm(nmat, n, n, n, one, Vt, 1, n, sv, p->gw_S4, 0, n, ss, zero, p->gw_S2, n, ss, st));
        CK(launch_cgemm(nmat, n, n, n, one, p->gw_S2, 0, n, ss, Vt, 3, n, sv, zero, p->gw_S3, n, ss, st));
        CK(launch_herm_sum(nmat, n, p->gw_S3, ss, st));
        // h(G) = V h(Lambda) V^H = Vt^T conj(h o Vt)
        CK(launch_scale_vecs(nmat, n, p->gw_lam, thresh, Vt, p->gw_S4, sv, n, 0, st));
        CK(launch_cgemm(nmat, n, n, n, one, Vt, 1, n, sv, p->gw_S4, 3, n, sv, zero, p->gw_S2, n, ss, st));
        // Bbar^T = h(G)^T Zt + (Gbar + Gbar^H)^T Bt
        CK(launch_cgemm(nmat, n, len, n, one, p->gw_S2, 1, n, ss, p->gw_Z, 0, len, sbl, zero, p->gw_Bbar, len, sbl, st));
        CK(launch_cgemm(nmat, n, len, n, one, p->gw_S3, 1, n, ss, Bt, 0, len, sbl, one, p->gw_Bbar, len, sbl, st));
        if (Z_out) {
            // S_t(B)^T = h(G)^T Bt
            CK(launch_cgemm(nmat, n, len, n, one, p->gw_S2, 1, n, ss, Bt, 0, len, sbl, zero, p->gw_Zo, len, sbl, st));
            CK(launch_vm_to_natural(gs, p->gw_Zo, (cf *)Z_out, st));
        }
        CK(launch_vm_to_natural(gs, p->gw_Bbar, (cf *)Abar, st));
        return SELR_OK;
    } else {
        // the eigenpairs above t^2 only (as in selr_svt), with their tridiagonal-basis
        // vectors kept for the resolvent solves; then the low-rank form of the derivative
        if ((long long)nmat * n * (n + 1) / 2 > p->packed_elems) return SELR_ERR_SHAPE;
        EigArgs ea;
        memset(&ea, 0, sizeof(ea));
        ea.B0 = p->gw_S1;
        ea.Gp = p->gw_Gp;
        ea.lam = p->gw_lam;
        ea.V = Vt;
        ea.rank = p->gw_rank;
        ea.tri = p->gw_tri;
        ea.status = p->status;
        ea.zsave = p->gw_zs;
        CK(launch_gram(gs, 0, nmat, p->gw_S1, p->gw_Gp, nullptr, st));
        CK(launch_heig(gs, 0, nmat, ea, st));
        LrBuffers lb2;
        lb2.U = p->gw_U; lb2.Gv = p->gw_Gv; lb2.W = p->gw_W; lb2.Y = p->gw_Yv;
        lb2.C11 = p->gw_C11; lb2.M2 = p->gw_M2; lb2.X = p->gw_X; lb2.Ab = p->gw_Ab; lb2.tpart = p->gw_tpart;
        CK(launch_lowrank_vjp(gs, nmat, p->gw_S1, p->gw_Z, Vt, p->gw_lam, p->gw_rank, thresh, lb2, tbar, p->gw_Bbar,
                              Z_out ? p->gw_Zo : nullptr, ea, st));
        if (Z_out) CK(launch_vm_to_natural(gs, p->gw_Zo, (cf *)Z_out, st));
        CK(launch_vm_to_natural(gs, p->gw_Bbar, (cf *)Abar, st));
        return SELR_OK;
    }
}

extern "C" selr_status selr_dc_vjp(selr_plan *p, const uint8_t *mask, const void *Kbar, void *adj_out, void *Ybar,
                                   selr_stream stream) {
    if (!p || !mask || !Kbar || !adj_out) return SELR_ERR_INVALID_ARG;
    if (p->n_inst != 1 || p->spirit) return SELR_ERR_UNSUPPORTED;
    DcArgs a;
    memset(&a, 0, sizeof(a));
    a.model2d = p->model2d;
    a.L = p->L; a.J = p->J; a.M = p->M; a.N = p->N;
    a.mask = mask;
    a.da = p->inst[0].da; a.db = p->inst[0].db;
    a.lambda = p->d.lambda;
    a.beta = p->d.beta;
    CK(launch_dc_vjp(a, (const cf *)Kbar, (cf *)adj_out, (cf *)Ybar, (cudaStream_t)stream));
    return SELR_OK;
}

extern "C" selr_status selr_axpby(int64_t n, float a, const void *x, float b, const void *y, float c, const void *z,
                                  void *out, selr_stream stream) {
    if (n < 0 || !x || !out) return SELR_ERR_INVALID_ARG;
    CK(launch_axpbypcz(n, a, (const cf *)x, b, (const cf *)y, c, (const cf *)z, (cf *)out, (cudaStream_t)stream));
    return SELR_OK;
}

extern "C" selr_status selr_dot_re(selr_plan *p, int64_t n, const void *x, const void *y, float *out,
                                   selr_stream stream) {
    if (!p || n < 0 || !x || !y || !out) return SELR_ERR_INVALID_ARG;
    selr_status ws = grad_workspace(p);
    if (ws != SELR_OK) return ws;
    CK(launch_dot_re(n, (const cf *)x, (const cf *)y, p->gw_part, out, (cudaStream_t)stream));
    return SELR_OK;
}

// ---------------------------------------------------------------- autotuning
// Times a short solve (2 iterations, graph-captured when the plan is batched and
// the stream is not the legacy default stream) for every candidate setting on
// the caller's own data and keeps the fastest: the Gram precision among those
// with FP32-level accuracy (FP32, 3xTF32; one-pass TF32 only if flags bit 0),
// the inverse-iteration chunk (8 or 16 vectors per pass), and for the Jacobi
// method the sweep cap (twice the largest number of sweeps any matrix needed, + 2).
static selr_status time_solve(selr_plan *p, const void *Y, const uint8_t *mask, void *X, cudaStream_t st,
                              float *ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SELR_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SELR_ERR_CUDA; }
    selr_status s = selr_solve(p, Y, mask, X, nullptr, 0, nullptr, nullptr, (selr_stream)st);       // warm / capture
    float best = 3.4e38f;
    for (int rep = 0; rep < 2 && s == SELR_OK; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess) { s = SELR_ERR_CUDA; break; }
        s = selr_solve(p, Y, mask, X, nullptr, 0, nullptr, nullptr, (selr_stream)st);
        if (s != SELR_OK) break;
        float t = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) { s = SELR_ERR_CUDA; break; }
        best = t < best ? t : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return s;
}

extern "C" selr_status selr_plan_autotune(selr_plan *p, const void *Y, const uint8_t *mask, void *X_scratch,
                                          int32_t flags, selr_stream stream) {
    if (!p || !Y || !mask || !X_scratch) return SELR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int max_iter = p->d.max_iter;
    const float tol = p->d.tol;
    const int prof = p->prof_on;
    p->d.max_iter = 2;
    p->d.tol = -1.f;
    p->prof_on = 0;
    drop_graphs(p);
    selr_status s = SELR_OK;
    if (p->d.svd_method == SELR_SVD_JACOBI) {
        // sweep cap from the sweeps the matrices actually needed in two iterations
        s = selr_solve(p, Y, mask, X_scratch, nullptr, 0, nullptr, nullptr, stream);
        if (s == SELR_OK) {
            int *h = (int *)malloc(sizeof(int) * (size_t)p->gs.total);
            if (!h) s = SELR_ERR_ALLOC;
            else {
                if (cudaMemcpy(h, p->mat_status, sizeof(int) * (size_t)p->gs.total, cudaMemcpyDeviceToHost) !=
                    cudaSuccess)
                    s = SELR_ERR_CUDA;
                int mx = 0;
                bool capped = false;
                for (int i = 0; s == SELR_OK && i < p->gs.total; ++i) {
                    if (h[i] < 0) capped = true;
                    mx = h[i] > mx ? h[i] : mx;
                }
                // later iterations start further from convergence than none, but keep a margin
                if (s == SELR_OK && !capped && mx > 0 && 2 * mx + 2 < p->d.jacobi_max_sweeps)
                    p->d.jacobi_max_sweeps = 2 * mx + 2;
                free(h);
            }
        }
    } else {
        const int grams[5] = {SELR_GRAM_FP32, SELR_GRAM_3XTF32, SELR_GRAM_BF16X6, SELR_GRAM_TF32, SELR_GRAM_BF16X3};
        const int ngram = (flags & 1) ? 5 : 3;
        const int chunks[2] = {16, 8};
        float best = 3.4e38f;
        int bg = p->d.gram_precision, bc = p->ev_chunk;
        for (int gi = 0; gi < ngram && s == SELR_OK; ++gi) {
            for (int ci = 0; ci < 2 && s == SELR_OK; ++ci) {
                p->d.gram_precision = grams[gi];
                p->ev_chunk = chunks[ci];
                drop_graphs(p);
                float ms = 0.f;
                s = time_solve(p, Y, mask, X_scratch, st, &ms);
                if (s == SELR_OK && ms < best) { best = ms; bg = grams[gi]; bc = chunks[ci]; }
            }
        }
        p->d.gram_precision = bg;
        p->ev_chunk = bc;
        // the two-stage reduction where the plan has its scratch and the choice is left open
        if (s == SELR_OK && p->sb && p->reduction == 0) {
            p->reduction = 2;
            drop_graphs(p);
            float ms = 0.f;
            s = time_solve(p, Y, mask, X_scratch, st, &ms);
            if (s != SELR_OK || ms >= best) p->reduction = 0;
        }
    }
    drop_graphs(p);
    p->d.max_iter = max_iter;
    p->d.tol = tol;
    p->prof_on = prof;
    if (s == SELR_OK) p->tuned = 1;
    return s;
}

extern "C" selr_status selr_plan_tuning(const selr_plan *p, int32_t *gram_precision, int32_t *ev_chunk,
                                        int32_t *jacobi_max_sweeps) {
    if (!p) return SELR_ERR_INVALID_ARG;
    if (gram_precision) *gram_precision = p->d.gram_precision;
    if (ev_chunk) *ev_chunk = p->ev_chunk;
    if (jacobi_max_sweeps) *jacobi_max_sweeps = p->d.jacobi_max_sweeps;
    return SELR_OK;
}

extern "C" selr_status selr_plan_set_tuning(selr_plan *p, int32_t gram_precision, int32_t ev_chunk) {
    if (!p) return SELR_ERR_INVALID_ARG;
    if (gram_precision != SELR_GRAM_FP32 && gram_precision != SELR_GRAM_TF32 && gram_precision != SELR_GRAM_3XTF32 &&
        gram_precision != SELR_GRAM_BF16X3 && gram_precision != SELR_GRAM_BF16X6)
        return SELR_ERR_INVALID_ARG;
    if (ev_chunk != 0 && ev_chunk != 8 && ev_chunk != 16) return SELR_ERR_INVALID_ARG;
    p->d.gram_precision = gram_precision;
    p->ev_chunk = ev_chunk;
    drop_graphs(p);
    return SELR_OK;
}

extern "C" selr_status selr_plan_get_reduction(const selr_plan *p, int32_t *mode) {
    if (!p || !mode) return SELR_ERR_INVALID_ARG;
    *mode = p->reduction;
    return SELR_OK;
}

extern "C" selr_status selr_plan_set_reduction(selr_plan *p, int32_t mode) {
    if (!p || mode < 0 || mode > 2) return SELR_ERR_INVALID_ARG;
    p->reduction = mode;
    drop_graphs(p);
    return SELR_OK;
}

extern "C" selr_status selr_set_iterations(selr_plan *p, int32_t max_iter, float tol) {
    if (!p || max_iter < 1 || !isfinite(tol)) return SELR_ERR_INVALID_ARG;
    p->d.max_iter = max_iter;
    p->d.tol = tol;
    return SELR_OK;
}

extern "C" selr_status selr_profile_enable(selr_plan *p, int32_t on) {
    if (!p) return SELR_ERR_INVALID_ARG;
    p->prof_on = on ? 1 : 0;
    return SELR_OK;
}

extern "C" selr_status selr_profile_read(selr_plan *p, int32_t stage, float *total_ms, int32_t *count) {
    if (!p || stage < 0 || stage >= NSTAGE || !total_ms) return SELR_ERR_INVALID_ARG;
    float tot = 0.f;
    int n = 0;
    for (int it = 0; it < p->prof_count; ++it) {
        const cudaEvent_t a = p->ev[((size_t)it * NSTAGE + stage) * 2];
        const cudaEvent_t b = p->ev[((size_t)it * NSTAGE + stage) * 2 + 1];
        if (cudaEventSynchronize(b) != cudaSuccess) return SELR_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return SELR_ERR_CUDA;
        tot += ms;
        ++n;
    }
    *total_ms = tot;
    if (count) *count = n;
    return SELR_OK;
}

extern "C" selr_status selr_selftest_wait(int32_t set_flag, int32_t limit_us) {
    if (limit_us < 1 || limit_us > 2000000 || (set_flag != 0 && set_flag != 1)) return SELR_ERR_INVALID_ARG;
    unsigned *d = nullptr;                     // [0] flag, [1] status
    if (cudaMalloc(&d, 2 * sizeof(unsigned)) != cudaSuccess) {
        g_last_error = cudaGetLastError();
        return SELR_ERR_ALLOC;
    }
    const unsigned init[2] = {(unsigned)set_flag, 0u};
    unsigned h[2] = {0u, 0u};
    cudaError_t e = cudaMemcpy(d, init, sizeof(init), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_wait_selftest(d, d + 1, (unsigned long long)limit_us * 1000ull, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        g_last_error = e;
        return SELR_ERR_CUDA;
    }
    if (h[1] & ST_TIMEOUT) return SELR_ERR_TIMEOUT;
    return h[0] == 0u ? SELR_OK : SELR_ERR_CUDA;    // a consumed flag is cleared
}

extern "C" selr_status selr_sync_status(selr_plan *p, selr_stream stream) {
    if (!p) return SELR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SELR_ERR_CUDA;
    unsigned h = 0;
    if (cudaMemcpy(&h, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return SELR_ERR_CUDA;
    if (cudaMemset(p->status, 0, sizeof(unsigned)) != cudaSuccess) return SELR_ERR_CUDA;
    if (h & ST_TIMEOUT) return SELR_ERR_TIMEOUT;
    if (h & ST_NONFINITE) return SELR_ERR_NONFINITE;
    if (h & ST_NOCONV) return SELR_ERR_NO_CONVERGENCE;
    return SELR_OK;
}
