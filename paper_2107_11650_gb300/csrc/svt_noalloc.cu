// selr_svt_noalloc: singular value thresholding of a batch of matrices that
// allocates no device memory.
//
// Some callers cannot allocate GPU memory once they are running: code that
// issues work while a CUDA stream is being captured into a graph (where a
// cudaMalloc is an error), real-time reconstruction services that reserve
// their whole memory budget up front, and host frameworks that own every
// device allocation through their own pool.  selr_svt needs a plan (which
// allocates its workspace) and so cannot serve them.  This entry point runs
// the same Jacobi SVT kernels on a fixed scratch area that lives in this
// translation unit as file-scope __device__ arrays: every GPU that loads the
// library holds it (about 17 MB) until the process exits.
//
// Host code cannot use the arrays' names as device addresses (in host code
// they are host-side stand-ins), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on it.  That first call should therefore come before any
// stream capture.  All calls on a device share the scratch, which keeps the
// previous call's contents; the status word is cleared on every call (and can
// be read back with selr_svt_noalloc_status), and calls that overlap on the
// GPU (different streams or host threads) race.
#include "selr_internal.cuh"

#include <math.h>
#include <mutex>
#include <string.h>

#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) cf g_na_work[SELR_SVT_NOALLOC_MAX_ELEMS];
static __device__ __align__(256) cf g_na_orig[SELR_SVT_NOALLOC_MAX_ELEMS];
static __device__ __align__(256) float g_na_sigma[SELR_SVT_NOALLOC_MAX_ELEMS / 4];
static __device__ __align__(256) int g_na_mat_status[SELR_SVT_NOALLOC_MAX_MATS];
static __device__ __align__(256) unsigned g_na_status[64];

struct NoallocPtrs {
    bool ready;
    cf *work, *orig;
    float *sigma;
    int *mat_status;
    unsigned *status;
};

static NoallocPtrs g_na_ptrs[NOALLOC_MAX_DEVICES];
static std::mutex g_na_lock;

// Per-device set-up on the current device: resolve the scratch addresses and
// opt the SVT kernels into large shared memory.  No allocation.
static selr_status noalloc_setup(int dev, NoallocPtrs *out) {
    std::lock_guard<std::mutex> guard(g_na_lock);
    NoallocPtrs &p = g_na_ptrs[dev];
    if (!p.ready) {
        NoallocPtrs q;
        memset(&q, 0, sizeof(q));
        if (cudaGetSymbolAddress((void **)&q.work, g_na_work) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&q.orig, g_na_orig) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&q.sigma, g_na_sigma) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&q.mat_status, g_na_mat_status) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&q.status, g_na_status) != cudaSuccess) {
            cudaGetLastError();
            return SELR_ERR_CUDA;
        }
        if (svt_init_attributes() != cudaSuccess) {
            cudaGetLastError();
            return SELR_ERR_CUDA;
        }
        q.ready = true;
        p = q;
    }
    *out = p;
    return SELR_OK;
}

extern "C" selr_status selr_svt_noalloc(void *A, int32_t nmat, int32_t rows, int32_t cols, float thresh,
                                        int32_t max_sweeps, float tol, int32_t *rank_out, selr_stream stream) {
    if (!A || nmat < 1 || rows < 1 || cols < 1 || !(thresh >= 0.f) || !isfinite(thresh) || max_sweeps < 1 ||
        !(tol > 0.f))
        return SELR_ERR_INVALID_ARG;
    const long long elems = (long long)nmat * rows * cols;
    const int s = rows < cols ? rows : cols, len = rows < cols ? cols : rows;
    if (elems > SELR_SVT_NOALLOC_MAX_ELEMS || nmat > SELR_SVT_NOALLOC_MAX_MATS || len > 512 || s > 1024 ||
        (long long)nmat * s > SELR_SVT_NOALLOC_MAX_ELEMS / 4)
        return SELR_ERR_SHAPE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return SELR_ERR_CUDA;
    }
    NoallocPtrs p;
    selr_status st = noalloc_setup(dev, &p);
    if (st != SELR_OK) return st;

    GroupSet gs;
    memset(&gs, 0, sizeof(gs));
    gs.n = 1;
    Group &g = gs.g[0];
    g.kind = G_ROW;
    g.nmat = nmat;
    g.rows = rows;
    g.cols = cols;
    g.trans = cols > rows ? 1 : 0;
    g.s = s;
    g.len = len;
    g.thresh = thresh;
    gs.start[0] = 0;
    gs.start[1] = nmat;
    gs.total = nmat;

    SvtArgs a;
    memset(&a, 0, sizeof(a));
    a.W = p.work;
    a.B0 = p.orig;
    a.sigma = p.sigma;
    a.mat_status = p.mat_status;
    a.status = p.status;
    a.max_sweeps = max_sweeps;
    a.tol = tol;
    a.mode = 0;
    a.Zout = (cf *)A;
    a.z_natural = 1;
    a.rank_out = rank_out;
    cudaStream_t cs = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(unsigned), cs) != cudaSuccess ||
        launch_natural_to_vm(gs, (const cf *)A, p.work, p.orig, cs) != cudaSuccess ||
        launch_jacobi(gs, 0, nmat, a, cs) != cudaSuccess || launch_svt_apply(gs, 0, nmat, a, cs) != cudaSuccess) {
        cudaGetLastError();
        return SELR_ERR_CUDA;
    }
    return SELR_OK;
}

extern "C" selr_status selr_svt_noalloc_status(selr_stream stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return SELR_ERR_CUDA;
    }
    NoallocPtrs p;
    selr_status st = noalloc_setup(dev, &p);
    if (st != SELR_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    unsigned h = 0;
    if (cudaMemcpyAsync(&h, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess) {
        cudaGetLastError();
        return SELR_ERR_CUDA;
    }
    if (h & ST_TIMEOUT) return SELR_ERR_TIMEOUT;
    if (h & ST_NONFINITE) return SELR_ERR_NONFINITE;
    if (h & ST_NOCONV) return SELR_ERR_NO_CONVERGENCE;
    return SELR_OK;
}
