// Gram matrices G = B^H B on the 5th-generation tensor cores (tcgen05, TF32
// operands, FP32 accumulation in tensor memory): the precision option of the
// SVT's first step (Eqs. 16-17 need the eigenpairs of G).
//
// Real form.  Row i of the vector-major storage is column b_i of B, complex
// interleaved: read as real numbers it is x_i = (Re b_i0, Im b_i0, Re b_i1, ...)
// of length K = 2 len.  With y_j the rotated copy (Im b_j0, -Re b_j0, ...),
//     Re G_ij = x_i . x_j,      Im G_ij = x_i . y_j,
// so G comes from two real products X X^T and X Y^T with K = 2 len, and X is
// the stored array itself.
//
// Precision.  TF32 keeps 10 mantissa bits.  mode 1 (TF32): one product per
// term.  mode 3 (3xTF32): x = x_h + x_l with x_h = tf32(x), x_l = tf32(x - x_h)
// and a.b ~ a_h.b_h + a_h.b_l + a_l.b_h, which recovers about FP32 accuracy
// (the dropped a_l.b_l term is 2^-22 relative).
//
// Kernel.  One CTA (4 warps) per matrix, s <= 256.  Accumulators: D_re and
// D_im, 128 lanes x N columns each (N = s rounded up to 16), in 2N <= 512
// tensor-memory columns.  Rows are processed in M-tiles of 128; K in chunks of
// 16 real elements, double-buffered in shared memory in the canonical K-major
// layout without swizzle (core matrices of 8 rows x 16 bytes; LBO = 128 bytes
// between core matrices along K, SBO = 512 bytes between 8-row groups).  All
// threads convert and store a chunk; one thread issues the MMAs (M = 128,
// N, K = 8) and commits them to the stage's mbarrier, which the threads wait on
// before refilling that stage.  Every wait is bounded: on expiry the kernel
// sets ST_TIMEOUT, waits (bounded) for its MMAs in flight, frees its tensor
// memory and returns.
#include "selr_internal.cuh"

#define GT_THREADS 128
#define GT_KC 16                  // real K elements per chunk (64 bytes per row)
#define GT_TILE_ROWS 256          // rows held per operand tile (s <= 256)
#define GT_TILE_BYTES (GT_TILE_ROWS * GT_KC * 4)   // 16 KB
#define GT_STAGE_BYTES (4 * GT_TILE_BYTES)         // Xh, Xl, Yh, Yl
#define GT_SMEM (2 * GT_STAGE_BYTES + 1024)        // two stages + alignment slack
#define GT_WAIT_NS 2000000000ull   // 2 s bound on any single wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Canonical K-major no-swizzle offset (bytes) of element (row r, k) in a tile
// whose rows hold GT_KC elements: core matrix (r / 8, k / 4) at
// ((r / 8) * (GT_KC / 4) + k / 4) * 128, then (r % 8) * 16 + (k % 4) * 4.
__device__ __forceinline__ uint32_t gt_off(int r, int k) {
    return (uint32_t)(((r >> 3) * (GT_KC / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), fixed
// constant 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t gt_desc(uint32_t addr) {
    const uint64_t lbo = 128 >> 4, sbo = (GT_KC / 4 * 128) >> 4;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__device__ __forceinline__ uint32_t gt_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void gt_mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void gt_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ uint64_t gt_now() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (at most GT_WAIT_NS) for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool gt_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gt_now();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (gt_now() - t0 > GT_WAIT_NS) return false;
    }
}

template <int MODE>
__global__ void __launch_bounds__(GT_THREADS, 1)
k_gram_tc(GroupSet gs, int mat_begin, const cf *B0, cf *Gp, const int *active, unsigned *status) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base_s;
    unsigned char *gsm = (unsigned char *)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    if (active) {
        if (g.kind == G_PE && active[mat / g.L] == 0) return;
        if (g.kind == G_PARAM && active[mat / g.N] == 0) return;
    }
    const int n = g.s, len = g.len, K = 2 * len;
    const int N = (n + 15) & ~15;                  // MMA N (multiple of 16 for M = 128)
    const int nk = (K + GT_KC - 1) / GT_KC;
    const int mtiles = (n + 127) / 128;
    const float *X = (const float *)(B0 + g.off + (long long)mat * n * len);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base_s))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = tmem_base_s;
    const uint32_t d_re = tm, d_im = tm + (uint32_t)N;
    const uint32_t idesc = gt_idesc(128, N);
    uint32_t waits[2] = {0u, 0u};                 // completed waits per stage (parity)
    bool ok = true;
    cf *G = Gp + g.poff + (long long)mat * ((long long)n * (n + 1) / 2);
    for (int mt = 0; mt < mtiles && ok; ++mt) {
        for (int kc = 0; kc < nk && ok; ++kc) {
            const int st = kc & 1;
            unsigned char *stage = gsm + st * GT_STAGE_BYTES;
            if (kc >= 2) {
                // every thread waits, then the block agrees on the outcome (no divergent exits)
                const bool w_ok = gt_wait(smem_u32(&bars[st]), waits[st] & 1);
                ++waits[st];
                if (!__syncthreads_and(w_ok)) { ok = false; break; }
            }
            // load, split and rotate chunk kc: complex pairs (k even)
            uint32_t *xh = (uint32_t *)stage, *xl = (uint32_t *)(stage + GT_TILE_BYTES);
            uint32_t *yh = (uint32_t *)(stage + 2 * GT_TILE_BYTES), *yl = (uint32_t *)(stage + 3 * GT_TILE_BYTES);
            const int rows = mtiles * 128 > N ? mtiles * 128 : N;     // rows referenced by A and B
            for (int idx = tid; idx < rows * (GT_KC / 2); idx += GT_THREADS) {
                const int r = idx / (GT_KC / 2), kp = idx - r * (GT_KC / 2);
                const int k = kc * GT_KC + 2 * kp;
                float re = 0.f, im = 0.f;
                if (r < n && k < K) {
                    const float2 v = *(const float2 *)(X + (long long)r * K + k);
                    re = v.x;
                    im = v.y;
                }
                const uint32_t hre = to_tf32(re), him = to_tf32(im);
                const uint32_t lre = MODE == 3 ? to_tf32(re - __uint_as_float(hre)) : 0u;
                const uint32_t lim = MODE == 3 ? to_tf32(im - __uint_as_float(him)) : 0u;
                const uint32_t o0 = gt_off(r, 2 * kp) >> 2, o1 = gt_off(r, 2 * kp + 1) >> 2;
                xh[o0] = hre; xh[o1] = him;
                yh[o0] = him; yh[o1] = hre ^ 0x80000000u;              // (Im, -Re)
                if (MODE == 3) {
                    xl[o0] = lre; xl[o1] = lim;
                    yl[o0] = lim; yl[o1] = lre ^ 0x80000000u;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t bxh = smem_u32(xh), bxl = smem_u32(xl), byh = smem_u32(yh), byl = smem_u32(yl);
                const uint32_t arow = (uint32_t)(mt * 128 / 8) * (GT_KC / 4 * 128);   // A rows mt*128..
#pragma unroll
                for (int k8 = 0; k8 < GT_KC / 8; ++k8) {
                    const uint32_t ko = (uint32_t)k8 * 2 * 128;                   // two core matrices
                    const uint32_t first = (kc == 0 && k8 == 0) ? 0u : 1u;
                    const uint64_t ah = gt_desc(bxh + arow + ko), al = gt_desc(bxl + arow + ko);
                    gt_mma(d_re, ah, gt_desc(bxh + ko), idesc, first);
                    gt_mma(d_im, ah, gt_desc(byh + ko), idesc, first);
                    if (MODE == 3) {
                        gt_mma(d_re, ah, gt_desc(bxl + ko), idesc, 1u);
                        gt_mma(d_im, ah, gt_desc(byl + ko), idesc, 1u);
                        gt_mma(d_re, al, gt_desc(bxh + ko), idesc, 1u);
                        gt_mma(d_im, al, gt_desc(byh + ko), idesc, 1u);
                    }
                }
                gt_commit(smem_u32(&bars[st]));
            }
        }
        if (!ok) break;
        // drain: the last one or two chunks of this M-tile
        bool d_ok = true;
        for (int kc = nk >= 2 ? nk - 2 : 0; kc < nk; ++kc) {
            const int st = kc & 1;
            d_ok = gt_wait(smem_u32(&bars[st]), waits[st] & 1) && d_ok;
            ++waits[st];
        }
        if (!__syncthreads_and(d_ok)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // accumulators -> packed lower triangle; thread owns row i, 16 columns per load
        const int i = mt * 128 + warp * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
        const int jmax = min(N, mt * 128 + 128);
        for (int j0 = 0; j0 < jmax; j0 += 16) {
            uint32_t vr[16], vi[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]),
                  "=r"(vr[7]), "=r"(vr[8]), "=r"(vr[9]), "=r"(vr[10]), "=r"(vr[11]), "=r"(vr[12]), "=r"(vr[13]),
                  "=r"(vr[14]), "=r"(vr[15])
                : "r"(d_re + lane_addr + (uint32_t)j0));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]),
                  "=r"(vi[7]), "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]), "=r"(vi[12]), "=r"(vi[13]),
                  "=r"(vi[14]), "=r"(vi[15])
                : "r"(d_im + lane_addr + (uint32_t)j0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (i < n) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int j = j0 + u;
                    if (j <= i) G[(long long)j * (2 * n - j + 1) / 2 + (i - j)] =
                        mk(__uint_as_float(vr[u]), __uint_as_float(vi[u]));
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok) {
        // ok is block-uniform here.  Let the MMAs already issued finish (bounded) before
        // the tensor memory is released; a commit that was never waited for is waited once.
        if (tid == 0) atomicOr(status, (unsigned)ST_TIMEOUT);
        for (int st = 0; st < 2; ++st) gt_wait(smem_u32(&bars[st]), waits[st] & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm) : "memory");
}

static bool g_gt_attr = false;

bool gram_tc_fits(const Group &g) { return g.s >= 1 && g.s <= 256 && g.len >= 1; }

cudaError_t launch_gram_tc(const GroupSet &gs, int mat_begin, int mat_count, const cf *B0, cf *Gp,
                           const int *active, int mode, unsigned *status, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    for (int k = 0; k < gs.n; ++k)
        if (!gram_tc_fits(gs.g[k])) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (!g_gt_attr) {
        e = cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
        if (e != cudaSuccess) return e;
        g_gt_attr = true;
    }
    if (mode == 3) k_gram_tc<3><<<mat_count, GT_THREADS, GT_SMEM, st>>>(gs, mat_begin, B0, Gp, active, status);
    else k_gram_tc<1><<<mat_count, GT_THREADS, GT_SMEM, st>>>(gs, mat_begin, B0, Gp, active, status);
    return cudaGetLastError();
}
