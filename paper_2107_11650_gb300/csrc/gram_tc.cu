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
// (the dropped a_l.b_l term is 2^-22 relative).  BF16 keeps 7 stored mantissa
// bits (kind::f16 with both operands bf16, K = 16 per MMA, at twice the TF32
// rate).  mode 4 (BF16x3): x = x_h + x_l, x_h = bf16(x), x_l = bf16(x - x_h),
// three products as above: the dropped terms and the rounding of x_l leave
// ~2^-16 relative.  mode 6 (BF16x6): x = x_h + x_m + x_l (each the bf16 of the
// remainder), the six products a_i.b_j with i + j <= 4 (indices 1..3), FP32
// level.  x - x_h is exact in FP32 in every split.
//
// Kernel.  One CTA (8 warps) per matrix, s <= 256, N = s rounded up to 16.
// s <= 192: one pass over K with two accumulator pairs in tensor memory,
// rows 0..127 x N columns and rows 128.. x columns 128..N-1 (the block below
// tile 0 is the conjugate transpose of tile 0's right part), 2N + 2(N - 128) <=
// 512 columns.  s > 192: two passes (rows 0..127, then 128..255) against all N
// columns.  K in chunks of 16 real elements, double-buffered in shared memory
// in three stages in the canonical K-major layout without swizzle (core matrices of 8 rows x 16
// bytes; LBO = 128 bytes between core matrices along K, SBO = 512 bytes between
// 8-row groups).  Each thread converts 4-element quads (one 16-byte store per
// tile) while its loads of the next chunk are in flight; one thread issues
// the MMAs (M = 128, K = 8) and commits them to the stage's mbarrier, which
// the threads wait on before refilling that stage.  Every wait is bounded: on expiry the kernel
// sets ST_TIMEOUT, waits (bounded) for its MMAs in flight, frees its tensor
// memory and returns.
#include "selr_internal.cuh"

#define GT_THREADS 256           // 8 warps convert; warp w reads TMEM lane quarter w % 4
#define GT_NS 3                  // shared-memory stages
#define GT_KC 16                  // real K elements per chunk (64 bytes per row)
#define GT_TILE_ROWS 256          // rows held per operand tile (s <= 256)
#define GT_TILE_BYTES (GT_TILE_ROWS * GT_KC * 4)   // 16 KB (TF32; a BF16 tile takes half)
#define GT_STAGE_BYTES (4 * GT_TILE_BYTES)         // Xh, Xl, Yh, Yl (BF16x6: six 8 KB tiles)
#define GT_SMEM (GT_NS * GT_STAGE_BYTES + 1024)    // stages + alignment slack
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

// The same layout for 16-bit elements: a row of a chunk is 32 bytes, two core
// matrices (8 rows x 8 elements) along K.
__device__ __forceinline__ uint32_t gb_off(int r, int k) {
    return (uint32_t)(((r >> 3) * (GT_KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), fixed
// constant 0b001 at bits 46-48, no swizzle.  LBO = 128 bytes between core
// matrices along K; SBO = bytes between 8-row groups (512 for TF32 chunks,
// 256 for BF16 chunks).
template <bool BF>
__device__ __forceinline__ uint64_t gt_desc(uint32_t addr) {
    const uint64_t lbo = 128 >> 4, sbo = (BF ? GT_KC / 8 * 128 : GT_KC / 4 * 128) >> 4;
    return (uint64_t)((addr & 0x3FFFF) >> 4) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Instruction descriptor, D F32 (bits 4-5 = 1), both operands K-major, N >> 3
// at bits 17-22, M >> 4 at 24-28; A and B types at bits 7-9 and 10-12:
// kind::tf32 TF32 = 2, kind::f16 BF16 = 1 (A and B always of the same type).
template <bool BF>
__device__ __forceinline__ uint32_t gt_idesc(int M, int N) {
    const uint32_t ty = BF ? 1u : 2u;
    return (1u << 4) | (ty << 7) | (ty << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <bool BF>
__device__ __forceinline__ void gt_mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if (BF)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// Two floats to a bf16 pair (round to nearest even), element lo in the low half.
__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
// (a, b) -> (b, -a) on a bf16 pair: swap the halves, flip the sign of the new high half.
__device__ __forceinline__ uint32_t bf_rot(uint32_t w) { return __byte_perm(w, 0, 0x1032) ^ 0x80000000u; }

__device__ __forceinline__ void st2(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
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

// 16-byte shared store of four 32-bit words.
__device__ __forceinline__ void st4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// Reads 16 tensor-memory columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// Issue the products of one K step (8 TF32 or 16 BF16 elements) into accumulator
// pair (dre, dim): A rows at byte offset arow, B rows at brow, tiles at k-offset
// ko.  x[t] / y[t]: the tiles of split term t of X and of its rotation Y.
template <int MODE>
__device__ __forceinline__ void gt_step(uint32_t dre, uint32_t dim, uint32_t idesc, const uint32_t *x,
                                        const uint32_t *y, uint32_t arow, uint32_t brow, uint32_t ko,
                                        uint32_t first) {
    constexpr bool BF = MODE >= 4;
    // products a_i . b_j of the split terms: (0,0), then (0,1), (1,0), then (0,2), (1,1), (2,0)
    constexpr int NP = MODE == 1 ? 1 : (MODE == 6 ? 6 : 3);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int i = (q == 2 || q == 4) ? 1 : (q == 5 ? 2 : 0);
        const int j = (q == 1 || q == 4) ? 1 : (q == 3 ? 2 : 0);
        const uint64_t a = gt_desc<BF>(x[i] + arow + ko);
        const uint32_t acc = q == 0 ? first : 1u;
        gt_mma<BF>(dre, a, gt_desc<BF>(x[j] + brow + ko), idesc, acc);
        gt_mma<BF>(dim, a, gt_desc<BF>(y[j] + brow + ko), idesc, acc);
    }
}

#define GT_QPR (GT_KC / 4)                                   // 4-element quads per row and chunk
#define GT_QPT (GT_TILE_ROWS * GT_QPR / GT_THREADS)          // quads per thread (4)

template <int MODE>
__global__ void __launch_bounds__(GT_THREADS, 1)
k_gram_tc(GroupSet gs, int mat_begin, const cf *B0, cf *Gp, const int *active, unsigned *status, unsigned *ready) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    __shared__ __align__(8) uint64_t bars[GT_NS];
    __shared__ uint32_t tmem_base_s;
    unsigned char *gsm = (unsigned char *)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    pdl_release_dependents();
    if (active) {
        if (g.kind == G_PE && active[g.aoff + mat / g.L] == 0) return;
        if (g.kind == G_PARAM && active[g.aoff + mat / g.N] == 0) return;
    }
    const int n = g.s, len = g.len, K = 2 * len;
    const int N = (n + 15) & ~15;                  // MMA N (multiple of 16 for M = 128)
    const int nk = (K + GT_KC - 1) / GT_KC;
    // N <= 192: one pass over K; tile 0 = rows 0..127 x all N columns, tile 1 = rows
    // 128.. x columns 128..N-1 (its columns < 128 are the conjugates of tile 0's).
    // N > 192: two passes, rows 0..127 then 128..255, each against all N columns.
    const bool single = N <= 192;
    const int npass = single ? 1 : 2;
    const int N1 = (single && N > 128) ? N - 128 : 0;
    const int rows = N > 128 ? 256 : 128;          // rows staged per chunk (zero beyond n)
    const int nq = rows * GT_QPR;
    const float *X = (const float *)(B0 + g.off + (long long)mat * n * len);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base_s))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < GT_NS; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = tmem_base_s;
    const uint32_t d0_re = tm, d0_im = tm + (uint32_t)N;
    const uint32_t d1_re = tm + 2u * N, d1_im = tm + 2u * N + (uint32_t)N1;
    constexpr bool BF = MODE >= 4;
    constexpr int NT = MODE == 1 ? 1 : (MODE == 6 ? 3 : 2);          // split terms
    constexpr uint32_t TILE = BF ? GT_TILE_BYTES / 2 : GT_TILE_BYTES;
    const uint32_t idesc0 = gt_idesc<BF>(128, N), idesc1 = N1 ? gt_idesc<BF>(128, N1) : 0u;
    const uint32_t rowgrp = BF ? GT_KC / 8 * 128 : GT_KC / 4 * 128;   // bytes per 8-row group (SBO)
    uint32_t waits[GT_NS] = {};                    // completed waits per stage (parity)
    bool ok = true;
    cf *G = Gp + g.poff + (long long)mat * ((long long)n * (n + 1) / 2);
    float2 pa[GT_QPT], pb[GT_QPT];                 // prefetched quads of the next chunk
    auto gload = [&](int kc) {
#pragma unroll
        for (int u = 0; u < GT_QPT; ++u) {
            const int idx = tid + GT_THREADS * u;
            const int r = idx / GT_QPR, q = idx - r * GT_QPR;
            const int k = kc * GT_KC + 4 * q;
            pa[u] = make_float2(0.f, 0.f);
            pb[u] = make_float2(0.f, 0.f);
            if (idx < nq && r < n) {
                const float *xr = X + (long long)r * K;
                if (k < K) pa[u] = *(const float2 *)(xr + k);
                if (k + 2 < K) pb[u] = *(const float2 *)(xr + k + 2);
            }
        }
    };
    for (int pass = 0; pass < npass && ok; ++pass) {
        gload(0);
        for (int kc = 0; kc < nk && ok; ++kc) {
            const int st = kc % GT_NS;
            unsigned char *stage = gsm + st * GT_STAGE_BYTES;
            if (kc >= GT_NS) {
                // every thread waits, then the block agrees on the outcome (no divergent exits)
                const bool w_ok = gt_wait(smem_u32(&bars[st]), waits[st] & 1);
                ++waits[st];
                if (!__syncthreads_and(w_ok)) { ok = false; break; }
            }
            float2 ca[GT_QPT], cb[GT_QPT];
#pragma unroll
            for (int u = 0; u < GT_QPT; ++u) { ca[u] = pa[u]; cb[u] = pb[u]; }
            if (kc + 1 < nk) gload(kc + 1);            // next chunk's loads in flight meanwhile
            // tiles of the split terms of X (x[t]) and of the rotation Y (y[t])
            uint32_t xt[3], yt[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                xt[t] = smem_u32(stage) + (uint32_t)t * TILE;
                yt[t] = smem_u32(stage) + (uint32_t)(NT + t) * TILE;
            }
#pragma unroll
            for (int u = 0; u < GT_QPT; ++u) {
                const int idx = tid + GT_THREADS * u;
                if (idx >= nq) continue;
                const int r = idx / GT_QPR, q = idx - r * GT_QPR;
                // (re0, im0, re1, im1) and the rotation (im0, -re0, im1, -re1)
                if (!BF) {
                    const uint32_t off = gt_off(r, 4 * q);
                    const uint32_t h0 = to_tf32(ca[u].x), h1 = to_tf32(ca[u].y);
                    const uint32_t h2 = to_tf32(cb[u].x), h3 = to_tf32(cb[u].y);
                    st4(xt[0] + off, h0, h1, h2, h3);
                    st4(yt[0] + off, h1, h0 ^ 0x80000000u, h3, h2 ^ 0x80000000u);
                    if (MODE == 3) {
                        const uint32_t l0 = to_tf32(ca[u].x - __uint_as_float(h0));
                        const uint32_t l1 = to_tf32(ca[u].y - __uint_as_float(h1));
                        const uint32_t l2 = to_tf32(cb[u].x - __uint_as_float(h2));
                        const uint32_t l3 = to_tf32(cb[u].y - __uint_as_float(h3));
                        st4(xt[1] + off, l0, l1, l2, l3);
                        st4(yt[1] + off, l1, l0 ^ 0x80000000u, l3, l2 ^ 0x80000000u);
                    }
                } else {
                    const uint32_t off = gb_off(r, 4 * q);
                    float ra = ca[u].x, ia = ca[u].y, rb = cb[u].x, ib = cb[u].y;   // remainders
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        const uint32_t w0 = to_bf16x2(ra, ia), w1 = to_bf16x2(rb, ib);
                        st2(xt[t] + off, w0, w1);
                        st2(yt[t] + off, bf_rot(w0), bf_rot(w1));
                        ra -= bf_lo(w0); ia -= bf_hi(w0); rb -= bf_lo(w1); ib -= bf_hi(w1);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // TF32: two K = 8 steps (two core matrices each); BF16: one K = 16 step
#pragma unroll
                for (int k8 = 0; k8 < (BF ? 1 : GT_KC / 8); ++k8) {
                    const uint32_t ko = (uint32_t)k8 * 2 * 128;
                    const uint32_t first = (kc == 0 && k8 == 0) ? 0u : 1u;
                    if (single) {
                        gt_step<MODE>(d0_re, d0_im, idesc0, xt, yt, 0u, 0u, ko, first);
                        if (N1) gt_step<MODE>(d1_re, d1_im, idesc1, xt, yt, 16u * rowgrp, 16u * rowgrp, ko, first);
                    } else {
                        gt_step<MODE>(d0_re, d0_im, idesc0, xt, yt, (uint32_t)pass * 16u * rowgrp, 0u, ko, first);
                    }
                }
                gt_commit(smem_u32(&bars[st]));
            }
        }
        if (!ok) break;
        // drain: the chunks of this pass not waited for yet
        bool d_ok = true;
        for (int kc = nk >= GT_NS ? nk - GT_NS : 0; kc < nk; ++kc) {
            const int st = kc % GT_NS;
            d_ok = gt_wait(smem_u32(&bars[st]), waits[st] & 1) && d_ok;
            ++waits[st];
        }
        if (!__syncthreads_and(d_ok)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // warp w reads lane quarter w % 4 (rows) and every other group of 16 columns
        const int wq = warp & 3, wh = warp >> 2;
        const uint32_t lane_addr = (uint32_t)(wq * 32) << 16;
        {
            // tile 0 (single pass) or this pass's rows (two passes)
            const int a = (single ? 0 : pass * 128) + wq * 32 + lane;
            const int jmax = single ? N : min(N, pass * 128 + 128);
            for (int j0 = 16 * wh; j0 < jmax; j0 += 32) {
                uint32_t vr[16], vi[16];
                tm_ld16(d0_re + lane_addr + (uint32_t)j0, vr);
                tm_ld16(d0_im + lane_addr + (uint32_t)j0, vi);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (a < n) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int c = j0 + u;                          // value = G(a, c)
                        if (c >= n) continue;
                        const float re = __uint_as_float(vr[u]), im = __uint_as_float(vi[u]);
                        if (c <= a) G[(long long)c * (2 * n - c + 1) / 2 + (a - c)] = mk(re, im);
                        else if (single) G[(long long)a * (2 * n - a + 1) / 2 + (c - a)] = mk(re, -im);
                    }
                }
            }
        }
        if (single && N1) {
            const int a = 128 + wq * 32 + lane;
            for (int j0 = 16 * wh; j0 < N1; j0 += 32) {
                uint32_t vr[16], vi[16];
                tm_ld16(d1_re + lane_addr + (uint32_t)j0, vr);
                tm_ld16(d1_im + lane_addr + (uint32_t)j0, vi);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (a < n) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int c = 128 + j0 + u;                    // value = G(a, c)
                        if (c < n && c <= a)
                            G[(long long)c * (2 * n - c + 1) / 2 + (a - c)] =
                                mk(__uint_as_float(vr[u]), __uint_as_float(vi[u]));
                    }
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
        for (int st = 0; st < GT_NS; ++st) gt_wait(smem_u32(&bars[st]), waits[st] & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm) : "memory");
    publish_flag(flag_of(ready, g, mat));
}

static bool g_gt_attr = false;

bool gram_tc_fits(const Group &g) { return g.s >= 1 && g.s <= 256 && g.len >= 1; }

cudaError_t launch_gram_tc(const GroupSet &gs, int mat_begin, int mat_count, const cf *B0, cf *Gp,
                           const int *active, int mode, unsigned *status, unsigned *ready, cudaStream_t st) {
    if (mat_count <= 0) return cudaSuccess;
    for (int k = 0; k < gs.n; ++k)
        if (!gram_tc_fits(gs.g[k])) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (!g_gt_attr) {
        e = cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_tc<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
        if (e != cudaSuccess) return e;
        g_gt_attr = true;
    }
    if (mode == 3) k_gram_tc<3><<<mat_count, GT_THREADS, GT_SMEM, st>>>(gs, mat_begin, B0, Gp, active, status, ready);
    else if (mode == 4) k_gram_tc<4><<<mat_count, GT_THREADS, GT_SMEM, st>>>(gs, mat_begin, B0, Gp, active, status, ready);
    else if (mode == 6) k_gram_tc<6><<<mat_count, GT_THREADS, GT_SMEM, st>>>(gs, mat_begin, B0, Gp, active, status, ready);
    else k_gram_tc<1><<<mat_count, GT_THREADS, GT_SMEM, st>>>(gs, mat_begin, B0, Gp, active, status, ready);
    return cudaGetLastError();
}
