// Peak-rate probe for the roofline denominators (a measurement utility, not
// part of the reconstruction): the FP32 FMA rate of this GPU, measured with
// independent FMA chains on every SM.
#include "selr_internal.cuh"

#define PROBE_THREADS 256
#define PROBE_CTAS_PER_SM 8
#define PROBE_CHAINS 16

// Each thread runs PROBE_CHAINS independent chains x <- x a + b (scalar FFMA,
// or packed FFMA2 with two lanes per chain).  The result is stored only if it
// equals a value it never takes, so the work cannot be removed.
template <bool PACKED>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(float *out, int iters, float a, float b) {
    float s = 0.f;
    if (PACKED) {
        float2 x[PROBE_CHAINS / 2];
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS / 2; ++k) x[k] = make_float2(1e-3f * threadIdx.x + k, 0.5f * k);
        const float2 av = make_float2(a, a), bv = make_float2(b, b);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS / 2; ++k) x[k] = __ffma2_rn(x[k], av, bv);
        }
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS / 2; ++k) s += x[k].x + x[k].y;
    } else {
        float x[PROBE_CHAINS];
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = 1e-3f * threadIdx.x + k;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    }
    if (s == -1234.5f) out[0] = s;
}

extern "C" selr_status selr_probe_fp32_peak(int32_t packed, int32_t iters, float *tflops_out, float *ms_out) {
    if (!tflops_out || iters < 1 || iters > (1 << 20) || (packed != 0 && packed != 1)) return SELR_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return SELR_ERR_CUDA;
    }
    float *out = nullptr;
    if (cudaMalloc((void **)&out, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return SELR_ERR_ALLOC;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    selr_status st = SELR_OK;
    const dim3 grid(sms * PROBE_CTAS_PER_SM);
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = SELR_ERR_CUDA;
    for (int rep = 0; rep < 2 && st == SELR_OK; ++rep) {    // the first launch warms the clocks up
        if (cudaEventRecord(e0, 0) != cudaSuccess) { st = SELR_ERR_CUDA; break; }
        if (packed) k_fma_probe<true><<<grid, PROBE_THREADS>>>(out, iters, 0.999f, 1e-3f);
        else k_fma_probe<false><<<grid, PROBE_THREADS>>>(out, iters, 0.999f, 1e-3f);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, 0) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = SELR_ERR_CUDA;
    }
    if (st == SELR_OK) {
        const double flops = (double)grid.x * PROBE_THREADS * PROBE_CHAINS * 2.0 * iters;
        *tflops_out = (float)(flops / (ms * 1e-3) / 1e12);
        if (ms_out) *ms_out = ms;
    } else {
        cudaGetLastError();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
