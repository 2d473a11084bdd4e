// Batched centred unitary 1D DFT (Sec. III-A: F^1D, F^PE, F^2D as two passes).
//
// F x = fftshift(fft(ifftshift(x))) / sqrt(n) for even n.  With
// e^{-2 pi i (k - n/2)(m - n/2)/n} = e^{-2 pi i k m / n} (-1)^k (-1)^m (-1)^{n/2},
// the centred transform is a plain DFT of (-1)^m x[m] followed by a
// multiplication of output k by (-1)^{k + n/2} / sqrt(n).
//
// The DFT itself is a Stockham autosort FFT (radices 4, 2, 3, 5) run in shared
// memory on a tile of FFT_V vectors per CTA.  Vectors along a strided axis are
// tiled across the contiguous axis so global loads and stores coalesce.
#include "selr_internal.cuh"

#include <math.h>
#include <stdlib.h>

#define FFT_V 8
#define FFT_THREADS 256
#define FFT_MAX_N 1024

static bool fft_factor(int n, FftTable *t) {
    if (n < 2 || (n & 1)) return false;
    int m = n, k = 0;
    const int order[4] = {4, 2, 3, 5};
    for (int oi = 0; oi < 4; ++oi) {
        const int R = order[oi];
        while (m % R == 0) {
            if (k >= 24) return false;
            t->radix[k++] = R;
            m /= R;
        }
    }
    if (m != 1) return false;
    t->n = n;
    t->nst = k;
    return true;
}

cudaError_t fft_table_build(int n, FftTable *t, cf **tw_dev) {
    if (n > FFT_MAX_N || !fft_factor(n, t)) return cudaErrorInvalidValue;
    cf *h = (cf *)malloc(sizeof(cf) * n);
    if (!h) return cudaErrorMemoryAllocation;
    for (int k = 0; k < n; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)n;
        h[k] = mk((float)cos(a), (float)sin(a));
    }
    cf *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(cf) * n);
    if (e == cudaSuccess) e = cudaMemcpy(d, h, sizeof(cf) * n, cudaMemcpyHostToDevice);
    free(h);
    if (e != cudaSuccess) {
        if (d) cudaFree(d);
        return e;
    }
    t->tw = d;
    *tw_dev = d;
    return cudaSuccess;
}

// R-point DFT in registers: y[q] = sum_r v[r] exp(-+ 2 pi i r q / R).
template <int R>
__device__ __forceinline__ void small_dft(cf *v, int inverse) {
    if (R == 2) {
        cf a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        cf a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        cf c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        // d * (-i) for forward, d * (+i) for inverse
        cf dr = inverse ? mk(-d.y, d.x) : mk(d.y, -d.x);
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, dr);
        v[3] = csub(b, dr);
    } else if (R == 3) {
        const float c1 = -0.5f, s1 = 0.86602540378443864676f;   // cos, sin of 2 pi / 3
        const float s = inverse ? s1 : -s1;
        cf a = v[0], b = v[1], c = v[2];
        cf t = cadd(b, c), u = csub(b, c);
        v[0] = cadd(a, t);
        cf m1 = mk(a.x + c1 * t.x, a.y + c1 * t.y);
        cf m2 = mk(-s * u.y, s * u.x);                             // i * s * u
        v[1] = cadd(m1, m2);
        v[2] = csub(m1, m2);
    } else {  // R == 5
        const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
        const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
        const float sg = inverse ? 1.f : -1.f;
        cf a = v[0];
        cf t1 = cadd(v[1], v[4]), u1 = csub(v[1], v[4]);
        cf t2 = cadd(v[2], v[3]), u2 = csub(v[2], v[3]);
        v[0] = cadd(a, cadd(t1, t2));
        cf r1 = mk(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
        cf r2 = mk(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
        // i * sg * (s1 u1 + s2 u2) and i * sg * (s2 u1 - s1 u2)
        cf q1 = mk(s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y);
        cf q2 = mk(s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y);
        cf i1 = mk(-sg * q1.y, sg * q1.x), i2 = mk(-sg * q2.y, sg * q2.x);
        v[1] = cadd(r1, i1);
        v[4] = csub(r1, i1);
        v[2] = cadd(r2, i2);
        v[3] = csub(r2, i2);
    }
}

template <int R>
__device__ __forceinline__ void stockham_stage(const cf *src, cf *dst, int n, int ld, int Ns,
                                               const cf *tw, int inverse) {
    const int nb = n / R;
    const int tstep0 = n / (Ns * R);
    for (int idx = threadIdx.x; idx < FFT_V * nb; idx += blockDim.x) {
        const int t = idx / nb, j = idx - t * nb;
        const int k = j % Ns;
        cf v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cf x = src[t * ld + j + r * nb];
            if (r > 0 && k > 0) {
                cf w = tw[r * k * tstep0];
                if (inverse) w = cconj(w);
                x = cmul(x, w);
            }
            v[r] = x;
        }
        small_dft<R>(v, inverse);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[t * ld + base + r * Ns] = v[r];
    }
}

__global__ void __launch_bounds__(FFT_THREADS) k_fft(const cf *in, cf *out, FftTable t,
                                                     long long outer, long long inner, int inverse) {
    extern __shared__ cf fsm[];
    const int n = t.n, ld = n + 1;
    cf *bufA = fsm, *bufB = fsm + FFT_V * ld;
    const long long nvec = outer * inner;
    const long long v0 = (long long)blockIdx.x * FFT_V;
    const float post = ((n >> 1) & 1 ? -1.f : 1.f) * rsqrtf((float)n);

    for (int idx = threadIdx.x; idx < FFT_V * n; idx += blockDim.x) {
        int tv, k;
        if (inner == 1) { tv = idx / n; k = idx - tv * n; }
        else { k = idx / FFT_V; tv = idx - k * FFT_V; }
        const long long v = v0 + tv;
        cf x = mk(0.f, 0.f);
        if (v < nvec) {
            const long long o = v / inner, i = v - o * inner;
            x = in[(o * n + k) * inner + i];
        }
        if (k & 1) x = mk(-x.x, -x.y);
        bufA[tv * ld + k] = x;
    }
    __syncthreads();
    cf *src = bufA, *dst = bufB;
    int Ns = 1;
    for (int st = 0; st < t.nst; ++st) {
        const int R = t.radix[st];
        if (R == 4) stockham_stage<4>(src, dst, n, ld, Ns, t.tw, inverse);
        else if (R == 2) stockham_stage<2>(src, dst, n, ld, Ns, t.tw, inverse);
        else if (R == 3) stockham_stage<3>(src, dst, n, ld, Ns, t.tw, inverse);
        else stockham_stage<5>(src, dst, n, ld, Ns, t.tw, inverse);
        __syncthreads();
        cf *tmp = src; src = dst; dst = tmp;
        Ns *= R;
    }
    for (int idx = threadIdx.x; idx < FFT_V * n; idx += blockDim.x) {
        int tv, k;
        if (inner == 1) { tv = idx / n; k = idx - tv * n; }
        else { k = idx / FFT_V; tv = idx - k * FFT_V; }
        const long long v = v0 + tv;
        if (v < nvec) {
            const long long o = v / inner, i = v - o * inner;
            const float s = (k & 1) ? -post : post;
            out[(o * n + k) * inner + i] = cscale(src[tv * ld + k], s);
        }
    }
}

// ---- compile-time lengths: the same transform with the radix schedule, the strides and every
// index division fixed at compile time (the lengths of the workloads; others use k_fft).
__host__ __device__ constexpr int fft_radix_at(int n, int s) {
    const int order[4] = {4, 2, 3, 5};
    int m = n, k = 0;
    for (int oi = 0; oi < 4; ++oi)
        while (m % order[oi] == 0) {
            if (k == s) return order[oi];
            ++k;
            m /= order[oi];
        }
    return 0;
}
__host__ __device__ constexpr int fft_nstages(int n) {
    int k = 0;
    while (fft_radix_at(n, k) != 0) ++k;
    return k;
}

template <int N, int R, int NS>
__device__ __forceinline__ void stockham_stage_c(const cf *src, cf *dst, const cf *tw, int inverse) {
    constexpr int nb = N / R, tstep0 = N / (NS * R), ld = N + 1;
    for (int idx = threadIdx.x; idx < FFT_V * nb; idx += FFT_THREADS) {
        const int t = idx / nb, j = idx - t * nb;
        const int k = j % NS;
        cf v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cf x = src[t * ld + j + r * nb];
            if (r > 0 && k > 0) {
                cf w = tw[r * k * tstep0];
                if (inverse) w = cconj(w);
                x = cmul(x, w);
            }
            v[r] = x;
        }
        small_dft<R>(v, inverse);
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[t * ld + base + r * NS] = v[r];
    }
}

// Stages S.. of length N (NS = product of the radices before S); returns the buffer that holds
// the result.
template <int N, int S, int NS>
__device__ __forceinline__ cf *fft_stages(cf *src, cf *dst, const cf *tw, int inverse) {
    if constexpr (S < fft_nstages(N)) {
        constexpr int R = fft_radix_at(N, S);
        stockham_stage_c<N, R, NS>(src, dst, tw, inverse);
        __syncthreads();
        return fft_stages<N, S + 1, NS * R>(dst, src, tw, inverse);
    } else {
        return src;
    }
}

template <int N>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_n(const cf *in, cf *out, const cf *tw, unsigned nvec,
                                                       unsigned inner, int inverse) {
    extern __shared__ cf fsm[];
    constexpr int ld = N + 1;
    cf *bufA = fsm, *bufB = fsm + FFT_V * ld;
    const unsigned v0 = blockIdx.x * FFT_V;
    const float post = ((N >> 1) & 1 ? -1.f : 1.f) * rsqrtf((float)N);
    for (int idx = threadIdx.x; idx < FFT_V * N; idx += FFT_THREADS) {
        int tv, k;
        if (inner == 1) { tv = idx / N; k = idx - tv * N; }
        else { k = idx / FFT_V; tv = idx - k * FFT_V; }
        const unsigned v = v0 + tv;
        cf x = mk(0.f, 0.f);
        if (v < nvec) {
            const unsigned o = v / inner, i = v - o * inner;
            x = in[((long long)o * N + k) * inner + i];
        }
        if (k & 1) x = mk(-x.x, -x.y);
        bufA[tv * ld + k] = x;
    }
    __syncthreads();
    const cf *res = fft_stages<N, 0, 1>(bufA, bufB, tw, inverse);
    for (int idx = threadIdx.x; idx < FFT_V * N; idx += FFT_THREADS) {
        int tv, k;
        if (inner == 1) { tv = idx / N; k = idx - tv * N; }
        else { k = idx / FFT_V; tv = idx - k * FFT_V; }
        const unsigned v = v0 + tv;
        if (v < nvec) {
            const unsigned o = v / inner, i = v - o * inner;
            const float sc = (k & 1) ? -post : post;
            out[((long long)o * N + k) * inner + i] = cscale(res[tv * ld + k], sc);
        }
    }
}

#define FFT_SIZES(X) X(64) X(128) X(160) X(192) X(240) X(256) X(288) X(320) X(384) X(480) X(512)

// Called once per process before the first launch (plan creation).
cudaError_t fft_init_attributes() {
    const int mx = (int)(sizeof(cf) * 2 * FFT_V * (FFT_MAX_N + 1));
    cudaError_t e = cudaFuncSetAttribute(k_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
#define FFT_ATTR(n) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft_n<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    FFT_SIZES(FFT_ATTR)
#undef FFT_ATTR
    return e;
}

cudaError_t launch_fft(const cf *in, cf *out, const FftTable &t, long long outer, long long inner,
                       int inverse, cudaStream_t st) {
    const long long nvec = outer * inner;
    if (nvec == 0) return cudaSuccess;
    const size_t smem = sizeof(cf) * 2 * FFT_V * (t.n + 1);
    const long long grid = (nvec + FFT_V - 1) / FFT_V;
    if (nvec < (1ll << 31) && inner < (1ll << 31)) {
        switch (t.n) {
#define FFT_CASE(n) \
            case n: \
                k_fft_n<n><<<(unsigned)grid, FFT_THREADS, smem, st>>>(in, out, t.tw, (unsigned)nvec, (unsigned)inner, \
                                                                      inverse); \
                return cudaGetLastError();
            FFT_SIZES(FFT_CASE)
#undef FFT_CASE
            default:
                break;
        }
    }
    k_fft<<<(unsigned)grid, FFT_THREADS, smem, st>>>(in, out, t, outer, inner, inverse);
    return cudaGetLastError();
}
