// Evaluation of reconstructions (Sec. IV and Supplement S3): SSOS coil
// combination, RLNE, MSSIM and the pixel-by-pixel T2 fit of parameter
// imaging.  Reductions run in one CTA in a fixed order (deterministic), so no
// entry point here needs device workspace beyond the caller's outputs.
#include "selr_internal.cuh"

#include <math.h>

#define MT_RED 1024
#define MS_WIN 11
#define MS_HALF 5
#define T2_MAXL 32
#define T2_ITERS 60

// ------------------------------------------------------------------ SSOS
// out[b][p] = sqrt(sum_j |X[b][j][p]|^2)
__global__ void k_ssos(const cf *X, int nb, int J, long long npix, float *out) {
    const long long tot = (long long)nb * npix;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / npix, p = i - b * npix;
        const cf *x = X + b * J * npix + p;
        float s = 0.f;
        for (int j = 0; j < J; ++j) s += cabs2(x[(long long)j * npix]);
        out[i] = sqrtf(s);
    }
}

extern "C" selr_status selr_ssos(const void *X, int32_t nb, int32_t J, int64_t npix, float *out, selr_stream stream) {
    if (!X || !out || nb < 1 || J < 1 || npix < 1) return SELR_ERR_INVALID_ARG;
    const long long tot = (long long)nb * npix;
    const int blocks = (int)min((tot + 255) / 256, (long long)152 * 8);
    k_ssos<<<blocks, 256, 0, (cudaStream_t)stream>>>((const cf *)X, nb, J, npix, out);
    return cudaGetLastError() == cudaSuccess ? SELR_OK : SELR_ERR_CUDA;
}

// Fixed-order block sum of one double (every thread gets the result).
__device__ double block_sum_d(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = MT_RED / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ RLNE
__global__ void __launch_bounds__(MT_RED) k_rlne(const float *x, const float *xh, long long n, float *out) {
    __shared__ double red[MT_RED];
    double num = 0.0, den = 0.0;
    for (long long i = threadIdx.x; i < n; i += MT_RED) {
        const double a = x[i], d = (double)x[i] - (double)xh[i];
        num += d * d;
        den += a * a;
    }
    num = block_sum_d(num, red);
    den = block_sum_d(den, red);
    if (threadIdx.x == 0) out[0] = den > 0.0 ? (float)sqrt(num / den) : 0.f;
}

extern "C" selr_status selr_rlne(const float *x, const float *xhat, int64_t n, float *out, selr_stream stream) {
    if (!x || !xhat || !out || n < 1) return SELR_ERR_INVALID_ARG;
    k_rlne<<<1, MT_RED, 0, (cudaStream_t)stream>>>(x, xhat, n, out);
    return cudaGetLastError() == cudaSuccess ? SELR_OK : SELR_ERR_CUDA;
}

// ----------------------------------------------------------------- MSSIM
struct MsWin {
    float w[MS_WIN * MS_WIN];
};

// One thread per valid window position (i, j): Gaussian-weighted means, then
// variances and covariance about them (two passes over the 121 taps).
__global__ void k_ssim_map(const float *A, const float *B, int M, int N, float C1, float C2, MsWin win, float *map) {
    const int Mv = M - MS_WIN + 1, Nv = N - MS_WIN + 1;
    const long long tot = (long long)Mv * Nv;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / Nv), j = (int)(q - (long long)i * Nv);
        float ma = 0.f, mb = 0.f;
        for (int u = 0; u < MS_WIN; ++u)
            for (int v = 0; v < MS_WIN; ++v) {
                const float w = win.w[u * MS_WIN + v];
                const long long o = (long long)(i + u) * N + (j + v);
                ma = fmaf(w, A[o], ma);
                mb = fmaf(w, B[o], mb);
            }
        float va = 0.f, vb = 0.f, cab = 0.f;
        for (int u = 0; u < MS_WIN; ++u)
            for (int v = 0; v < MS_WIN; ++v) {
                const float w = win.w[u * MS_WIN + v];
                const long long o = (long long)(i + u) * N + (j + v);
                const float da = A[o] - ma, db = B[o] - mb;
                va = fmaf(w, da * da, va);
                vb = fmaf(w, db * db, vb);
                cab = fmaf(w, da * db, cab);
            }
        map[q] = ((2.f * ma * mb + C1) * (2.f * cab + C2)) / ((ma * ma + mb * mb + C1) * (va + vb + C2));
    }
}

__global__ void __launch_bounds__(MT_RED) k_mean(const float *v, long long n, float *out) {
    __shared__ double red[MT_RED];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += MT_RED) s += v[i];
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) out[0] = (float)(s / (double)n);
}

__global__ void __launch_bounds__(MT_RED) k_max(const float *v, long long n, float *out) {
    __shared__ float red[MT_RED];
    float m = -INFINITY;
    for (long long i = threadIdx.x; i < n; i += MT_RED) m = fmaxf(m, v[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = MT_RED / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

extern "C" selr_status selr_mssim(const float *A, const float *B, int32_t M, int32_t N, float L, float *ssim_map,
                                  float *out, selr_stream stream) {
    if (!A || !B || !ssim_map || !out || M < MS_WIN || N < MS_WIN || !(L > 0.f) || !isfinite(L))
        return SELR_ERR_INVALID_ARG;
    MsWin win;
    double g[MS_WIN], gs = 0.0;
    for (int u = 0; u < MS_WIN; ++u) {
        const double r = (double)(u - MS_HALF) / 1.5;
        g[u] = exp(-0.5 * r * r);
    }
    for (int u = 0; u < MS_WIN; ++u)
        for (int v = 0; v < MS_WIN; ++v) gs += g[u] * g[v];
    for (int u = 0; u < MS_WIN; ++u)
        for (int v = 0; v < MS_WIN; ++v) win.w[u * MS_WIN + v] = (float)(g[u] * g[v] / gs);
    const float C1 = (0.01f * L) * (0.01f * L), C2 = (0.03f * L) * (0.03f * L);
    const long long tot = (long long)(M - MS_WIN + 1) * (N - MS_WIN + 1);
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)min((tot + 255) / 256, (long long)152 * 8);
    k_ssim_map<<<blocks, 256, 0, st>>>(A, B, M, N, C1, C2, win, ssim_map);
    if (cudaGetLastError() != cudaSuccess) return SELR_ERR_CUDA;
    k_mean<<<1, MT_RED, 0, st>>>(ssim_map, tot, out);
    return cudaGetLastError() == cudaSuccess ? SELR_OK : SELR_ERR_CUDA;
}

extern "C" selr_status selr_max(const float *v, int64_t n, float *out, selr_stream stream) {
    if (!v || !out || n < 1) return SELR_ERR_INVALID_ARG;
    k_max<<<1, MT_RED, 0, (cudaStream_t)stream>>>(v, n, out);
    return cudaGetLastError() == cudaSuccess ? SELR_OK : SELR_ERR_CUDA;
}

// ---------------------------------------------------------------- T2 fit
struct TeArgs {
    double te[T2_MAXL];
};

// One thread per pixel: log-linear start, then Levenberg-Marquardt on
// (M0, R2 = 1 / T2) for f = sum_l (M0 exp(-R2 TE_l) - S_l)^2, in FP64.
__global__ void k_t2_fit(const float *S, TeArgs ta, int L, long long npix, double t2min, double t2max, float *T2,
                         float *M0) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
        double s[T2_MAXL];
        bool pos = true;
        for (int l = 0; l < L; ++l) {
            s[l] = S[(long long)l * npix + p];
            pos = pos && s[l] > 0.0;
        }
        float t2o = nanf(""), m0o = nanf("");
        if (pos) {
            // log-linear least squares: log s = log m0 - r te
            double st = 0, sy = 0, stt = 0, sty = 0;
            for (int l = 0; l < L; ++l) {
                const double y = log(s[l]);
                st += ta.te[l]; sy += y; stt += ta.te[l] * ta.te[l]; sty += ta.te[l] * y;
            }
            const double den = L * stt - st * st;
            const double slope = den != 0.0 ? (L * sty - st * sy) / den : 0.0;
            double m = exp((sy - slope * st) / L);
            double r = slope < 0.0 ? -slope : 1.0 / t2max;
            auto cost = [&](double mm, double rr) {
                double c = 0.0;
                for (int l = 0; l < L; ++l) {
                    const double d = mm * exp(-rr * ta.te[l]) - s[l];
                    c += d * d;
                }
                return c;
            };
            double f = cost(m, r), mu = 1e-3;
            for (int it = 0; it < T2_ITERS; ++it) {
                double a11 = 0, a12 = 0, a22 = 0, g1 = 0, g2 = 0;
                for (int l = 0; l < L; ++l) {
                    const double e = exp(-r * ta.te[l]);
                    const double j1 = e, j2 = -m * ta.te[l] * e, res = m * e - s[l];
                    a11 += j1 * j1; a12 += j1 * j2; a22 += j2 * j2;
                    g1 += j1 * res; g2 += j2 * res;
                }
                bool moved = false;
                for (int tries = 0; tries < 8 && !moved; ++tries) {
                    const double b11 = a11 * (1.0 + mu), b22 = a22 * (1.0 + mu);
                    const double det = b11 * b22 - a12 * a12;
                    if (!(det > 0.0)) { mu *= 10.0; continue; }
                    const double dm = -(b22 * g1 - a12 * g2) / det, dr = -(b11 * g2 - a12 * g1) / det;
                    const double fn = cost(m + dm, r + dr);
                    if (fn <= f) {
                        m += dm; r += dr; f = fn;
                        mu = fmax(mu * 0.1, 1e-12);
                        moved = true;
                    } else {
                        mu *= 10.0;
                    }
                }
                if (!moved) break;
            }
            if (r > 0.0 && 1.0 / r >= t2min && 1.0 / r <= t2max) {
                t2o = (float)(1.0 / r);
                m0o = (float)m;
            }
        }
        T2[p] = t2o;
        if (M0) M0[p] = m0o;
    }
}

extern "C" selr_status selr_t2_fit(const float *S, const float *te_ms, int32_t L, int64_t npix, float t2_min,
                                   float t2_max, float *T2_out, float *M0_out, selr_stream stream) {
    if (!S || !te_ms || !T2_out || L < 2 || L > T2_MAXL || npix < 1 || !(t2_min > 0.f) || !(t2_max > t2_min))
        return SELR_ERR_INVALID_ARG;
    TeArgs ta;
    for (int l = 0; l < L; ++l) {
        if (!isfinite(te_ms[l])) return SELR_ERR_INVALID_ARG;
        ta.te[l] = te_ms[l];
    }
    const int blocks = (int)min((long long)((npix + 127) / 128), (long long)152 * 8);
    k_t2_fit<<<blocks, 128, 0, (cudaStream_t)stream>>>(S, ta, L, npix, t2_min, t2_max, T2_out, M0_out);
    return cudaGetLastError() == cudaSuccess ? SELR_OK : SELR_ERR_CUDA;
}
