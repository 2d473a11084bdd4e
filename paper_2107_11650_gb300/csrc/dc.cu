// X-update (Eq. 15 without the SPIRiT term; Eq. S7) as a pointwise divide in
// k-space, the relative-change reduction of the stopping rule (Algorithms S1 /
// S2), and small fill helpers.
//
//   K' = (lambda U Y + beta (a + b)) / (lambda U + beta (d_a + d_b))
// where a, b are the lift adjoints already transformed to k-space and d_a,
// d_b the diagonal normal operators of the lifts:
//   2D:    d_a = d_r(k_n), d_b = d_c(k_m),  d(k) = c(k)|w(k)|^2 [+ c(n-1-k)|w(n-1-k)|^2 (VC)]
//   param: d_a = d_pe(k_n), d_b = c_P(l)    (parameter lift: H*H = diag(c_P), no F, no W).
// lambda <= 0: hard data consistency (K' = Y where sampled).  A point with a
// zero left-hand side is unconstrained; it is set to 0 (minimum norm).
//
// One CTA per FE row m reduces ||K'-K||^2 and ||K||^2 over (l, j, k_n) in a
// fixed order, so the parameter models get per-m ratios and the 2D models the
// fixed-order sum over m: results are run-to-run deterministic.
#include "selr_internal.cuh"

#define DC_THREADS 256

__global__ void __launch_bounds__(DC_THREADS) k_dc(DcArgs a) {
    const int m = blockIdx.x;
    const int L = a.L, J = a.J, M = a.M, N = a.N;
    __shared__ double red[2][DC_THREADS / 32];
    const bool act = !a.active || a.active[m];
    double dsum = 0.0, nsum = 0.0;
    bool bad = false;
    const int per = L * J * N;
    for (int idx = threadIdx.x; idx < per; idx += DC_THREADS) {
        const int kn = idx % N;
        const int lj = idx / N;
        const int j = lj % J, l = lj / J;
        const long long i = (((long long)l * J + j) * M + m) * N + kn;
        const cf k0 = a.K[i];
        nsum += (double)cabs2(k0);
        if (!act) continue;
        const float u = a.mask[((long long)l * M + m) * N + kn] ? 1.f : 0.f;
        const cf ab = cadd(a.a[i], a.b[i]);
        const float dd = a.da[kn] + (a.model2d ? a.db[m] : a.db[l]);
        const cf y = a.Y[i];
        cf kn_;
        if (a.lambda > 0.f) {
            const float den = a.lambda * u + a.beta * dd;
            const float num_r = a.lambda * u * y.x + a.beta * ab.x;
            const float num_i = a.lambda * u * y.y + a.beta * ab.y;
            kn_ = den != 0.f ? mk(num_r / den, num_i / den) : mk(0.f, 0.f);
        } else {
            kn_ = u > 0.f ? y : (dd != 0.f ? mk(ab.x / dd, ab.y / dd) : mk(0.f, 0.f));
        }
        if (!isfinite(kn_.x) || !isfinite(kn_.y)) bad = true;
        const cf df = csub(kn_, k0);
        dsum += (double)cabs2(df);
        a.K[i] = kn_;
    }
    if (bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    // fixed-order block reduction
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = dsum; red[1][w] = nsum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d = 0.0, n = 0.0;
        for (int k = 0; k < DC_THREADS / 32; ++k) { d += red[0][k]; n += red[1][k]; }
        a.partial[2 * m] = d;
        a.partial[2 * m + 1] = n;
    }
}

cudaError_t launch_dc(const DcArgs &a, cudaStream_t st) {
    k_dc<<<a.M, DC_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

// rel[0] = sum_m d_m / sum_m n_m ; per_m: rel[1 + m] = d_m / n_m and
// active_next[m] &= !(rel_m < tol) when tol > 0.
__global__ void k_rel_finalize(const double *partial, int M, int per_m, float tol, float *rel, int *active_next) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double d = 0.0, n = 0.0;
        for (int m = 0; m < M; ++m) { d += partial[2 * m]; n += partial[2 * m + 1]; }
        rel[0] = n > 0.0 ? (float)(d / n) : 0.f;
    }
    if (per_m) {
        for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
            const double n = partial[2 * m + 1];
            const float r = n > 0.0 ? (float)(partial[2 * m] / n) : 0.f;
            rel[1 + m] = r;
            if (active_next && tol > 0.f && r < tol) active_next[m] = 0;
        }
    }
}

cudaError_t launch_rel_finalize(const double *partial, int M, int per_m, float tol, float *rel,
                                int *active_next, cudaStream_t st) {
    k_rel_finalize<<<(M + 255) / 256, 256, 0, st>>>(partial, M, per_m, tol, rel, active_next);
    return cudaGetLastError();
}

__global__ void k_fill(cf *p, long long n, cf v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_fill_i(int *p, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_copy_i(const int *s, int *d, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = s[i];
}

cudaError_t launch_fill(cf *p, long long n, cf v, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = min((n + 255) / 256, (long long)152 * 16);
    k_fill<<<(unsigned)blocks, 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}
cudaError_t launch_fill_i(int *p, long long n, int v, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = min((n + 255) / 256, (long long)152 * 16);
    k_fill_i<<<(unsigned)blocks, 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}
cudaError_t launch_copy_active(const int *src, int *dst, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_copy_i<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
