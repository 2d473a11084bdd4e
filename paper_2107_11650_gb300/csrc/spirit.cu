// SPIRiT (Eq. 3 / Eq. 6): calibration of the kernel from the ACS rows, and the
// X-update of SHLR-S / SHLR-SV (Eq. 15 with the lambda_1 (G - I)^* (G - I) term).
//
// G predicts every k-space sample of coil j from the samples of all coils in a
// ks x ks neighbourhood (the sample itself excluded):
//     (G K)_j[m, n] = sum_{j', a, b} g[j][j'][a][b] K_j'[m + a - h, n + b - h],   h = ks / 2,
// circular in k-space, hence a pixelwise J x J matrix in the image domain:
//     Ghat_jj'(r) = sqrt(M N) F2D(kernel g[j][j'] placed at (M/2 + a - h, N/2 + b - h))(r).
// Calibration: every kernel position inside the ACS block (the acs centre rows,
// all columns) gives one row of A (its J ks^2 neighbourhood samples); per target
// coil j, (A_-j^H A_-j + mu I) g_j = A_-j^H a_j with A_-j = A without the
// column of (j, centre), mu = reg trace(A_-j^H A_-j) / (J ks^2 - 1), in FP64
// (C = A^H A once, then one Cholesky per coil).
// X-update in k-space: (lambda U + beta d + lambda_1 F (Ghat - I)^H (Ghat - I) F*) K = lambda U Y
// + beta (transformed lift adjoints), by conjugate gradients preconditioned with
// the diagonal lambda U + beta d + lambda_1 c_j' (c_j' = 1 + sum_{j,a,b} |g[j][j'][a][b]|^2,
// the k-space diagonal of (G - I)^H (G - I)), a fixed number of iterations
// from the previous iterate.  The dot products reduce over a fixed grid into
// per-CTA partials that every consumer sums in the same order (deterministic);
// the CG scalars never leave the device, so the whole X-update can be captured
// in a CUDA graph.
#include "selr_internal.cuh"

#include <math.h>

#define SP_T 256
#define SP_GT 128
#define SP_ST 512
#define SP_MAXJ 32

__device__ __forceinline__ double2 dmulc(double2 a, double2 b) {     // conj(a) b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ------------------------------------------------------------ calibration
// C[q1][q2] = sum over kernel positions of conj(A[pos][q1]) A[pos][q2],
// q = j' ks^2 + a ks + b <-> Y[j'][m + a - h][n + b - h].  C is Hermitian: the entries
// q2 <= q1 are summed (the products of two FP32 values are exact in the FP64 FMAs) and
// mirrored, in two interleaved chains (even and odd n) added at the end.
__global__ void __launch_bounds__(SP_GT) k_sp_gram(const cf *Y, int J, int M, int N, int ks, int r0, int r1,
                                                   double2 *C) {
    const int nu = J * ks * ks, h = ks / 2;
    const int q1 = blockIdx.x, q2 = blockIdx.y * SP_GT + threadIdx.x;
    if (q2 > q1 || q2 >= nu) return;
    const int j1 = q1 / (ks * ks), a1 = (q1 / ks) % ks, b1 = q1 % ks;
    const int j2 = q2 / (ks * ks), a2 = (q2 / ks) % ks, b2 = q2 % ks;
    double ar0 = 0.0, ai0 = 0.0, ar1 = 0.0, ai1 = 0.0;
    for (int m = r0 + h; m < r1 - h; ++m) {
        const cf *y1 = Y + ((long long)j1 * M + (m + a1 - h)) * N + (b1 - h);
        const cf *y2 = Y + ((long long)j2 * M + (m + a2 - h)) * N + (b2 - h);
        int n = h;
        for (; n + 1 < N - h; n += 2) {
            const cf u0 = y1[n], v0 = y2[n], u1 = y1[n + 1], v1 = y2[n + 1];
            ar0 = fma((double)u0.x, (double)v0.x, fma((double)u0.y, (double)v0.y, ar0));
            ai0 = fma((double)u0.x, (double)v0.y, fma(-(double)u0.y, (double)v0.x, ai0));
            ar1 = fma((double)u1.x, (double)v1.x, fma((double)u1.y, (double)v1.y, ar1));
            ai1 = fma((double)u1.x, (double)v1.y, fma(-(double)u1.y, (double)v1.x, ai1));
        }
        if (n < N - h) {
            const cf u0 = y1[n], v0 = y2[n];
            ar0 = fma((double)u0.x, (double)v0.x, fma((double)u0.y, (double)v0.y, ar0));
            ai0 = fma((double)u0.x, (double)v0.y, fma(-(double)u0.y, (double)v0.x, ai0));
        }
    }
    const double2 acc = make_double2(ar0 + ar1, ai0 + ai1);
    C[(long long)q1 * nu + q2] = acc;
    C[(long long)q2 * nu + q1] = make_double2(acc.x, -acc.y);
}

// One CTA per target coil j0 + blockIdx.x: S = C without (t, t) row/column
// + mu I, Cholesky S = L L^H in place in `work`, then the two triangular
// solves; writes g[j][0..nu) (entry t = 0).
__global__ void __launch_bounds__(SP_ST) k_sp_solve(const double2 *C, int J, int ks, double reg, int j0,
                                                    double2 *work, cf *g, unsigned *status) {
    __shared__ double s_mu;
    __shared__ double2 s_x;
    const int nu = J * ks * ks, ns = nu - 1;
    const int j = j0 + blockIdx.x;
    if (j >= J) return;
    const int h = ks / 2, t = j * ks * ks + h * ks + h;
    double2 *S = work + (long long)blockIdx.x * ((long long)ns * ns + ns);
    double2 *x = S + (long long)ns * ns;
    auto src = [&](int i) { return i < t ? i : i + 1; };        // index in C of reduced index i
    double tr = 0.0;
    for (int i = threadIdx.x; i < ns; i += SP_ST) tr += C[(long long)src(i) * nu + src(i)].x;
    __shared__ double red[SP_ST];
    red[threadIdx.x] = tr;
    __syncthreads();
    for (int s = SP_ST / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_mu = reg * red[0] / ns;
    __syncthreads();
    const double mu = s_mu;
    for (long long e = threadIdx.x; e < (long long)ns * ns; e += SP_ST) {
        const int r = (int)(e / ns), c = (int)(e - (long long)r * ns);
        double2 v = C[(long long)src(r) * nu + src(c)];
        if (r == c) v.x += mu;
        S[e] = v;
    }
    for (int i = threadIdx.x; i < ns; i += SP_ST) x[i] = C[(long long)src(i) * nu + t];
    __syncthreads();
    // right-looking Cholesky (lower triangle, row-major S[r][c], c <= r)
    for (int k = 0; k < ns; ++k) {
        if (threadIdx.x == 0) {
            const double d = S[(long long)k * ns + k].x;
            if (!(d > 0.0)) atomicOr(status, (unsigned)ST_NONFINITE);
            S[(long long)k * ns + k] = make_double2(d > 0.0 ? sqrt(d) : 1.0, 0.0);
        }
        __syncthreads();
        const double dk = S[(long long)k * ns + k].x;
        for (int r = k + 1 + threadIdx.x; r < ns; r += SP_ST) {
            double2 v = S[(long long)r * ns + k];
            S[(long long)r * ns + k] = make_double2(v.x / dk, v.y / dk);
        }
        __syncthreads();
        // trailing lower triangle: warp per row r, lanes over its columns c <= r
        for (int r = k + 1 + (int)(threadIdx.x >> 5); r < ns; r += SP_ST / 32) {
            const double2 lr = S[(long long)r * ns + k];
            double2 *Sr = S + (long long)r * ns;
            for (int c = k + 1 + (int)(threadIdx.x & 31); c <= r; c += 32) {
                const double2 lc = S[(long long)c * ns + k];
                // S[r][c] -= L[r][k] conj(L[c][k])
                double2 v = Sr[c];
                v.x -= lr.x * lc.x + lr.y * lc.y;
                v.y -= lr.y * lc.x - lr.x * lc.y;
                Sr[c] = v;
            }
        }
        __syncthreads();
    }
    // L y = x (forward), L^H g = y (backward)
    for (int k = 0; k < ns; ++k) {
        if (threadIdx.x == 0) {
            const double dk = S[(long long)k * ns + k].x;
            s_x = make_double2(x[k].x / dk, x[k].y / dk);
            x[k] = s_x;
        }
        __syncthreads();
        const double2 yk = s_x;
        for (int r = k + 1 + threadIdx.x; r < ns; r += SP_ST) {
            const double2 l = S[(long long)r * ns + k];
            x[r].x -= l.x * yk.x - l.y * yk.y;
            x[r].y -= l.x * yk.y + l.y * yk.x;
        }
        __syncthreads();
    }
    for (int k = ns - 1; k >= 0; --k) {
        if (threadIdx.x == 0) {
            const double dk = S[(long long)k * ns + k].x;
            s_x = make_double2(x[k].x / dk, x[k].y / dk);
            x[k] = s_x;
        }
        __syncthreads();
        const double2 gk = s_x;
        for (int r = threadIdx.x; r < k; r += SP_ST) {
            const double2 l = S[(long long)k * ns + r];       // (L^H)[r][k] = conj(L[k][r])
            x[r].x -= l.x * gk.x + l.y * gk.y;
            x[r].y -= l.x * gk.y - l.y * gk.x;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < nu; i += SP_ST) {
        double2 v = i == t ? make_double2(0.0, 0.0) : x[i < t ? i : i - 1];
        if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(status, (unsigned)ST_NONFINITE);
        g[(long long)j * nu + i] = mk((float)v.x, (float)v.y);
    }
}

// Gm[j][j'] = kernel g[j][j'] placed at (M/2 + a - h, N/2 + b - h), zero elsewhere;
// cj[j'] = 1 + sum_{j, a, b} |g[j][j'][a][b]|^2.
__global__ void k_sp_place(const cf *g, int J, int M, int N, int ks, cf *Gm, float *cj) {
    const long long tot = (long long)J * J * M * N;
    const int h = ks / 2, kk = ks * ks;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long pl = e / ((long long)M * N);
        const int pix = (int)(e - pl * M * N), m = pix / N, n = pix - m * N;
        const int a = m - M / 2 + h, b = n - N / 2 + h;
        Gm[e] = (a >= 0 && a < ks && b >= 0 && b < ks) ? g[pl * kk + a * ks + b] : mk(0.f, 0.f);
    }
    if (blockIdx.x == 0) {
        for (int jp = threadIdx.x; jp < J; jp += blockDim.x) {
            double s = 1.0;
            for (int j = 0; j < J; ++j)
                for (int q = 0; q < kk; ++q) s += cabs2(g[((long long)j * J + jp) * kk + q]);
            cj[jp] = (float)s;
        }
    }
}

// Gm <- sqrt(M N) Gm - I (after the forward 2D transform of every plane).
__global__ void k_sp_finish_g(cf *Gm, int J, int M, int N) {
    const long long tot = (long long)J * J * M * N, MN = (long long)M * N;
    const float sc = sqrtf((float)M * (float)N);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long pl = e / MN;
        cf v = cscale(Gm[e], sc);
        if (pl / J == pl % J) v.x -= 1.f;
        Gm[e] = v;
    }
}

__global__ void k_sp_hpix(const cf *Gm, int J, long long MN, cf *Hm);

static int sp_blocks(long long n) { return (int)min((n + SP_T - 1) / SP_T, (long long)SP_NB); }

cudaError_t launch_spirit_calibrate(const SpiritArgs &s, const cf *Y, cudaStream_t st) {
    const int nu = s.J * s.ks * s.ks;
    const int r0 = s.M / 2 - s.acs / 2, r1 = r0 + s.acs;
    k_sp_gram<<<dim3(nu, (nu + SP_GT - 1) / SP_GT), SP_GT, 0, st>>>(Y, s.J, s.M, s.N, s.ks, r0, r1, s.cal_C);
    cudaError_t e = cudaGetLastError();
    for (int j0 = 0; j0 < s.J && e == cudaSuccess; j0 += SELR_SPIRIT_SLOTS) {
        const int ng = min(SELR_SPIRIT_SLOTS, s.J - j0);
        k_sp_solve<<<ng, SP_ST, 0, st>>>(s.cal_C, s.J, s.ks, (double)s.reg, j0, s.cal_work, s.g, s.status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const long long tot = (long long)s.J * s.J * s.M * s.N;
    k_sp_place<<<sp_blocks(tot), SP_T, 0, st>>>(s.g, s.J, s.M, s.N, s.ks, s.Gm, s.cj);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_fft(s.Gm, s.Gm, s.ftN, (long long)s.J * s.J * s.M, 1, 0, st)) != cudaSuccess) return e;
    if ((e = launch_fft(s.Gm, s.Gm, s.ftM, (long long)s.J * s.J, s.N, 0, st)) != cudaSuccess) return e;
    k_sp_finish_g<<<sp_blocks(tot), SP_T, 0, st>>>(s.Gm, s.J, s.M, s.N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long MN = (long long)s.M * s.N;
    k_sp_hpix<<<(int)min((MN + 127) / 128, (long long)152 * 16), 128, 0, st>>>(s.Gm, s.J, MN, s.Hm);
    return cudaGetLastError();
}

// ------------------------------------------------------------ CG X-update
// Every pixel: H = (Ghat - I)^H (Ghat - I), the J x J Hermitian operator of the SPIRiT term in
// the image domain, stored as its upper triangle (j1 <= j2, row by row) with pixels
// contiguous: Hm[idx][pix], idx = 0 .. J (J + 1) / 2 - 1.  Once per calibration.
__global__ void __launch_bounds__(128) k_sp_hpix(const cf *Gm, int J, long long MN, cf *Hm) {
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < MN; pix += (long long)gridDim.x * blockDim.x) {
        long long idx = 0;
        for (int j1 = 0; j1 < J; ++j1)
            for (int j2 = j1; j2 < J; ++j2, ++idx) {
                cf a = mk(0.f, 0.f);
                for (int j = 0; j < J; ++j)
                    a = cadd(a, cmulc(Gm[((long long)j * J + j1) * MN + pix], Gm[((long long)j * J + j2) * MN + pix]));
                Hm[idx * MN + pix] = a;
            }
    }
}

// Every pixel: t <- H t (J <= JM coils; the vectors in registers, each stored entry of H read
// once: H[j1][j2] v[j2] into u[j1] and conj(H[j1][j2]) v[j1] into u[j2]).
template <int JM>
__global__ void __launch_bounds__(128) k_sp_pix(cf *t, const cf *Hm, int J, long long MN) {
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < MN; pix += (long long)gridDim.x * blockDim.x) {
        cf v[JM], u[JM];
#pragma unroll
        for (int j = 0; j < JM; ++j) {
            v[j] = j < J ? t[(long long)j * MN + pix] : mk(0.f, 0.f);
            u[j] = mk(0.f, 0.f);
        }
        const cf *h = Hm + pix;
#pragma unroll
        for (int j1 = 0; j1 < JM; ++j1) {
            if (j1 < J) {
#pragma unroll
                for (int j2 = j1; j2 < JM; ++j2) {
                    if (j2 < J) {
                        const cf hv = *h;
                        h += MN;
                        u[j1] = cadd(u[j1], cmul(hv, v[j2]));
                        if (j2 != j1) u[j2] = cadd(u[j2], cmulc(hv, v[j1]));
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < JM; ++j)
            if (j < J) t[(long long)j * MN + pix] = u[j];
    }
}

// First kernel of an X-update: x = K (the CG starts from the previous iterate), and the
// diagonals of this solve per element i = (j M + m) N + n: dv = lambda U + beta (d_r(n) + d_c(m))
// and the preconditioner pdv = dv + lambda_1 c_j (32-bit index arithmetic: nK < 2^32).
__global__ void __launch_bounds__(SP_T) k_sp_begin(SpiritArgs s) {
    const unsigned MN = (unsigned)s.M * (unsigned)s.N;
    for (long long i = blockIdx.x * (long long)SP_T + threadIdx.x; i < s.nK; i += (long long)SP_NB * SP_T) {
        const unsigned ui = (unsigned)i, pix = ui % MN, j = ui / MN, m = pix / (unsigned)s.N;
        const unsigned n = pix - m * (unsigned)s.N;
        const float d = s.lambda * (s.mask[pix] ? 1.f : 0.f) + s.beta * (s.da[n] + s.db[m]);
        s.dv[i] = d;
        s.pdv[i] = d + s.lambda1 * s.cj[j];
        s.x[i] = s.K[i];
    }
}

// fixed-order sum of this CTA's values into part[blockIdx.x]
__device__ __forceinline__ void sp_partial(double v, double *part) {
    __shared__ double red[SP_T / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < SP_T / 32; ++k) s += red[k];
        part[blockIdx.x] = s;
    }
}

// Sum of the SP_NB per-CTA partials in one fixed order (lane l adds entries l, l + 32, ...,
// then a butterfly whose partners add the same two values), formed once per CTA by warp 0
// and broadcast through shared memory: every thread of every CTA gets the same bits.
__device__ __forceinline__ double sp_block_sum(const double *part, double *slot) {
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int k = threadIdx.x; k < SP_NB; k += 32) v += part[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *slot = v;
    }
    __syncthreads();
    return *slot;
}

// q = diag v + lambda_1 t; optional partial of Re <v, q>.
__global__ void __launch_bounds__(SP_T) k_sp_combine(SpiritArgs s, const cf *v, double *part) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)SP_T + threadIdx.x; i < s.nK; i += (long long)SP_NB * SP_T) {
        const cf vi = v[i], ti = s.t[i];
        const float d = s.dv[i];
        const cf qi = mk(d * vi.x + s.lambda1 * ti.x, d * vi.y + s.lambda1 * ti.y);
        s.q[i] = qi;
        acc += (double)vi.x * qi.x + (double)vi.y * qi.y;
    }
    if (part) sp_partial(acc, part);
}

// r = lambda U Y + beta (a + b) - q;  z = r / P;  p = z;  partial r.z
__global__ void __launch_bounds__(SP_T) k_sp_init(SpiritArgs s, double *part) {
    double acc = 0.0;
    const unsigned MN = (unsigned)s.M * (unsigned)s.N;
    for (long long i = blockIdx.x * (long long)SP_T + threadIdx.x; i < s.nK; i += (long long)SP_NB * SP_T) {
        const float u = s.mask[(unsigned)i % MN] ? 1.f : 0.f;
        const cf ab = cadd(s.adjA[i], s.adjB[i]), y = s.Y[i], qi = s.q[i];
        const cf ri = mk(s.lambda * u * y.x + s.beta * ab.x - qi.x, s.lambda * u * y.y + s.beta * ab.y - qi.y);
        const float pd = s.pdv[i];
        const cf zi = mk(ri.x / pd, ri.y / pd);
        s.r[i] = ri;
        s.z[i] = zi;
        s.p[i] = zi;
        acc += (double)ri.x * zi.x + (double)ri.y * zi.y;
    }
    sp_partial(acc, part);
}

// alpha = rz / pq;  x += alpha p;  r -= alpha q;  z = r / P;  partial of the new r.z
__global__ void __launch_bounds__(SP_T) k_sp_update(SpiritArgs s, const double *rz_old, const double *pq,
                                                    double *rz_new) {
    __shared__ double s_sums[2];
    const double den = sp_block_sum(pq, &s_sums[0]);
    const double num = sp_block_sum(rz_old, &s_sums[1]);
    const float alpha = den != 0.0 ? (float)(num / den) : 0.f;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)SP_T + threadIdx.x; i < s.nK; i += (long long)SP_NB * SP_T) {
        const cf pi = s.p[i], qi = s.q[i];
        cf xi = s.x[i], ri = s.r[i];
        xi = mk(xi.x + alpha * pi.x, xi.y + alpha * pi.y);
        ri = mk(ri.x - alpha * qi.x, ri.y - alpha * qi.y);
        const float pd = s.pdv[i];
        const cf zi = mk(ri.x / pd, ri.y / pd);
        s.x[i] = xi;
        s.r[i] = ri;
        s.z[i] = zi;
        acc += (double)ri.x * zi.x + (double)ri.y * zi.y;
    }
    sp_partial(acc, rz_new);
}

// p = z + (rz_new / rz_old) p
__global__ void __launch_bounds__(SP_T) k_sp_pupdate(SpiritArgs s, const double *rz_old, const double *rz_new) {
    __shared__ double s_sums[2];
    const double o = sp_block_sum(rz_old, &s_sums[0]);
    const double nw = sp_block_sum(rz_new, &s_sums[1]);
    const float bcg = o != 0.0 ? (float)(nw / o) : 0.f;
    for (long long i = blockIdx.x * (long long)SP_T + threadIdx.x; i < s.nK; i += (long long)SP_NB * SP_T) {
        const cf zi = s.z[i], pi = s.p[i];
        s.p[i] = mk(zi.x + bcg * pi.x, zi.y + bcg * pi.y);
    }
}

// Per row m: ||x - K||^2 and ||K||^2 over (j, n) in a fixed order (the partials of
// the stopping ratio, as the pointwise X-update writes them), then K = x.
__global__ void __launch_bounds__(SP_T) k_sp_finish(SpiritArgs s) {
    const int m = blockIdx.x;
    double d = 0.0, nn = 0.0;
    bool bad = false;
    for (int idx = threadIdx.x; idx < s.J * s.N; idx += SP_T) {
        const int j = idx / s.N, n = idx - j * s.N;
        const long long i = ((long long)j * s.M + m) * s.N + n;
        const cf k0 = s.K[i], x = s.x[i];
        if (!isfinite(x.x) || !isfinite(x.y)) bad = true;
        nn += (double)cabs2(k0);
        d += (double)cabs2(csub(x, k0));
        s.K[i] = x;
    }
    if (bad) atomicOr(s.status, (unsigned)ST_NONFINITE);
    __shared__ double red[2][SP_T / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = d; red[1][threadIdx.x >> 5] = nn; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < SP_T / 32; ++k) { a += red[0][k]; b += red[1][k]; }
        s.partial[2 * m] = a;
        s.partial[2 * m + 1] = b;
    }
}

// q = A v  (A = diag + lambda_1 F (Ghat - I)^H (Ghat - I) F*); partial Re <v, q> if part
static cudaError_t sp_apply(const SpiritArgs &s, const cf *v, double *part, cudaStream_t st) {
    cudaError_t e;
    if ((e = launch_fft(v, s.t, s.ftN, (long long)s.J * s.M, 1, 1, st)) != cudaSuccess) return e;
    if ((e = launch_fft(s.t, s.t, s.ftM, s.J, s.N, 1, st)) != cudaSuccess) return e;
    const long long MN = (long long)s.M * s.N;
    const int nb = (int)min((MN + 127) / 128, (long long)152 * 16);
    if (s.J <= 4) k_sp_pix<4><<<nb, 128, 0, st>>>(s.t, s.Hm, s.J, MN);
    else if (s.J <= 8) k_sp_pix<8><<<nb, 128, 0, st>>>(s.t, s.Hm, s.J, MN);
    else if (s.J <= 16) k_sp_pix<16><<<nb, 128, 0, st>>>(s.t, s.Hm, s.J, MN);
    else k_sp_pix<SP_MAXJ><<<nb, 128, 0, st>>>(s.t, s.Hm, s.J, MN);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_fft(s.t, s.t, s.ftN, (long long)s.J * s.M, 1, 0, st)) != cudaSuccess) return e;
    if ((e = launch_fft(s.t, s.t, s.ftM, s.J, s.N, 0, st)) != cudaSuccess) return e;
    k_sp_combine<<<SP_NB, SP_T, 0, st>>>(s, v, part);
    return cudaGetLastError();
}

cudaError_t launch_spirit_x_update(const SpiritArgs &s, cudaStream_t st) {
    cudaError_t e;
    double *rz0 = s.part, *rz1 = s.part + SP_NB, *pq = s.part + 2 * SP_NB;
    k_sp_begin<<<SP_NB, SP_T, 0, st>>>(s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = sp_apply(s, s.x, nullptr, st)) != cudaSuccess) return e;
    k_sp_init<<<SP_NB, SP_T, 0, st>>>(s, rz0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int it = 0; it < s.cg_iters; ++it) {
        double *ro = (it & 1) ? rz1 : rz0, *rn = (it & 1) ? rz0 : rz1;
        if ((e = sp_apply(s, s.p, pq, st)) != cudaSuccess) return e;
        k_sp_update<<<SP_NB, SP_T, 0, st>>>(s, ro, pq, rn);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (it + 1 < s.cg_iters) {
            k_sp_pupdate<<<SP_NB, SP_T, 0, st>>>(s, ro, rn);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    k_sp_finish<<<s.M, SP_T, 0, st>>>(s);
    return cudaGetLastError();
}
