// Hankel lift (Eq. 2, Eq. 4, Eq. 7/8) and its real adjoint (the L^T terms of
// Eq. 15 / S7).
//
// Lift:    A[mat][r][c] = w[r+q] v_ch[r+q]                  (plain channel ch < J)
//                         w[r+q] conj(v_j[nv-1-(r+q)])       (virtual coil ch = J+j)
//          + D[mat][r][c] / beta,   c = ch*p + q.
// Adjoint: out_j[k] = conj(w[k]) sum_{r+q=k} E[r][j p + q]
//                   + w[k'] conj(sum_{r+q=k'} E[r][(J+j) p + q]),  k' = nv-1-k.
// The adjoint is a gather over anti-diagonals (no atomics), so it is
// deterministic.  Both kernels are bandwidth-bound streams over the lifted
// arrays: one thread per output element, consecutive threads on consecutive
// addresses of the vector-major workspaces.
#include "selr_internal.cuh"

#define LIFT_THREADS 256
#define LIFT_PER_BLOCK 1024
#define ADJ_SLICES 4

__global__ void __launch_bounds__(LIFT_THREADS)
k_lift(GroupSet gs, int mat_begin, const cf *D, int d_natural, float inv_beta, cf *out, cf *out2,
       int out_natural) {
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int per = g.rows * g.cols;
    const long long mbase = g.off + (long long)mat * per;
    for (int idx = blockIdx.y * LIFT_PER_BLOCK + threadIdx.x; idx < min(per, (int)(blockIdx.y + 1) * LIFT_PER_BLOCK);
         idx += LIFT_THREADS) {
        int r, c;
        if (out_natural) { r = idx / g.cols; c = idx - r * g.cols; }
        else {
            const int v = idx / g.len, e = idx - v * g.len;
            if (g.trans) { r = v; c = e; } else { r = e; c = v; }
        }
        cf val = lift_value(g, mat, r, c);
        if (D) {
            const long long di = d_natural ? mbase + (long long)r * g.cols + c
                                           : g.off + vm_index(g, mat, r, c);
            const cf d = D[di];
            val = mk(val.x + d.x * inv_beta, val.y + d.y * inv_beta);
        }
        out[mbase + idx] = val;
        if (out2) out2[mbase + idx] = val;
    }
}

cudaError_t launch_lift(const GroupSet &gs, int gfirst, int mat_begin, int mat_count, const cf *D,
                        int d_natural, float inv_beta, cf *out, cf *out2, int out_natural,
                        const int *active, cudaStream_t st) {
    (void)gfirst;
    (void)active;
    if (mat_count <= 0) return cudaSuccess;
    int maxper = 0;
    for (int k = 0; k < gs.n; ++k) maxper = max(maxper, gs.g[k].rows * gs.g[k].cols);
    dim3 grid(mat_count, (maxper + LIFT_PER_BLOCK - 1) / LIFT_PER_BLOCK);
    k_lift<<<grid, LIFT_THREADS, 0, st>>>(gs, mat_begin, D, d_natural, inv_beta, out, out2, out_natural);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(LIFT_THREADS)
k_adjoint(GroupSet gs, int mat_begin, const cf *E, int e_natural) {
    int mat;
    const int gi = find_group(gs, mat_begin + blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const long long mbase = g.off + (long long)mat * g.rows * g.cols;
    const int total = g.J * g.nv;
    // blockIdx.y: slice of the J nv outputs (ADJ_SLICES CTAs per matrix, for more loads in flight)
    for (int idx = blockIdx.y * LIFT_THREADS + threadIdx.x; idx < total; idx += LIFT_THREADS * gridDim.y) {
        const int j = idx / g.nv, k = idx - j * g.nv;
        // plain channel j
        cf s = mk(0.f, 0.f);
        {
            const int q0 = max(0, k - g.rows + 1), q1 = min(g.p - 1, k);
            for (int q = q0; q <= q1; ++q) {
                const int r = k - q, c = j * g.p + q;
                const long long ei = e_natural ? mbase + (long long)r * g.cols + c : g.off + vm_index(g, mat, r, c);
                s = cadd(s, E[ei]);
            }
        }
        cf out = g.w ? cmulc(g.w[k], s) : s;
        if (g.vc) {
            const int kk = g.nv - 1 - k;
            cf t = mk(0.f, 0.f);
            const int q0 = max(0, kk - g.rows + 1), q1 = min(g.p - 1, kk);
            for (int q = q0; q <= q1; ++q) {
                const int r = kk - q, c = (g.J + j) * g.p + q;
                const long long ei = e_natural ? mbase + (long long)r * g.cols + c : g.off + vm_index(g, mat, r, c);
                t = cadd(t, E[ei]);
            }
            t = cconj(t);
            out = cadd(out, g.w ? cmul(g.w[kk], t) : t);
        }
        g.dst[src_index(g, mat, j, k)] = out;
    }
}

cudaError_t launch_adjoint(const GroupSet &gs, int gfirst, int mat_begin, int mat_count,
                           const cf *E, int e_natural, cudaStream_t st) {
    (void)gfirst;
    if (mat_count <= 0) return cudaSuccess;
    int maxout = 0;
    for (int k = 0; k < gs.n; ++k) maxout = max(maxout, gs.g[k].J * gs.g[k].nv);
    // a few large matrices (the 2D lifts): several CTAs per matrix; many small ones (the
    // parameter lifts): one CTA each already fills the GPU
    const int slices = mat_count >= 1024 ? 1 : max(1, min(ADJ_SLICES, (maxout + LIFT_THREADS - 1) / LIFT_THREADS));
    k_adjoint<<<dim3(mat_count, slices), LIFT_THREADS, 0, st>>>(gs, mat_begin, E, e_natural);
    return cudaGetLastError();
}

// Copy natural-layout matrices [nmat][rows][cols] into vector-major storage.
__global__ void __launch_bounds__(LIFT_THREADS)
k_nat_to_vm(GroupSet gs, const cf *A, cf *out, cf *out2) {
    int mat;
    const int gi = find_group(gs, blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int per = g.rows * g.cols;
    const long long mbase = g.off + (long long)mat * per;
    for (int idx = blockIdx.y * LIFT_PER_BLOCK + threadIdx.x; idx < min(per, (int)(blockIdx.y + 1) * LIFT_PER_BLOCK);
         idx += LIFT_THREADS) {
        const int v = idx / g.len, e = idx - v * g.len;
        int r, c;
        if (g.trans) { r = v; c = e; } else { r = e; c = v; }
        const cf val = A[mbase + (long long)r * g.cols + c];
        out[mbase + idx] = val;
        if (out2) out2[mbase + idx] = val;
    }
}

cudaError_t launch_natural_to_vm(const GroupSet &gs, const cf *A, cf *out, cf *out2, cudaStream_t st) {
    if (gs.total <= 0) return cudaSuccess;
    int maxper = 0;
    for (int k = 0; k < gs.n; ++k) maxper = max(maxper, gs.g[k].rows * gs.g[k].cols);
    dim3 grid(gs.total, (maxper + LIFT_PER_BLOCK - 1) / LIFT_PER_BLOCK);
    k_nat_to_vm<<<grid, LIFT_THREADS, 0, st>>>(gs, A, out, out2);
    return cudaGetLastError();
}

// Copy vector-major matrices back to natural layout [nmat][rows][cols].
__global__ void __launch_bounds__(LIFT_THREADS)
k_vm_to_nat(GroupSet gs, const cf *in, cf *A) {
    int mat;
    const int gi = find_group(gs, blockIdx.x, &mat);
    const Group &g = gs.g[gi];
    const int per = g.rows * g.cols;
    const long long mbase = g.off + (long long)mat * per;
    for (int idx = blockIdx.y * LIFT_PER_BLOCK + threadIdx.x; idx < min(per, (int)(blockIdx.y + 1) * LIFT_PER_BLOCK);
         idx += LIFT_THREADS) {
        const int v = idx / g.len, e = idx - v * g.len;
        int r, c;
        if (g.trans) { r = v; c = e; } else { r = e; c = v; }
        A[mbase + (long long)r * g.cols + c] = in[mbase + idx];
    }
}

cudaError_t launch_vm_to_natural(const GroupSet &gs, const cf *in, cf *A, cudaStream_t st) {
    if (gs.total <= 0) return cudaSuccess;
    int maxper = 0;
    for (int k = 0; k < gs.n; ++k) maxper = max(maxper, gs.g[k].rows * gs.g[k].cols);
    dim3 grid(gs.total, (maxper + LIFT_PER_BLOCK - 1) / LIFT_PER_BLOCK);
    k_vm_to_nat<<<grid, LIFT_THREADS, 0, st>>>(gs, in, A);
    return cudaGetLastError();
}
