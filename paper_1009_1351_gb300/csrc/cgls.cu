// Data step (Sec. 2.2): the CGLS box per phase with P_n = Sigma^{-1/2} P_i,
// y_n = Sigma^{-1/2} y_i, warm-started at u^(0) = f^(k-1); or the gradient
// step of Eq. 4.  Vectors are FP32; every norm is a deterministic per-block
// FP32-tree / FP64 sum followed by an FP64 sum over blocks (scalar kernels
// below), so the step sizes a_i, b_i are formed in FP64.
//
// Reading for a zero denominator (the paper does not say): once
// ||P_n s||^2 = 0 or ||P_n^T r||^2 = 0 for a phase, that phase's CGLS stops
// (a_i = 0 from then on) and g_i = u_i.
#include "internal.cuh"

namespace tnlm {

// Sum partials[0 .. n) in a fixed order: thread-strided FP64 sums, then an
// FP64 tree over the block.  256 threads, so each thread loads only a few
// partials (the dependent loads, not the adds, set the time).  Called by
// the whole block; every thread returns the total.
constexpr int kScalarThreads = 256;
__device__ __forceinline__ double block_sum_partials(const double* p, int n, double* sh) {
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += kScalarThreads) s += p[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = kScalarThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    const double t = sh[0];
    __syncthreads();
    return t;
}

struct ScalArgs {
    const double* part_s;  // sinogram-side partials [N][ps]
    const double* part_i;  // image-side partials [N][pi]
    int ps, pi;
    DevState st;
};

// After r^(0) = y_n - P_n u^(0) and s^(0) = P_n^T r^(0):
// gamma = ||s^(0)||^2, res0 = ||r^(0)||^2, CGLS active.
__global__ void __launch_bounds__(kScalarThreads) k_cgls_init_scalars(ScalArgs a) {
    __shared__ double sh[kScalarThreads];
    const int i = blockIdx.x;
    const double g = block_sum_partials(a.part_i + (size_t)i * a.pi, a.pi, sh);
    const double r = block_sum_partials(a.part_s + (size_t)i * a.ps, a.ps, sh);
    if (threadIdx.x == 0) {
        a.st.gamma[i] = g;
        a.st.res0[i] = r;
        a.st.active[i] = 1;
        if (!isfinite(g) || !isfinite(r)) atomicOr(a.st.err, 1);
    }
}

// Step 1: a = ||P_n^T r||^2 / ||P_n s||^2.
__global__ void __launch_bounds__(kScalarThreads) k_cgls_a(ScalArgs a) {
    __shared__ double sh[kScalarThreads];
    const int i = blockIdx.x;
    const double den = block_sum_partials(a.part_s + (size_t)i * a.ps, a.ps, sh);
    if (threadIdx.x == 0) {
        const double gam = a.st.gamma[i];
        if (!a.st.active[i] || den == 0.0 || gam == 0.0) {
            a.st.active[i] = 0;
            a.st.a[i] = 0.0;
        } else {
            a.st.a[i] = gam / den;
        }
        if (!isfinite(den)) atomicOr(a.st.err, 1);
    }
}

// Step 4: b = ||P_n^T r^(m+1)||^2 / ||P_n^T r^(m)||^2.
__global__ void __launch_bounds__(kScalarThreads) k_cgls_b(ScalArgs a) {
    __shared__ double sh[kScalarThreads];
    const int i = blockIdx.x;
    const double gnew = block_sum_partials(a.part_i + (size_t)i * a.pi, a.pi, sh);
    if (threadIdx.x == 0) {
        if (a.st.active[i]) {
            a.st.b[i] = gnew / a.st.gamma[i];
            a.st.gamma[i] = gnew;
        } else {
            a.st.b[i] = 0.0;
        }
    }
}

static ScalArgs scal_args(const tnlm_geometry* g, const Workspace& ws) {
    ScalArgs a;
    a.part_s = ws.part;
    a.ps = proj_blocks_per_phase(g);
    a.part_i = ws.part + (size_t)g->N * a.ps;
    a.pi = bp_blocks_per_phase(g);
    a.st = ws.st;
    return a;
}

cudaError_t launch_cgls_init_scalars(const tnlm_geometry* g, const Workspace& ws, cudaStream_t st) {
    k_cgls_init_scalars<<<g->N, kScalarThreads, 0, st>>>(scal_args(g, ws));
    return cudaGetLastError();
}
cudaError_t launch_cgls_a(const tnlm_geometry* g, const Workspace& ws, cudaStream_t st) {
    k_cgls_a<<<g->N, kScalarThreads, 0, st>>>(scal_args(g, ws));
    return cudaGetLastError();
}
cudaError_t launch_cgls_b(const tnlm_geometry* g, const Workspace& ws, cudaStream_t st) {
    k_cgls_b<<<g->N, kScalarThreads, 0, st>>>(scal_args(g, ws));
    return cudaGetLastError();
}

// Steps 2-3: u += a s (images) and, unless this is the last CGLS step,
// r -= a t with z = sqrt(w) r for the next adjoint (sinograms).
__global__ void __launch_bounds__(256) k_cgls_update_ur(float* __restrict__ u,
                                                        const float* __restrict__ s,
                                                        float* __restrict__ r,
                                                        float* __restrict__ z,
                                                        const float* __restrict__ t,
                                                        const float* __restrict__ sw,
                                                        const double* __restrict__ acoef,
                                                        size_t npx, size_t nsg, int N,
                                                        int with_r) {
    const size_t nI = npx * N, nS = with_r ? nsg * N : 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nI + nS; k += stride) {
        if (k < nI) {
            const float a = (float)acoef[k / npx];
            u[k] = fmaf(a, s[k], u[k]);
        } else {
            const size_t q = k - nI;
            const float a = (float)acoef[q / nsg];
            const float rr = fmaf(-a, t[q], r[q]);
            r[q] = rr;
            z[q] = sw[q] * rr;
        }
    }
}

static int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_cgls_update_ur(const tnlm_geometry* g, const Workspace& ws, const float* s,
                                  bool with_r, cudaStream_t st) {
    const size_t npx = (size_t)g->nx * g->ny, nsg = (size_t)g->V * g->B;
    const size_t n = npx * g->N + (with_r ? nsg * g->N : 0);
    k_cgls_update_ur<<<grid_for(n), 256, 0, st>>>(ws.u, s, ws.r, ws.z, ws.t, ws.sw, ws.st.a,
                                                   npx, nsg, g->N, with_r ? 1 : 0);
    return cudaGetLastError();
}

// Step 5 (s = P_n^T r^(m+1) + b s) is fused into the layout preparation of
// s for the next projection (k_prep_dual<2>, project.cu).

// Eq. 4 with s = P^T w (y - P f) already formed: g = f + s / beta.
__global__ void __launch_bounds__(256) k_grad_final(float* __restrict__ u,
                                                    const float* __restrict__ s, float inv_beta,
                                                    size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        u[k] = fmaf(inv_beta, s[k], u[k]);
}

cudaError_t launch_grad_final(const tnlm_geometry* g, const Workspace& ws, double beta,
                              cudaStream_t st) {
    const size_t n = (size_t)g->nx * g->ny * g->N;
    k_grad_final<<<grid_for(n), 256, 0, st>>>(ws.u, ws.s, (float)(1.0 / beta), n);
    return cudaGetLastError();
}

// sqrt(Sigma^{-1}); a negative or non-finite entry raises the numeric flag.
__global__ void __launch_bounds__(256) k_sqrt(const float* __restrict__ w, float* __restrict__ sw,
                                              size_t n, int* err) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const float v = w[k];
        if (!(v >= 0.f) || isinf(v)) {
            atomicOr(err, 2);
            sw[k] = 0.f;
        } else {
            sw[k] = sqrtf(v);
        }
    }
}

cudaError_t launch_sqrt(const float* w, float* sw, size_t n, int* err, cudaStream_t st) {
    k_sqrt<<<grid_for(n), 256, 0, st>>>(w, sw, n, err);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_fill(float* __restrict__ p, float v, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) p[k] = v;
}

cudaError_t launch_fill(float* p, float v, size_t n, cudaStream_t st) {
    k_fill<<<grid_for(n), 256, 0, st>>>(p, v, n);
    return cudaGetLastError();
}

}  // namespace tnlm
