// Initial image of the TNLM algorithm box (step 1): filtered backprojection
// of the projections of all N phases together, for the equiangular arc
// detector.  The paper does not name the filter; this is the equiangular
// fan-beam FBP with the discrete ramp kernel:
//   R'(g_k) = R(g_k) sid cos(g_k)
//   Q(g_n)  = dg sum_k R'(g_k) c(n - k),  c(0) = 1/(8 dg^2), c(even) = 0,
//             c(odd n) = -1/(2 pi^2 sin^2(n dg))
//   f(x)    = sum over all N V views of dbeta Q(g'(x)) / L(x)^2, dbeta = 2 pi / (N V)
// with g'(x) the fan angle of x seen from the source, L its distance to the
// source, Q read by linear interpolation (zero beyond the detector).  Every
// phase of the output receives the same image.
#include "internal.cuh"

#include <math.h>

namespace tnlm {

// Q[v][n] for one view per block; kernel taps (FP64-built table) and the
// weighted projections of the view are staged in shared memory.  Only the
// odd offsets and 0 contribute.
__global__ void __launch_bounds__(256) k_fbp_filter(const float* __restrict__ y,
                                                    const float* __restrict__ taps,   // [2B - 1]
                                                    const float2* __restrict__ bin,
                                                    float* __restrict__ Q, int B, float sid,
                                                    float dg) {
    extern __shared__ float fsm[];
    float* r = fsm;          // [B]
    float* c = fsm + B;      // [2B - 1]
    const size_t v = blockIdx.x;
    for (int k = threadIdx.x; k < B; k += blockDim.x) r[k] = y[v * B + k] * sid * bin[k].x;
    for (int k = threadIdx.x; k < 2 * B - 1; k += blockDim.x) c[k] = taps[k];
    __syncthreads();
    for (int n = threadIdx.x; n < B; n += blockDim.x) {
        float acc = r[n] * c[B - 1];
        // k = n - 1, n - 3, ... and k = n + 1, n + 3, ...
        for (int k = n - 1; k >= 0; k -= 2) acc = fmaf(r[k], c[n - k + B - 1], acc);
        for (int k = n + 1; k < B; k += 2) acc = fmaf(r[k], c[n - k + B - 1], acc);
        Q[v * B + n] = dg * acc;
    }
}

__global__ void __launch_bounds__(256) k_fbp_backproject(const float* __restrict__ Q,
                                                         const float2* __restrict__ view,
                                                         float* __restrict__ img, int nx, int ny,
                                                         int N, int M, int B, float sidp,
                                                         float inv_dg, float half_b, float scale) {
    const int ix = blockIdx.x * 16 + (threadIdx.x & 15);
    const int iy = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (ix >= nx || iy >= ny) return;
    const float cx = (float)ix - 0.5f * (nx - 1);
    const float cy = (float)iy - 0.5f * (ny - 1);
    float acc = 0.f;
    for (int v = 0; v < M; ++v) {
        const float2 vt = view[v];
        const float X = vt.y * cx - vt.x * cy;                  // across the central ray
        const float Y = sidp - (vt.x * cx + vt.y * cy);         // along it
        const float u = fmaf(atanf(X / Y), inv_dg, half_b);
        const float fl = floorf(u);
        const int k0 = (int)fl;
        const float t = u - fl;
        const float* q = Q + (size_t)v * B;
        float val = 0.f;
        if (k0 >= 0 && k0 < B) val = (1.f - t) * __ldg(q + k0);
        if (k0 + 1 >= 0 && k0 + 1 < B) val = fmaf(t, __ldg(q + k0 + 1), val);
        acc += val / fmaf(X, X, Y * Y);
    }
    acc *= scale;
    const size_t npx = (size_t)nx * ny;
    for (int i = 0; i < N; ++i) img[i * npx + (size_t)iy * nx + ix] = acc;
}

// Per-phase variant: phase i is reconstructed from its own V views only
// (dbeta = 2 pi / V), one grid layer per phase.
__global__ void __launch_bounds__(256) k_fbp_backproject_phase(const float* __restrict__ Q,
                                                               const float2* __restrict__ view,
                                                               float* __restrict__ img, int nx, int ny,
                                                               int V, int B, float sidp, float inv_dg,
                                                               float half_b, float scale) {
    const int ix = blockIdx.x * 16 + (threadIdx.x & 15);
    const int iy = blockIdx.y * 16 + (threadIdx.x >> 4);
    const int i = blockIdx.z;
    if (ix >= nx || iy >= ny) return;
    const float cx = (float)ix - 0.5f * (nx - 1);
    const float cy = (float)iy - 0.5f * (ny - 1);
    float acc = 0.f;
    for (int v = i * V; v < (i + 1) * V; ++v) {
        const float2 vt = view[v];
        const float X = vt.y * cx - vt.x * cy;
        const float Y = sidp - (vt.x * cx + vt.y * cy);
        const float u = fmaf(atanf(X / Y), inv_dg, half_b);
        const float fl = floorf(u);
        const int k0 = (int)fl;
        const float t = u - fl;
        const float* q = Q + (size_t)v * B;
        float val = 0.f;
        if (k0 >= 0 && k0 < B) val = (1.f - t) * __ldg(q + k0);
        if (k0 + 1 >= 0 && k0 + 1 < B) val = fmaf(t, __ldg(q + k0 + 1), val);
        acc += val / fmaf(X, X, Y * Y);
    }
    img[((size_t)i * ny + iy) * nx + ix] = acc * scale;
}

cudaError_t launch_fbp_phases(const tnlm_geometry* g, const float* y, float* Q, float* img,
                              cudaStream_t st) {
    const int M = g->N * g->V;
    const float dg = (float)(g->bin_mm / g->sdd);
    const size_t smem = sizeof(float) * (3 * (size_t)g->B - 1);
    k_fbp_filter<<<M, 256, smem, st>>>(y, g->d_fbp_taps, g->d_bin, Q, g->B, (float)g->sid, dg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double scale = 2.0 * 3.14159265358979323846 / (double)g->V / (g->pixel * g->pixel);
    dim3 grid((g->nx + 15) / 16, (g->ny + 15) / 16, g->N);
    k_fbp_backproject_phase<<<grid, 256, 0, st>>>(Q, g->d_view, img, g->nx, g->ny, g->V, g->B,
                                                  (float)(g->sid / g->pixel), (float)(g->sdd / g->bin_mm),
                                                  0.5f * (float)(g->B - 1), (float)scale);
    return cudaGetLastError();
}

cudaError_t launch_fbp(const tnlm_geometry* g, const float* y, float* Q, float* img,
                       cudaStream_t st) {
    const int M = g->N * g->V;
    const float dg = (float)(g->bin_mm / g->sdd);
    const size_t smem = sizeof(float) * (3 * (size_t)g->B - 1);
    k_fbp_filter<<<M, 256, smem, st>>>(y, g->d_fbp_taps, g->d_bin, Q, g->B, (float)g->sid, dg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // dbeta / L^2 with L in mm: the pixel-unit L^2 is scaled by pixel^2
    const double scale = 2.0 * 3.14159265358979323846 / (double)M / (g->pixel * g->pixel);
    dim3 grid((g->nx + 15) / 16, (g->ny + 15) / 16);
    k_fbp_backproject<<<grid, 256, 0, st>>>(Q, g->d_view, img, g->nx, g->ny, g->N, M, g->B,
                                            (float)(g->sid / g->pixel), (float)(g->sdd / g->bin_mm),
                                            0.5f * (float)(g->B - 1), (float)scale);
    return cudaGetLastError();
}

}  // namespace tnlm
