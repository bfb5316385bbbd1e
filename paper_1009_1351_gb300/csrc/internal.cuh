// Internal declarations of the TNLM CUDA library (not part of the ABI).
//
// Data layout in HBM (per geometry handle; N phases, image nx x ny, V views,
// B bins, window W = 2*rho+1):
//   images        [N][ny][nx]             f, u (CGLS iterate / g), s, grad
//   dual layout   R [N][ny][nx+4], T [N][nx][ny+4] of float2: the projector's
//                 input in row-major and column-major form with two zero pad
//                 positions on each side of a line, entry q holding
//                 (X[q] - X[q+1], X[q+1]), so that every ray reads one pair
//                 per line at consecutive addresses across a warp whichever
//                 axis it marches along.
//   sinograms     [N][V][B]               r, z = sqrt(w) r, t, sqrt(w)
//   D planes      [N pairs][W*W][py][px]  patch distances of pair (i, i+1)
//                 with a halo of rho rows and ox >= rho columns holding +inf
//   u ping-pong   2 x [N][py][px]         Gauss-Jacobi iterates, zero halo
//   minima        [2][N][ny][nx]          row minima of D per direction
//   partials      FP64 per-block sums, reduced in a fixed order (deterministic)
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tnlm.h"

namespace tnlm {

constexpr int kMaxPatch = 15;
constexpr int kMaxWindow = 31;
#ifndef TNLM_PROJ_THREADS
#define TNLM_PROJ_THREADS 128
#endif
constexpr int kProjThreads = TNLM_PROJ_THREADS;   // rays per projector block
constexpr int kWTileX = 32, kWTileY = 16;  // weight kernel output tile
constexpr int kGjTileX = 32, kGjTileY = 8; // Gauss-Jacobi tile

struct PadPlane {
    int px, py;   // pitch (floats) and rows
    int ox, oy;   // interior origin
    size_t plane; // px * py
};

// Per-phase scalars of the data step and the per-iteration monitors.
struct DevState {
    double* gamma;     // [N] ||P_n^T r||^2 of the current CGLS step
    double* a;         // [N]
    double* b;         // [N]
    double* res0;      // [N] ||r^(0)||^2 (data term of f^(k-1))
    int* active;       // [N] CGLS not stopped
    double* hist_rel;  // [kcap]
    double* hist_res;  // [kcap]
    double* hist_clamp; // [kcap] pixels clamped by the positivity step
    double* hist_tnlm; // [kcap] TNLM term of Eq. 1 (monitor on)
    double* res_final; // data term of the final image (monitor on)
    int* iter;         // outer iteration counter (device)
    int* err;          // numeric fault flag
};

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    int rho = -1;      // window radius the buffers are sized for
    int kcap = 0;      // history capacity
    // images
    float *u = nullptr, *s = nullptr, *gr = nullptr;
    float* s2 = nullptr;     // CGLS direction, second buffer (updates alternate between s and s2)
    float *R = nullptr, *T = nullptr;   // float2 pairs (see the dual layout above)
    // sinograms
    float *r = nullptr, *z = nullptr, *t = nullptr, *sw = nullptr;
    float* bps = nullptr;    // backprojection partial images [4][N][ny][nx]
    // TNLM step
    PadPlane pp{};
    float* D = nullptr;      // [N][W*W][py][px]
    float* U0 = nullptr;     // [N][py][px]
    float* U1 = nullptr;
    float* mins = nullptr;   // [2][N][ny][nx]  (next, prev)
    float* zn = nullptr;     // [2][N][ny][nx]  normalisers (public weights call only)
    // reductions
    double* part = nullptr;  // partial sums
    size_t part_len = 0;
    double* part2 = nullptr; // second partial array (relative change, clamp count)
    double* part3 = nullptr; // monitor partials (TNLM term per sweep block)
    float* gjsum = nullptr;  // TMA sweep: partial sums of window halves [tile][2][4][256] float4
    int* gjcnt = nullptr;    // TMA sweep: halves done per tile (0 between sweeps)
    DevState st{};
    // TMA descriptors of the distance planes [N*W2max][py][px]: boxes of
    // 64 x 16 (forward rows) and 68 x 16 (backward rows) floats
    CUtensorMap tmF{};
    CUtensorMap tmB{};
    // and of the Gauss-Jacobi iterates U0 / U1 [N][py][px]: box 80 x 30
    CUtensorMap tmU0{};
    CUtensorMap tmU1{};
    bool tm_ok = false;
};

}  // namespace tnlm

struct tnlm_geometry {
    int device;
    int nx, ny, N, V, B;
    double pixel, bin_mm, sid, sdd;
    float2* d_view = nullptr;   // [N*V] (cos t, sin t)
    float2* d_bin = nullptr;    // [B] (cos g, sin g)
    float4* d_ray = nullptr;    // [N*V*B] per-ray marching constants (kk, alpha, 1/|kk|, +-L)
    int4* d_vcls = nullptr;     // [N*V] bin ranges (lo, hi) of the column-marching rays (x, y)
                                // and of the row-marching rays (z, w) of each view; lo > hi: none
    float* d_fbp_taps = nullptr; // [2B-1] discrete equiangular ramp kernel of the initial FBP
    tnlm::Workspace ws;
    // changes whenever ensure_ws replaces the workspace allocation: the
    // buffer offsets depend on the window radius and history capacity it
    // was sized for, and a new allocation may reuse a freed address, so
    // captured graphs are keyed on this counter rather than on the address
    unsigned long long ws_gen = 0;
    int cta_slots_bp = 0;       // resident backprojector CTAs on the device
    int cta_slots_gj = 0;       // resident TMA-sweep CTAs on the device
    int num_sms = 0;            // streaming multiprocessors of the device
    // launch choices set by tnlm_autotune (0 = built-in heuristic); tune_gen
    // changes whenever they do, so captured graphs are re-captured
    int tune_bp_groups = 0;     // view groups (CTAs) per backprojection tile
    int tune_gj_tpb = 0;        // tiles per CTA of the TMA sweep
    int tune_gj_split = 0;      // window halves per tile of the TMA sweep (0: by wave fill)
    unsigned tune_gen = 0;
    unsigned long long uid = 0; // unique per handle (graph and batch keys)
    // CUDA graph of one outer iteration (see api.cu)
    void* graph = nullptr;
    // profiling: launch counters and event-bracketed timing (see api.cu)
    unsigned prof_mask = 0;
    long long launches[TNLM_KCLASS_COUNT] = {0, 0, 0, 0, 0, 0};
    void* prof = nullptr;
};

namespace tnlm {

// ---- launchers (defined in the .cu files) --------------------------------
struct ProjOut {
    int mode;              // 0: q, 1: r = sw (y - q), z = sw r, 2: t = sw q
    float* q;              // mode 0 output / mode 2 t
    float* r;              // mode 1
    float* z;              // mode 1
    const float* y;        // mode 1
    const float* sw;       // modes 1, 2
    double* part;          // modes 1, 2: [N*V*nchunk] partial sums of squares
};
int proj_blocks_per_phase(const tnlm_geometry* g);
cudaError_t launch_prep_dual(const tnlm_geometry* g, const float* img, float* R, float* T,
                             cudaStream_t st);
cudaError_t launch_prep_dual_copy(const tnlm_geometry* g, const float* img, float* cp, float* R,
                                  float* T, cudaStream_t st);
cudaError_t launch_prep_dual_update(const tnlm_geometry* g, const float* s, float* s_new, const float* gr,
                                    const double* bcoef, const int* active, float* R, float* T,
                                    cudaStream_t st);
cudaError_t launch_project(const tnlm_geometry* g, const float* R, const float* T,
                           const ProjOut& o, cudaStream_t st);
cudaError_t prepare_backproject(int* slots);
cudaError_t prepare_weights(int* gj_slots);
cudaError_t prepare_weights_tc();                 // tensor-core variant (mixed precision)
bool weights_tc_supported(int patch, int window);
cudaError_t launch_weights_tc(const tnlm_geometry* g, const Workspace& ws, int patch, int window,
                              const float* gimg, cudaStream_t st);   // also counts resident TMA-sweep CTAs
int bp_blocks_per_phase(const tnlm_geometry* g);
int bp_max_groups(const tnlm_geometry* g);      // largest useful view-group count
size_t static_scratch_floats();
cudaError_t static_scratch_ptr(float** out);
size_t bp_scratch_floats(const tnlm_geometry* g);
// scratch: partial images of the view groups ([4][N][ny][nx]); NULL = one group
cudaError_t launch_backproject(const tnlm_geometry* g, const float* sino, float* img,
                               double* part, float* scratch, cudaStream_t st);

// initial image (filtered backprojection of all views); Q: [N*V*B] scratch
cudaError_t launch_fbp(const tnlm_geometry* g, const float* y, float* Q, float* img,
                       cudaStream_t st);
cudaError_t launch_fbp_phases(const tnlm_geometry* g, const float* y, float* Q, float* img,
                              cudaStream_t st);

// CGLS vector / scalar kernels
cudaError_t launch_cgls_init_scalars(const tnlm_geometry* g, const Workspace& ws,
                                     cudaStream_t st);
cudaError_t launch_cgls_a(const tnlm_geometry* g, const Workspace& ws, cudaStream_t st);
cudaError_t launch_cgls_update_ur(const tnlm_geometry* g, const Workspace& ws, const float* s, bool with_r,
                                  cudaStream_t st);
cudaError_t launch_cgls_b(const tnlm_geometry* g, const Workspace& ws, cudaStream_t st);
cudaError_t launch_grad_final(const tnlm_geometry* g, const Workspace& ws, double beta,
                              cudaStream_t st);
cudaError_t launch_sqrt(const float* w, float* sw, size_t n, int* err, cudaStream_t st);
cudaError_t launch_fill(float* p, float v, size_t n, cudaStream_t st);

// TNLM step kernels
// store = false: only the row minima (and u^(0)) -- the distances are
// recomputed by the fused sweep
cudaError_t launch_weights(const tnlm_geometry* g, const Workspace& ws, int patch, int window,
                           const float* gimg, cudaStream_t st, bool store = true);
// Gauss-Jacobi sweep that recomputes the patch distances of both directions
// from g instead of reading the stored array (fout != NULL: the last sweep)
cudaError_t launch_gj_fused(const tnlm_geometry* g, const Workspace& ws, int patch, int window, double h,
                            double mu_hat, const float* gimg, const float* uin, float* uout, float* fout,
                            int clamp, cudaStream_t st);
cudaError_t prepare_gj_fused();
bool fused_supported(int patch, int window);
cudaError_t launch_gj_sweep(const tnlm_geometry* g, const Workspace& ws, int window, double h,
                            double mu_hat, const float* gimg, const float* uin, float* uout,
                            float* fout, int clamp, cudaStream_t st);
cudaError_t launch_finalize_nogj(const tnlm_geometry* g, const Workspace& ws, const float* gimg,
                                 float* fout, int clamp, cudaStream_t st);
cudaError_t launch_iter_scalars(const tnlm_geometry* g, const Workspace& ws, int nblocks, bool monitor,
                                cudaStream_t st);
// monitor: TNLM term of Eq. 1 from the stored distances and the result f
cudaError_t launch_tnlm_energy(const tnlm_geometry* g, const Workspace& ws, int window, double h,
                               const float* f, cudaStream_t st);
int tnlm_energy_blocks(const tnlm_geometry* g);
cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t st);
int gj_blocks(const tnlm_geometry* g);
int gj_tma_split(const tnlm_geometry* g);
// Poll limit of the TMA sweep's pipeline waits (not of its final drain);
// lowered only by tnlm_debug_wait_limit to exercise the timeout path.
extern long g_gj_wait_limit;
size_t gj_split_floats(const tnlm_geometry* g);
cudaError_t launch_weights_norm(const tnlm_geometry* g, const Workspace& ws, int window,
                                double h, cudaStream_t st);
cudaError_t launch_weights_export(const tnlm_geometry* g, const Workspace& ws, int window,
                                  float* d_dist, float* d_norm, cudaStream_t st);
// encode ws.tmF / ws.tmB for the distance planes (false if TMA is unavailable)
bool encode_distance_maps(Workspace& ws, int N);

// ---- device helpers -------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block reduction: each warp reduces in FP32 (a depth-5 tree), warp totals
// are combined in FP64 in warp order by thread 0.  Deterministic.
template <int NT>
__device__ __forceinline__ double block_sum(float v, double* sh, int tid) {
    v = warp_sum(v);
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    double tot = 0.0;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) tot += sh[k];
    }
    __syncthreads();
    return tot;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// mbarrier helpers (shared by the TMA sweep and the tensor-core weights).
// Every wait is bounded: after kSpinLimit polls it gives up and returns false.
// ---------------------------------------------------------------------------
constexpr long kSpinLimit = 1L << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long limit = kSpinLimit) {
    for (long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
}  // namespace tnlm
