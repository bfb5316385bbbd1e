// C ABI of the TNLM library: argument checks, geometry tables, workspace and
// the outer iteration of the TNLM algorithm box (Sec. 2.2).
#include "internal.cuh"

#include <stdlib.h>

#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

using namespace tnlm;

namespace {

thread_local char g_err[512] = "";
std::atomic<int> g_fail_after{0};

tnlm_status fail(tnlm_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

tnlm_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(TNLM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(TNLM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

cudaError_t dev_alloc(void** p, size_t n) {
    *p = nullptr;
    int f = g_fail_after.load();
    while (f > 0) {
        if (g_fail_after.compare_exchange_weak(f, f - 1)) {
            if (f == 1) return cudaErrorMemoryAllocation;
            break;
        }
    }
    return cudaMalloc(p, n);
}

struct DeviceGuard {
    int prev = -1;
    cudaError_t err;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Event pairs recorded around timed launches; reused after each read.
struct Profiler {
    std::vector<cudaEvent_t> ev;   // 2 per timed launch
    std::vector<int> cls;          // class of each pair
    size_t used = 0;               // pairs recorded since the last read
};

// Counts one launch of class c and, if c is timed, brackets it with events.
struct LaunchScope {
    tnlm_geometry* g;
    int c;
    cudaStream_t st;
    cudaEvent_t end = nullptr;
    LaunchScope(const tnlm_geometry* gc, int cls, cudaStream_t s)
        : g(const_cast<tnlm_geometry*>(gc)), c(cls), st(s) {
        g->launches[c]++;
        if (!(g->prof_mask & (1u << c))) return;
        Profiler* P = (Profiler*)g->prof;
        if (!P) g->prof = P = new Profiler();
        if (P->used * 2 + 2 > P->ev.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
            P->ev.push_back(a);
            P->ev.push_back(b);
            P->cls.push_back(c);
        }
        P->cls[P->used] = c;
        cudaEventRecord(P->ev[2 * P->used], st);
        end = P->ev[2 * P->used + 1];
        P->used++;
    }
    ~LaunchScope() {
        if (end) cudaEventRecord(end, st);
    }
};

#define LK(cls, call, what)                                     \
    do {                                                        \
        cudaError_t e_;                                         \
        {                                                       \
            LaunchScope ls_(g, cls, st);                        \
            e_ = (call);                                        \
        }                                                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);      \
    } while (0)

tnlm_status check_params(const tnlm_params* p) {
    if (!p) return fail(TNLM_ERR_INVALID_ARG, "params is NULL");
    if (!(p->mu_hat >= 0.0) || !isfinite(p->mu_hat))
        return fail(TNLM_ERR_INVALID_ARG, "mu_hat must be finite and >= 0");
    if (!(p->h > 0.0) || !isfinite(p->h)) return fail(TNLM_ERR_INVALID_ARG, "h must be finite and > 0");
    if (p->patch < 1 || p->patch > kMaxPatch || (p->patch & 1) == 0)
        return fail(TNLM_ERR_INVALID_ARG, "patch must be odd and in [1, %d]", kMaxPatch);
    if (p->window < 1 || p->window > kMaxWindow || (p->window & 1) == 0)
        return fail(TNLM_ERR_INVALID_ARG, "window must be odd and in [1, %d]", kMaxWindow);
    if (p->m1 < 0 || p->m2 < 0 || p->k_outer < 0)
        return fail(TNLM_ERR_INVALID_ARG, "m1, m2 and k_outer must be >= 0");
    if (p->m1 > 1000 || p->m2 > 100000 || p->k_outer > 1000000)
        return fail(TNLM_ERR_INVALID_ARG, "iteration counts out of range");
    if (p->data_step != TNLM_DATA_CGLS && p->data_step != TNLM_DATA_GRAD)
        return fail(TNLM_ERR_INVALID_ARG, "data_step must be TNLM_DATA_CGLS or TNLM_DATA_GRAD");
    if (p->data_step == TNLM_DATA_GRAD && (!(p->beta > 0.0) || !isfinite(p->beta)))
        return fail(TNLM_ERR_INVALID_ARG, "beta must be finite and > 0 for the gradient step");
    if (p->clamp != 0 && p->clamp != 1) return fail(TNLM_ERR_INVALID_ARG, "clamp must be 0 or 1");
    if (!(p->tol >= 0.0) || !isfinite(p->tol)) return fail(TNLM_ERR_INVALID_ARG, "tol must be >= 0");
    if (p->tol > 0.0 && p->tol_check_every < 1)
        return fail(TNLM_ERR_INVALID_ARG, "tol_check_every must be >= 1 when tol > 0");
    if (p->precision != TNLM_PREC_FP32 && p->precision != TNLM_PREC_MIXED)
        return fail(TNLM_ERR_INVALID_ARG, "precision must be TNLM_PREC_FP32 or TNLM_PREC_MIXED");
    if (p->precision == TNLM_PREC_MIXED && !weights_tc_supported(p->patch, p->window))
        return fail(TNLM_ERR_INVALID_ARG, "mixed precision supports patch <= 7 and window in [3, 15]");
    if (p->monitor != 0 && p->monitor != 1) return fail(TNLM_ERR_INVALID_ARG, "monitor must be 0 or 1");
    if (p->recompute != 0 && p->recompute != 1) return fail(TNLM_ERR_INVALID_ARG, "recompute must be 0 or 1");
    if (p->recompute && p->precision == TNLM_PREC_MIXED)
        return fail(TNLM_ERR_INVALID_ARG, "recompute takes the FP32 distances (precision must be TNLM_PREC_FP32)");
    if (p->recompute && !fused_supported(p->patch, p->window))
        return fail(TNLM_ERR_INVALID_ARG, "recompute supports patch <= 7 and window <= 15");
    return TNLM_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Byte layout of the workspace for window radius rho and history capacity kcap.
struct WsLayout {
    size_t off_u, off_s, off_s2, off_gr, off_R, off_T, off_r, off_z, off_t, off_sw, off_bps, off_D, off_U0, off_U1,
        off_mins, off_zn, off_part, off_part2, off_part3, off_gjs, off_gjc, off_state, total;
    size_t part_len, part2_len;
    PadPlane pp;
};

WsLayout ws_layout(const tnlm_geometry* g, int rho, int kcap) {
    WsLayout L{};
    const size_t npx = (size_t)g->nx * g->ny, N = g->N;
    const size_t nsg = (size_t)g->V * g->B;
    // interior starts at a 32-byte aligned column (a DRAM sector) with at
    // least one spare float4 beyond the window radius on each side
    // (vectorised Gauss-Jacobi windows), and whole 64 x 16 Gauss-Jacobi
    // tiles fit inside every plane.  With the interior at a sector boundary
    // a 64-float row of the weights' stores covers 8 whole sectors instead
    // of touching 9 partly (measured at 512^2, d = 7, W = 15: 0.85 -> 0.67 ms
    // per weights launch, 257 -> 29 MB of DRAM reads for partial-sector
    // fills).  The pitch is 16 floats past a multiple of 128 bytes: a pitch
    // of whole 128-byte lines made the sweep 1.5 % slower (0.560 against
    // 0.550 ms).
    const int ox = (int)align_up(align_up((size_t)rho, 4) + 4, 8);
    L.pp.ox = ox;
    L.pp.oy = rho;
    L.pp.px = (int)align_up(align_up((size_t)g->nx, 64) + 2 * ox, 32) + 16;
    L.pp.py = (int)align_up((size_t)g->ny, 16) + 2 * rho;
    L.pp.plane = (size_t)L.pp.px * L.pp.py;
    const size_t W2 = (size_t)(2 * rho + 1) * (2 * rho + 1);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.off_u = take(4 * npx * N);
    L.off_s = take(4 * npx * N);
    L.off_s2 = take(4 * npx * N);
    L.off_gr = take(4 * npx * N);
    L.off_R = take(8 * (size_t)g->ny * (g->nx + 4) * N);    // float2 pairs
    L.off_T = take(8 * (size_t)g->nx * (g->ny + 4) * N);
    L.off_r = take(4 * nsg * N);
    L.off_z = take(4 * nsg * N);
    L.off_t = take(4 * nsg * N);
    L.off_sw = take(4 * nsg * N);
    L.off_bps = take(4 * bp_scratch_floats(g));
    L.off_D = take(4 * L.pp.plane * W2 * N);
    L.off_U0 = take(4 * L.pp.plane * N);
    L.off_U1 = take(4 * L.pp.plane * N);
    L.off_mins = take(4 * 2 * npx * N);
    L.off_zn = take(4 * 2 * npx * N);
    L.part_len = N * (size_t)proj_blocks_per_phase(g) + N * (size_t)bp_blocks_per_phase(g);
    L.part2_len = 3 * (size_t)gj_blocks(g);
    L.off_part = take(8 * L.part_len);
    L.off_part2 = take(8 * L.part2_len);
    L.off_part3 = take(8 * (size_t)tnlm_energy_blocks(g));
    L.off_gjs = take(4 * gj_split_floats(g));
    L.off_gjc = take(4 * (size_t)gj_blocks(g));
    // state: gamma, a, b, res0 [N] doubles; hist 4 x kcap doubles; res_final;
    // active [N], iter, err ints
    L.off_state = take(8 * (4 * N + 4 * (size_t)kcap + 1) + 4 * (N + 2));
    L.total = o;
    return L;
}

tnlm_status ensure_ws(tnlm_geometry* g, int rho, int kcap, cudaStream_t st) {
    Workspace& ws = g->ws;
    if (ws.base && ws.rho >= rho && ws.kcap >= kcap) return TNLM_OK;
    const int nrho = ws.base ? (ws.rho > rho ? ws.rho : rho) : rho;
    const int nk = ws.base ? (ws.kcap > kcap ? ws.kcap : kcap) : kcap;
    WsLayout L = ws_layout(g, nrho, nk < 1 ? 1 : nk);
    void* base = nullptr;
    cudaError_t e = dev_alloc(&base, L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TNLM_ERR_OOM, "workspace allocation of %zu bytes failed: %s", L.total,
                    cudaGetErrorString(e));
    }
    if (ws.base) {
        cudaStreamSynchronize(st);
        cudaFree(ws.base);
    }
    char* b = (char*)base;
    ws = Workspace{};
    g->ws_gen++;
    ws.base = base;
    ws.bytes = L.total;
    ws.rho = nrho;
    ws.kcap = nk < 1 ? 1 : nk;
    ws.u = (float*)(b + L.off_u);
    ws.s = (float*)(b + L.off_s);
    ws.s2 = (float*)(b + L.off_s2);
    ws.gr = (float*)(b + L.off_gr);
    ws.R = (float*)(b + L.off_R);
    ws.T = (float*)(b + L.off_T);
    ws.r = (float*)(b + L.off_r);
    ws.z = (float*)(b + L.off_z);
    ws.t = (float*)(b + L.off_t);
    ws.sw = (float*)(b + L.off_sw);
    ws.bps = (float*)(b + L.off_bps);
    ws.pp = L.pp;
    ws.D = (float*)(b + L.off_D);
    ws.U0 = (float*)(b + L.off_U0);
    ws.U1 = (float*)(b + L.off_U1);
    ws.mins = (float*)(b + L.off_mins);
    ws.zn = (float*)(b + L.off_zn);
    ws.part = (double*)(b + L.off_part);
    ws.part_len = L.part_len;
    ws.part2 = (double*)(b + L.off_part2);
    ws.part3 = (double*)(b + L.off_part3);
    ws.gjsum = (float*)(b + L.off_gjs);
    ws.gjcnt = (int*)(b + L.off_gjc);
    const size_t N = g->N;
    double* sd = (double*)(b + L.off_state);
    ws.st.gamma = sd;
    ws.st.a = sd + N;
    ws.st.b = sd + 2 * N;
    ws.st.res0 = sd + 3 * N;
    ws.st.hist_rel = sd + 4 * N;
    ws.st.hist_res = sd + 4 * N + ws.kcap;
    ws.st.hist_clamp = sd + 4 * N + 2 * (size_t)ws.kcap;
    ws.st.hist_tnlm = sd + 4 * N + 3 * (size_t)ws.kcap;
    ws.st.res_final = sd + 4 * N + 4 * (size_t)ws.kcap;
    int* si = (int*)(sd + 4 * N + 4 * (size_t)ws.kcap + 1);
    ws.st.active = si;
    ws.st.iter = si + N;
    ws.st.err = si + N + 1;
    // zero everything (pads of R/T, halos of U0/U1, state), then +inf in D
    ws.tm_ok = encode_distance_maps(ws, g->N);
    CK(cudaMemsetAsync(base, 0, L.total, st), "workspace clear");
    LK(TNLM_KCLASS_PREP, launch_fill(ws.D, INFINITY, (L.off_U0 - L.off_D) / 4, st), "distance halo fill");
    return TNLM_OK;
}

tnlm_status check_geom_handle(const tnlm_geometry* g) {
    if (!g) return fail(TNLM_ERR_INVALID_ARG, "geometry handle is NULL");
    return TNLM_OK;
}

// One outer iteration of the TNLM algorithm box on the handle's workspace.
tnlm_status outer_iteration(tnlm_geometry* g, const tnlm_params* p, const float* d_y, float* d_f,
                            cudaStream_t st) {
    Workspace& ws = g->ws;
    const size_t nps = (size_t)g->N * proj_blocks_per_phase(g);
    double* part_s = ws.part;
    double* part_i = ws.part + nps;
    // ---- data step: r0 = sqrt(w)(y - P f), s0 = P_n^T r0 (CGLS) / w(y - P f) back-projected (Eq. 4)
    LK(TNLM_KCLASS_PREP, launch_prep_dual_copy(g, d_f, ws.u, ws.R, ws.T, st), "prep");
    ProjOut o{};
    o.mode = 1; o.r = ws.r; o.z = ws.z; o.y = d_y; o.sw = ws.sw; o.part = part_s;
    LK(TNLM_KCLASS_PROJECT, launch_project(g, ws.R, ws.T, o, st), "project");
    LK(TNLM_KCLASS_BACKPROJECT, launch_backproject(g, ws.z, ws.s, part_i, ws.bps, st), "backproject");
    LK(TNLM_KCLASS_CGLS, launch_cgls_init_scalars(g, ws, st), "scalars");
    if (p->data_step == TNLM_DATA_GRAD) {
        LK(TNLM_KCLASS_CGLS, launch_grad_final(g, ws, p->beta, st), "gradient step");
    } else {
        // the direction lives in sbuf[cur]; each update writes the other buffer
        float* sbuf[2] = {ws.s, ws.s2};
        int cur = 0;
        for (int m = 0; m < p->m1; ++m) {
            const bool last = m == p->m1 - 1;
            // from the second step on, the direction update s = P_n^T r + b s
            // is fused into the layout preparation of s
            if (m == 0) {
                LK(TNLM_KCLASS_PREP, launch_prep_dual(g, sbuf[0], ws.R, ws.T, st), "prep");
            } else {
                LK(TNLM_KCLASS_PREP,
                   launch_prep_dual_update(g, sbuf[cur], sbuf[cur ^ 1], ws.gr, ws.st.b, ws.st.active,
                                           ws.R, ws.T, st),
                   "cgls s + prep");
                cur ^= 1;
            }
            ProjOut ot{};
            ot.mode = 2; ot.q = ws.t; ot.sw = ws.sw; ot.part = part_s;
            LK(TNLM_KCLASS_PROJECT, launch_project(g, ws.R, ws.T, ot, st), "project");
            LK(TNLM_KCLASS_CGLS, launch_cgls_a(g, ws, st), "cgls a");
            LK(TNLM_KCLASS_CGLS, launch_cgls_update_ur(g, ws, sbuf[cur], !last, st), "cgls update");
            if (last) break;
            LK(TNLM_KCLASS_BACKPROJECT, launch_backproject(g, ws.z, ws.gr, part_i, ws.bps, st), "backproject");
            LK(TNLM_KCLASS_CGLS, launch_cgls_b(g, ws, st), "cgls b");
        }
    }
    // ---- TNLM step: weights from g = ws.u, Gauss-Jacobi, positivity
    if (p->m2 > 0 || p->monitor) {
        if (p->precision == TNLM_PREC_MIXED)
            LK(TNLM_KCLASS_WEIGHTS, launch_weights_tc(g, ws, p->patch, p->window, ws.u, st), "weights (tensor cores)");
        else    // with recompute only the row minima are needed (the monitor reads the distances)
            LK(TNLM_KCLASS_WEIGHTS,
               launch_weights(g, ws, p->patch, p->window, ws.u, st, !(p->recompute && !p->monitor)), "weights");
    }
    if (p->m2 > 0 && p->recompute) {
        float* bufs[2] = {ws.U0, ws.U1};
        for (int m = 0; m < p->m2; ++m) {
            const bool last = m == p->m2 - 1;
            LK(TNLM_KCLASS_GJ, launch_gj_fused(g, ws, p->patch, p->window, p->h, p->mu_hat, ws.u, bufs[m & 1],
                                               last ? nullptr : bufs[(m + 1) & 1], last ? d_f : nullptr,
                                               p->clamp, st),
               "gauss-jacobi (distances recomputed)");
        }
    } else if (p->m2 > 0) {
        float* bufs[2] = {ws.U0, ws.U1};
        for (int m = 0; m < p->m2; ++m) {
            const bool last = m == p->m2 - 1;
            LK(TNLM_KCLASS_GJ, launch_gj_sweep(g, ws, p->window, p->h, p->mu_hat, ws.u, bufs[m & 1],
                               last ? nullptr : bufs[(m + 1) & 1], last ? d_f : nullptr, p->clamp,
                               st),
               "gauss-jacobi");
        }
    } else {
        LK(TNLM_KCLASS_GJ, launch_finalize_nogj(g, ws, ws.u, d_f, p->clamp, st), "finalize");
    }
    if (p->monitor)
        LK(TNLM_KCLASS_CGLS, launch_tnlm_energy(g, ws, p->window, p->h, d_f, st), "TNLM term monitor");
    LK(TNLM_KCLASS_CGLS, launch_iter_scalars(g, ws, gj_blocks(g), p->monitor != 0, st), "monitors");
    return TNLM_OK;
}

// Monitor: the data term of the final image, ||sqrt(w)(y - P f)||^2, into
// st.res_final (one more projection after the last outer iteration).
tnlm_status final_data_term(tnlm_geometry* g, const float* d_y, const float* d_f, cudaStream_t st) {
    Workspace& ws = g->ws;
    LK(TNLM_KCLASS_PREP, launch_prep_dual(g, d_f, ws.R, ws.T, st), "prep");
    ProjOut o{};
    o.mode = 1; o.r = ws.r; o.z = ws.z; o.y = d_y; o.sw = ws.sw; o.part = ws.part;
    LK(TNLM_KCLASS_PROJECT, launch_project(g, ws.R, ws.T, o, st), "project");
    LK(TNLM_KCLASS_CGLS, launch_sum_partials(ws.part, g->N * proj_blocks_per_phase(g), ws.st.res_final, st),
       "data term");
    return TNLM_OK;
}

// One outer iteration captured as a CUDA graph on a handle-owned stream and
// replayed on the caller's stream.  The key is everything the captured
// launches depend on: the parameters that shape them, the caller's y and f
// pointers, the workspace allocation (by generation, not address), the
// launch tuning and the sweep's wait limit (a kernel argument).
struct GraphState {
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    tnlm_params p{};
    const float* y = nullptr;
    float* f = nullptr;
    unsigned long long ws_gen = 0;
    long wait_limit = 0;
    unsigned tune_gen = 0;
    long long launches[TNLM_KCLASS_COUNT] = {0, 0, 0, 0, 0, 0};  // kernels per replay
};

bool same_shape(const tnlm_params& a, const tnlm_params& b) {
    return a.mu_hat == b.mu_hat && a.h == b.h && a.beta == b.beta && a.patch == b.patch &&
           a.window == b.window && a.m1 == b.m1 && a.m2 == b.m2 && a.data_step == b.data_step &&
           a.clamp == b.clamp && a.precision == b.precision && a.monitor == b.monitor &&
           a.recompute == b.recompute;
}

tnlm_status ensure_graph(tnlm_geometry* g, const tnlm_params* p, const float* d_y, float* d_f) {
    GraphState* G = (GraphState*)g->graph;
    if (!G) g->graph = G = new GraphState();
    if (G->exec && G->y == d_y && G->f == d_f && G->ws_gen == g->ws_gen && same_shape(G->p, *p) &&
        G->tune_gen == g->tune_gen && G->wait_limit == g_gj_wait_limit)
        return TNLM_OK;
    if (G->exec) {
        cudaGraphExecDestroy(G->exec);
        G->exec = nullptr;
    }
    if (!G->cap) CK(cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking), "capture stream");
    long long before[TNLM_KCLASS_COUNT];
    for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) before[c] = g->launches[c];
    const unsigned mask = g->prof_mask;
    g->prof_mask = 0;
    CK(cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    tnlm_status s = outer_iteration(g, p, d_y, d_f, G->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(G->cap, &graph);
    g->prof_mask = mask;
    for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) {
        G->launches[c] = g->launches[c] - before[c];
        g->launches[c] = before[c];
    }
    if (s != TNLM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    const cudaError_t ei = cudaGraphInstantiate(&G->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        G->exec = nullptr;
        return cuda_fail(ei, "graph instantiate");
    }
    G->p = *p;
    G->y = d_y;
    G->f = d_f;
    G->ws_gen = g->ws_gen;
    G->wait_limit = g_gj_wait_limit;
    G->tune_gen = g->tune_gen;
    return TNLM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: measures the launch choices of the two kernels whose best shape
// depends on the device and the workload -- the number of view groups (CTAs)
// per backprojection tile, and for the TMA sweep the number of pixel tiles
// per CTA together with the window schedule (the whole window per work unit,
// or its rows in two halves as separate units) -- and keeps the fastest.
// Results are cached per device and shape.
// ---------------------------------------------------------------------------
std::atomic<unsigned long long> g_uid{1};
std::mutex g_tune_mu;
std::map<std::array<int, 8>, std::array<int, 3>> g_tune_cache;

std::array<int, 8> tune_key(const tnlm_geometry* g, const tnlm_params* p) {
    return {g->device, g->nx, g->ny, g->N, g->V, g->B, p->window, p->patch};
}

void set_tuning(tnlm_geometry* g, int bp_groups, int gj_tpb, int gj_split) {
    if (g->tune_bp_groups != bp_groups || g->tune_gj_tpb != gj_tpb || g->tune_gj_split != gj_split ||
        g->tune_gen == 0) {
        g->tune_bp_groups = bp_groups;
        g->tune_gj_tpb = gj_tpb;
        g->tune_gj_split = gj_split;
        g->tune_gen++;
    }
}

// Device time (ms) of one call of fn, the median-free mean of 'reps' calls
// after one warm-up call.
template <class F>
tnlm_status time_calls(cudaStream_t st, int reps, F fn, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a), "event");
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_fail(e, "event");
    }
    e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    *ms = t / reps;
    return TNLM_OK;
}

tnlm_status autotune(tnlm_geometry* g, const tnlm_params* p, const float* d_y, const float* d_winv,
                     const float* d_f0, cudaStream_t st) {
    const std::array<int, 8> key = tune_key(g, p);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            set_tuning(g, it->second[0], it->second[1], it->second[2]);
            return TNLM_OK;
        }
    }
    tnlm_status s = ensure_ws(g, (p->window - 1) / 2, p->k_outer < 1 ? 1 : p->k_outer, st);
    if (s != TNLM_OK) return s;
    Workspace& ws = g->ws;
    const size_t nimg = (size_t)g->N * g->nx * g->ny, nsg = (size_t)g->N * g->V * g->B;
    void* fbuf = nullptr;
    cudaError_t e = dev_alloc(&fbuf, sizeof(float) * nimg);
    if (e != cudaSuccess) return cuda_fail(e, "autotune scratch");
    float* f = (float*)fbuf;
    const unsigned mask = g->prof_mask;
    g->prof_mask = 0;
    long long before[TNLM_KCLASS_COUNT];
    for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) before[c] = g->launches[c];
    // one outer iteration from the caller's start image fills the workspace
    // (distances, minima, iterates) with the data the timed launches read
    auto run = [&]() -> tnlm_status {
        CK(cudaMemcpyAsync(f, d_f0, sizeof(float) * nimg, cudaMemcpyDeviceToDevice, st), "copy");
        CK(cudaMemsetAsync(ws.st.iter, 0, sizeof(int), st), "reset");
        LK(TNLM_KCLASS_PREP, launch_sqrt(d_winv, ws.sw, nsg, ws.st.err, st), "sqrt");
        tnlm_status r = outer_iteration(g, p, d_y, f, st);
        if (r != TNLM_OK) return r;
        int best_g = 1, best_t = 1, best_s = 1;
        float tb = INFINITY;
        for (int G = 1; G <= bp_max_groups(g); ++G) {
            g->tune_bp_groups = G;
            float ms = 0.f;
            r = time_calls(st, 3, [&]() { return launch_backproject(g, ws.z, ws.gr, nullptr, ws.bps, st); }, &ms);
            if (r != TNLM_OK) return r;
            if (ms < tb) { tb = ms; best_g = G; }
        }
        if (p->m2 > 0) {
            float tg = INFINITY;
            for (int sp = 1; sp <= 2; ++sp)
                for (int t = 1; t <= 3; ++t) {
                    g->tune_gj_tpb = t;
                    g->tune_gj_split = sp;
                    float ms = 0.f;
                    r = time_calls(st, 3, [&]() {
                        return launch_gj_sweep(g, ws, p->window, p->h, p->mu_hat, ws.u, ws.U0, ws.U1, nullptr,
                                               p->clamp, st);
                    }, &ms);
                    if (r != TNLM_OK) return r;
                    if (ms < tg) { tg = ms; best_t = t; best_s = sp; }
                }
        }
        g->tune_bp_groups = 0;
        g->tune_gj_tpb = 0;
        g->tune_gj_split = 0;
        set_tuning(g, best_g, best_t, p->m2 > 0 ? best_s : 0);
        CK(cudaMemsetAsync(ws.st.iter, 0, sizeof(int), st), "reset");
        CK(cudaMemsetAsync(ws.st.err, 0, sizeof(int), st), "reset");
        CK(cudaStreamSynchronize(st), "sync");
        return TNLM_OK;
    };
    s = run();
    g->prof_mask = mask;
    for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) g->launches[c] = before[c];
    cudaStreamSynchronize(st);
    cudaFree(fbuf);
    if (s != TNLM_OK) {
        g->tune_bp_groups = 0;
        g->tune_gj_tpb = 0;
        g->tune_gj_split = 0;
        return s;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {g->tune_bp_groups, g->tune_gj_tpb, g->tune_gj_split};
    return TNLM_OK;
}

// ---------------------------------------------------------------------------
// Batched reconstruction: one outer iteration of every slice of the batch is
// captured as a single CUDA graph -- one branch per slice, forked from and
// joined to a capture stream -- and the graph is replayed once per outer
// iteration, so kernels of different slices run side by side.  When slices
// with fewer iterations finish, the graph is re-captured without them.
// ---------------------------------------------------------------------------
// Device-side control of the batched loop graph.  Per slice: its own
// iteration counter and its stopping rule (k_outer; tol checked every
// 'every' iterations, the rule tnlm_reconstruct applies on the host).
struct GateSlice {
    const int* iter;
    const double* hist_rel;
    double tol;
    int k_outer;
    int every;
};

// Runs at the top of every pass of the WHILE body: sets each slice's IF
// condition (does it take another outer iteration?) and the WHILE
// condition (does any slice?).  A pass where no slice runs is the last.
__global__ void k_batch_gate(const GateSlice* __restrict__ s, const cudaGraphConditionalHandle* __restrict__ hs,
                             int n, cudaGraphConditionalHandle hw) {
    int any = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const GateSlice q = s[j];
        const int done = *q.iter;
        bool run = done < q.k_outer;
        if (run && q.tol > 0.0 && done > 0 && done % q.every == 0 && q.hist_rel[done - 1] < q.tol)
            run = false;
        cudaGraphSetConditional(hs[j], run ? 1u : 0u);
        any |= run ? 1 : 0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(hw, any ? 1u : 0u);
}

struct BatchItem {
    unsigned long long uid;
    unsigned tune_gen;
    unsigned long long ws_gen;
    long wait_limit;
    const float* y;
    float* f;
    tnlm_params p;
    bool operator==(const BatchItem& o) const {
        return uid == o.uid && tune_gen == o.tune_gen && ws_gen == o.ws_gen &&
               wait_limit == o.wait_limit && y == o.y && f == o.f && same_shape(p, o.p);
    }
};

struct BatchState {
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraphExec_t exec = nullptr;
    std::vector<BatchItem> key;
    std::vector<std::array<long long, TNLM_KCLASS_COUNT>> launches;   // per slice and replay
    // the whole run as one launch: a WHILE node around a gate kernel and one
    // IF node per slice (that slice's outer iteration)
    cudaGraphExec_t loop_exec = nullptr;
    std::vector<BatchItem> loop_key;
    bool loop_broken = false;          // the runtime refused the loop graph once: use replays
    GateSlice* gate = nullptr;                       // device [gate_cap]
    cudaGraphConditionalHandle* gate_h = nullptr;    // device [gate_cap]
    size_t gate_cap = 0;
    std::vector<cudaGraphConditionalHandle> handles;  // the loop graph's IF handles
    std::vector<std::array<long long, TNLM_KCLASS_COUNT>> loop_launches;   // per slice and iteration
};
std::mutex g_batch_mu;
std::map<int, BatchState*> g_batch;   // per device
thread_local int g_last_batch_loop = 0;

// Captures one outer iteration of every slice on the capture stream (which
// is already capturing) as a fork/join of per-slice branches.
tnlm_status capture_body(BatchState* B, const std::vector<tnlm_geometry*>& gs,
                         const std::vector<const tnlm_params*>& ps, const std::vector<const float*>& ys,
                         const std::vector<float*>& fs, cudaError_t* ce) {
    tnlm_status s = TNLM_OK;
    cudaError_t e = cudaEventRecord(B->events[0], B->cap);
    for (size_t j = 0; j < gs.size() && s == TNLM_OK && e == cudaSuccess; ++j) {
        tnlm_geometry* g = gs[j];
        e = cudaStreamWaitEvent(B->streams[j], B->events[0], 0);
        if (e != cudaSuccess) break;
        long long before[TNLM_KCLASS_COUNT];
        for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) before[c] = g->launches[c];
        const unsigned mask = g->prof_mask;
        g->prof_mask = 0;
        s = outer_iteration(g, ps[j], ys[j], fs[j], B->streams[j]);
        g->prof_mask = mask;
        for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) {
            B->launches[j][c] = g->launches[c] - before[c];
            g->launches[c] = before[c];
        }
        if (s != TNLM_OK) break;
        e = cudaEventRecord(B->events[j + 1], B->streams[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cap, B->events[j + 1], 0);
    }
    *ce = e;
    return s;
}

tnlm_status batch_resources(BatchState* B, size_t n) {
    if (!B->cap) CK(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking), "capture stream");
    while (B->streams.size() < n) {
        cudaStream_t t;
        CK(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking), "batch stream");
        B->streams.push_back(t);
    }
    while (B->events.size() < n + 1) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch event");
        B->events.push_back(ev);
    }
    if (B->gate_cap < n) {
        if (B->gate) cudaFree(B->gate);
        if (B->gate_h) cudaFree(B->gate_h);
        B->gate = nullptr;
        B->gate_h = nullptr;
        B->gate_cap = 0;
        void* p = nullptr;
        CK(dev_alloc(&p, sizeof(GateSlice) * n), "batch gate");
        B->gate = (GateSlice*)p;
        CK(dev_alloc(&p, sizeof(cudaGraphConditionalHandle) * n), "batch gate");
        B->gate_h = (cudaGraphConditionalHandle*)p;
        B->gate_cap = n;
    }
    B->launches.assign(n, {});
    return TNLM_OK;
}

// The whole batched run as ONE graph launch: a conditional WHILE node whose
// body is a gate kernel followed by one conditional IF node per slice, the
// IF body being that slice's outer iteration.  The gate decides on the
// device which slices take another iteration (k_outer, tolerance), so
// slices with different iteration counts or tolerances all run in the one
// launch.  Returns TNLM_OK with *built = false when the runtime does not
// accept the loop graph (the caller then replays the single-iteration
// graph).
tnlm_status loop_graph(BatchState* B, const std::vector<tnlm_geometry*>& gs,
                       const std::vector<const tnlm_params*>& ps, const std::vector<const float*>& ys,
                       const std::vector<float*>& fs, bool* built) {
    *built = false;
    if (B->loop_broken) return TNLM_OK;
    const char* env = getenv("TNLM_BATCH_REPLAY");     // force the replay path
    if (env && env[0] == '1') return TNLM_OK;
    const size_t n = gs.size();
    std::vector<BatchItem> key(n);
    for (size_t j = 0; j < n; ++j)
        key[j] = {gs[j]->uid, gs[j]->tune_gen, gs[j]->ws_gen, g_gj_wait_limit, ys[j], fs[j], *ps[j]};
    if (B->loop_exec && key == B->loop_key) {
        *built = true;
        return TNLM_OK;
    }
    if (B->loop_exec) {
        cudaGraphExecDestroy(B->loop_exec);
        B->loop_exec = nullptr;
    }
    tnlm_status s = batch_resources(B, n);
    if (s != TNLM_OK) return s;
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle hw;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node, gate;
    std::vector<cudaGraphConditionalHandle> hs(n);
    cudaGraph_t body = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, graph, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hw;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
        if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    for (size_t j = 0; j < n && e == cudaSuccess; ++j)
        e = cudaGraphConditionalHandleCreate(&hs[j], body, 0, 0);
    if (e == cudaSuccess) {
        const GateSlice* a0 = B->gate;
        const cudaGraphConditionalHandle* a1 = B->gate_h;
        int a2 = (int)n;
        cudaGraphConditionalHandle a3 = hw;
        void* args[] = {&a0, &a1, &a2, &a3};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)k_batch_gate;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(256);
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&gate, body, nullptr, 0, &kp);
    }
    for (size_t j = 0; j < n && e == cudaSuccess && s == TNLM_OK; ++j) {
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hs[j];
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t ifn;
        e = cudaGraphAddNode(&ifn, body, &gate, nullptr, 1, &ip);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(B->cap, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        tnlm_geometry* g = gs[j];
        long long before[TNLM_KCLASS_COUNT];
        for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) before[c] = g->launches[c];
        const unsigned mask = g->prof_mask;
        g->prof_mask = 0;
        s = outer_iteration(g, ps[j], ys[j], fs[j], B->cap);
        g->prof_mask = mask;
        for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) {
            B->launches[j][c] = g->launches[c] - before[c];
            g->launches[c] = before[c];
        }
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(B->cap, &out);
    }
    if (s != TNLM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->loop_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        B->loop_exec = nullptr;
        B->loop_broken = true;
        return TNLM_OK;
    }
    B->loop_key = key;
    B->handles = hs;
    B->loop_launches = B->launches;
    *built = true;
    return TNLM_OK;
}

tnlm_status batch_graph(BatchState* B, const std::vector<tnlm_geometry*>& gs,
                        const std::vector<const tnlm_params*>& ps, const std::vector<const float*>& ys,
                        const std::vector<float*>& fs) {
    std::vector<BatchItem> key(gs.size());
    for (size_t j = 0; j < gs.size(); ++j)
        key[j] = {gs[j]->uid, gs[j]->tune_gen, gs[j]->ws_gen, g_gj_wait_limit, ys[j], fs[j], *ps[j]};
    if (B->exec && key == B->key) return TNLM_OK;
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    tnlm_status s = batch_resources(B, gs.size());
    if (s != TNLM_OK) return s;
    CK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaSuccess;
    s = capture_body(B, gs, ps, ys, fs, &e);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(B->cap, &graph);
    if (s != TNLM_OK || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (s != TNLM_OK) return s;
        return cuda_fail(e != cudaSuccess ? e : ee, "batch capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        B->exec = nullptr;
        return cuda_fail(ei, "batch graph instantiate");
    }
    B->key = key;
    return TNLM_OK;
}

// Copies the monitors of the last reconstruction of g into rep and returns
// the status its device flags call for (flags are cleared).
tnlm_status read_report(tnlm_geometry* g, const tnlm_params* p, int done, tnlm_report* rep,
                        cudaStream_t st) {
    Workspace& ws = g->ws;
    int err = 0;
    CK(cudaMemcpyAsync(&err, ws.st.err, sizeof(int), cudaMemcpyDeviceToHost, st), "readback");
    const size_t n = done > 0 ? (size_t)done : 1;
    std::vector<double> hrel(n), hres(n), hcl(n), htn(n);
    double rfin = 0.0;
    if (done > 0) {
        CK(cudaMemcpyAsync(hrel.data(), ws.st.hist_rel, sizeof(double) * done, cudaMemcpyDeviceToHost,
                           st), "readback");
        CK(cudaMemcpyAsync(hres.data(), ws.st.hist_res, sizeof(double) * done, cudaMemcpyDeviceToHost,
                           st), "readback");
        CK(cudaMemcpyAsync(hcl.data(), ws.st.hist_clamp, sizeof(double) * done, cudaMemcpyDeviceToHost,
                           st), "readback");
        CK(cudaMemcpyAsync(htn.data(), ws.st.hist_tnlm, sizeof(double) * done, cudaMemcpyDeviceToHost,
                           st), "readback");
        if (p->monitor)
            CK(cudaMemcpyAsync(&rfin, ws.st.res_final, sizeof(double), cudaMemcpyDeviceToHost, st),
               "readback");
    }
    CK(cudaStreamSynchronize(st), "sync");
    if (rep) {
        // mu of Eq. 1 is mu_hat * beta (Eq. 7); the data term of the image
        // after iteration k is the residual the next iteration starts from
        const double mu = p->mu_hat * p->beta;
        rep->iterations = done;
        rep->rel_change = done > 0 ? hrel[done - 1] : 0.0;
        rep->data_residual = done > 0 ? hres[done - 1] : 0.0;
        rep->clamped = done > 0 ? (long long)hcl[done - 1] : 0;
        rep->tnlm_term = done > 0 && p->monitor ? htn[done - 1] : 0.0;
        rep->objective = done > 0 && p->monitor ? rfin + 0.5 * mu * htn[done - 1] : 0.0;
        for (int k = 0; k < done; ++k) {
            const double dk = k + 1 < done ? hres[k + 1] : rfin;
            if (rep->rel_change_hist) rep->rel_change_hist[k] = hrel[k];
            if (rep->residual_hist) rep->residual_hist[k] = hres[k];
            if (rep->clamped_hist) rep->clamped_hist[k] = (long long)hcl[k];
            if (p->monitor) {
                if (rep->tnlm_hist) rep->tnlm_hist[k] = htn[k];
                if (rep->data_hist) rep->data_hist[k] = dk;
                if (rep->objective_hist) rep->objective_hist[k] = dk + 0.5 * mu * htn[k];
            }
        }
    }
    if (err) {
        CK(cudaMemsetAsync(ws.st.err, 0, sizeof(int), st), "reset");
        if (err & 16) {   // a bounded wait of the TMA sweep ran out
            // a sweep that stopped early may leave half-done tile counters
            CK(cudaMemsetAsync(ws.gjcnt, 0, sizeof(int) * (size_t)gj_blocks(g), st), "reset");
            return fail(TNLM_ERR_TIMEOUT, "a device-side wait timed out (flags 0x%x)", err);
        }
        return fail(TNLM_ERR_NUMERIC, "non-finite value met on the device (flags 0x%x)", err);
    }
    return TNLM_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* tnlm_last_error(void) { return g_err; }

void tnlm_debug_fail_alloc_after(int n) { g_fail_after.store(n > 0 ? n : 0); }

void tnlm_debug_wait_limit(long polls) { g_gj_wait_limit = polls >= 0 ? polls : kSpinLimit; }

tnlm_status tnlm_create_geometry(const tnlm_geometry_desc* d, tnlm_geometry** out) {
    g_err[0] = 0;
    if (!out) return fail(TNLM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(TNLM_ERR_INVALID_ARG, "desc is NULL");
    if (d->nx < 1 || d->ny < 1 || d->nx > 8192 || d->ny > 8192)
        return fail(TNLM_ERR_INVALID_ARG, "nx, ny must be in [1, 8192]");
    if (d->n_phases < 3 || d->n_phases > 4096)
        return fail(TNLM_ERR_INVALID_ARG, "n_phases must be in [3, 4096]");
    if (d->n_views < 1 || d->n_bins < 1)
        return fail(TNLM_ERR_INVALID_ARG, "n_views and n_bins must be >= 1");
    if (d->n_bins > 4096) return fail(TNLM_ERR_INVALID_ARG, "n_bins must be <= 4096");
    if ((long long)d->n_phases * d->n_views > 1000000)
        return fail(TNLM_ERR_INVALID_ARG, "n_phases * n_views too large");
    if (!(d->pixel_mm > 0) || !(d->bin_mm > 0) || !isfinite(d->pixel_mm) || !isfinite(d->bin_mm))
        return fail(TNLM_ERR_INVALID_ARG, "pixel_mm and bin_mm must be finite and > 0");
    const double half_diag = 0.5 * d->pixel_mm * sqrt((double)d->nx * d->nx + (double)d->ny * d->ny);
    if (!(d->sid_mm > half_diag) || !isfinite(d->sid_mm))
        return fail(TNLM_ERR_INVALID_ARG, "sid_mm must exceed the image half-diagonal %.3f mm", half_diag);
    if (!(d->sdd_mm > d->sid_mm + half_diag) || !isfinite(d->sdd_mm))
        return fail(TNLM_ERR_INVALID_ARG, "sdd_mm must exceed sid_mm + image half-diagonal");
    if (d->detector != TNLM_DETECTOR_ARC) return fail(TNLM_ERR_INVALID_ARG, "only the arc detector is supported");
    const double fan = 0.5 * d->n_bins * d->bin_mm / d->sdd_mm;
    if (!(fan < 1.4)) return fail(TNLM_ERR_INVALID_ARG, "fan half-angle must be < 1.4 rad");
    if (!d->view_angles_rad) return fail(TNLM_ERR_INVALID_ARG, "view_angles_rad is NULL");
    const size_t NV = (size_t)d->n_phases * d->n_views;
    for (size_t k = 0; k < NV; ++k)
        if (!isfinite(d->view_angles_rad[k])) return fail(TNLM_ERR_INVALID_ARG, "non-finite view angle");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || d->device < 0 || d->device >= ndev) {
        cudaGetLastError();
        return fail(TNLM_ERR_INVALID_ARG, "device %d not available", d->device);
    }
    DeviceGuard dg(d->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");

    tnlm_geometry* g = new tnlm_geometry();
    g->uid = g_uid.fetch_add(1);
    g->device = d->device;
    g->nx = d->nx; g->ny = d->ny; g->N = d->n_phases; g->V = d->n_views; g->B = d->n_bins;
    g->pixel = d->pixel_mm; g->bin_mm = d->bin_mm; g->sid = d->sid_mm; g->sdd = d->sdd_mm;

    // per-view (cos t, sin t), per-bin (cos g, sin g), per-ray chord constants (FP64 -> FP32)
    std::vector<float2> hv(NV), hb(g->B);
    std::vector<float4> hr(NV * g->B);
    std::vector<int4> hc(NV);
    const double dg_ = g->bin_mm / g->sdd;
    for (int b = 0; b < g->B; ++b) {
        const double ga = (b - 0.5 * (g->B - 1)) * dg_;
        hb[b] = make_float2((float)cos(ga), (float)sin(ga));
    }
    // Ray (view, bin): direction u = -(cos(t+g), sin(t+g)); in pixel units about
    // the isocentre its line is u_x Y - u_y X = c0 with c0 = sid sin(g) / pixel.
    // A ray with |u_x| >= |u_y| marches over columns: at the left edge of column
    // k it is at row coordinate alpha + kk k; otherwise over rows, at column
    // coordinate alpha + kk k at the bottom edge of row k.
    const double hx = 0.5 * g->nx, hy = 0.5 * g->ny, sidp = g->sid / g->pixel;
    for (size_t v = 0; v < NV; ++v) {
        const double t = d->view_angles_rad[v];
        hv[v] = make_float2((float)cos(t), (float)sin(t));
        // the ray direction turns monotonically with b, so the rays of one
        // class normally form one bin run (at most one class change within a
        // fan narrower than 90 degrees); otherwise both ranges are the whole
        // detector and the backprojector tests every ray's class
        int first_cls = 0, prev_cls = 0, changes = 0, split = g->B;
        for (int b = 0; b < g->B; ++b) {
            const double ga = (b - 0.5 * (g->B - 1)) * dg_;
            const double ux = -cos(t + ga), uy = -sin(t + ga);
            const double c0 = sidp * sin(ga);
            double kk, alpha, ik, L;
            if (fabs(ux) >= fabs(uy)) {
                kk = uy / ux;
                alpha = c0 / ux - kk * hx + hy;
                ik = uy != 0.0 ? fabs(ux / uy) : INFINITY;
                L = g->pixel / fabs(ux);
            } else {
                kk = ux / uy;
                alpha = -c0 / uy - kk * hy + hx;
                ik = ux != 0.0 ? fabs(uy / ux) : INFINITY;
                L = -g->pixel / fabs(uy);
            }
            hr[v * g->B + b] = make_float4((float)kk, (float)alpha, (float)ik, (float)L);
            const int cls = L > 0.0 ? 0 : 1;
            if (b == 0) first_cls = cls;
            else if (cls != prev_cls && changes++ == 0) split = b;
            prev_cls = cls;
        }
        const int last = g->B - 1;
        if (changes > 1) hc[v] = make_int4(0, last, 0, last);
        else if (first_cls == 0) hc[v] = make_int4(0, split - 1, split, last);
        else hc[v] = make_int4(split, last, 0, split - 1);
    }
    // taps of the discrete equiangular ramp kernel (initial FBP)
    std::vector<float> ht(2 * (size_t)g->B - 1);
    for (int n = -(g->B - 1); n <= g->B - 1; ++n) {
        double v = 0.0;
        if (n == 0) v = 1.0 / (8.0 * dg_ * dg_);
        else if (n % 2 != 0) {
            const double sn = sin(n * dg_);
            v = -1.0 / (2.0 * 9.8696044010893586188 * sn * sn);   // pi^2
        }
        ht[n + g->B - 1] = (float)v;
    }
    void *pv = nullptr, *pb = nullptr, *pr = nullptr, *pt = nullptr, *pc = nullptr;
    cudaError_t e = dev_alloc(&pv, sizeof(float2) * NV);
    if (e == cudaSuccess) e = dev_alloc(&pb, sizeof(float2) * g->B);
    if (e == cudaSuccess) e = dev_alloc(&pr, sizeof(float4) * NV * g->B);
    if (e == cudaSuccess) e = dev_alloc(&pt, sizeof(float) * ht.size());
    if (e == cudaSuccess) e = dev_alloc(&pc, sizeof(int4) * NV);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(pv); cudaFree(pb); cudaFree(pr); cudaFree(pt); cudaFree(pc);
        delete g;
        return fail(e == cudaErrorMemoryAllocation ? TNLM_ERR_OOM : TNLM_ERR_CUDA,
                    "geometry table allocation failed: %s", cudaGetErrorString(e));
    }
    g->d_view = (float2*)pv; g->d_bin = (float2*)pb; g->d_ray = (float4*)pr;
    g->d_fbp_taps = (float*)pt;
    g->d_vcls = (int4*)pc;
    e = cudaMemcpy(pv, hv.data(), sizeof(float2) * NV, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pb, hb.data(), sizeof(float2) * g->B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pr, hr.data(), sizeof(float4) * NV * g->B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pt, ht.data(), sizeof(float) * ht.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pc, hc.data(), sizeof(int4) * NV, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        tnlm_destroy_geometry(g);
        return cuda_fail(e, "geometry table upload");
    }
    e = prepare_backproject(&g->cta_slots_bp);
    if (e == cudaSuccess) e = prepare_weights(&g->cta_slots_gj);
    if (e == cudaSuccess) e = prepare_weights_tc();
    if (e == cudaSuccess) e = prepare_gj_fused();
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) {
        tnlm_destroy_geometry(g);
        return cuda_fail(e, "kernel attributes");
    }
    *out = g;
    return TNLM_OK;
}

void tnlm_destroy_geometry(tnlm_geometry* g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->d_view);
    cudaFree(g->d_bin);
    cudaFree(g->d_ray);
    cudaFree(g->d_fbp_taps);
    cudaFree(g->d_vcls);
    cudaFree(g->ws.base);
    if (g->graph) {
        GraphState* G = (GraphState*)g->graph;
        if (G->exec) cudaGraphExecDestroy(G->exec);
        if (G->cap) cudaStreamDestroy(G->cap);
        delete G;
    }
    if (g->prof) {
        Profiler* P = (Profiler*)g->prof;
        for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
        delete P;
    }
    delete g;
}

tnlm_status tnlm_profile_enable(tnlm_geometry* g, unsigned int class_mask) {
    g_err[0] = 0;
    if (check_geom_handle(g) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    if (class_mask >> TNLM_KCLASS_COUNT) return fail(TNLM_ERR_INVALID_ARG, "unknown kernel class in mask");
    g->prof_mask = class_mask;
    return TNLM_OK;
}

tnlm_status tnlm_profile_read(tnlm_geometry* g, double* ms, long long* launches, int reset) {
    g_err[0] = 0;
    if (check_geom_handle(g) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    CK(cudaDeviceSynchronize(), "sync");
    double t[TNLM_KCLASS_COUNT] = {0, 0, 0, 0, 0, 0};
    Profiler* P = (Profiler*)g->prof;
    if (P) {
        for (size_t k = 0; k < P->used; ++k) {
            float e = 0.f;
            CK(cudaEventElapsedTime(&e, P->ev[2 * k], P->ev[2 * k + 1]), "event time");
            t[P->cls[k]] += e;
        }
    }
    for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) {
        if (ms) ms[c] = t[c];
        if (launches) launches[c] = g->launches[c];
    }
    if (reset) {
        if (P) P->used = 0;
        for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) g->launches[c] = 0;
    }
    return TNLM_OK;
}

tnlm_status tnlm_project(const tnlm_geometry* gc, const float* d_img, float* d_sino, void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(gc) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    if (!d_img || !d_sino) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_img) || !aligned16(d_sino)) return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    tnlm_geometry* g = const_cast<tnlm_geometry*>(gc);
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    tnlm_status s = ensure_ws(g, g->ws.base ? g->ws.rho : 0, g->ws.base ? g->ws.kcap : 1, st);
    if (s != TNLM_OK) return s;
    LK(TNLM_KCLASS_PREP, launch_prep_dual(g, d_img, g->ws.R, g->ws.T, st), "prep");
    ProjOut o{};
    o.mode = 0; o.q = d_sino;
    LK(TNLM_KCLASS_PROJECT, launch_project(g, g->ws.R, g->ws.T, o, st), "project");
    return TNLM_OK;
}

tnlm_status tnlm_project_static(const tnlm_geometry* gc, const float* d_img, float* d_sino,
                                void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(gc) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    if (!d_img || !d_sino) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_img) || !aligned16(d_sino)) return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    tnlm_geometry* g = const_cast<tnlm_geometry*>(gc);
    // row-major and column-major padded copies of the image (float2 pairs),
    // back to back
    const size_t nR = align_up(2 * (size_t)g->N * g->ny * (g->nx + 4), 64);
    const size_t nT = 2 * (size_t)g->N * g->nx * (g->ny + 4);
    if (nR + nT > static_scratch_floats())
        return fail(TNLM_ERR_INVALID_ARG,
                    "image too large for the static scratch: needs %zu floats, the array holds %zu",
                    nR + nT, static_scratch_floats());
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    float* base = nullptr;
    CK(static_scratch_ptr(&base), "cudaGetSymbolAddress");
    // the array keeps the previous call's contents: the zero pads are restored
    CK(cudaMemsetAsync(base, 0, sizeof(float) * (nR + nT), st), "scratch clear");
    LK(TNLM_KCLASS_PREP, launch_prep_dual(g, d_img, base, base + nR, st), "prep");
    ProjOut o{};
    o.mode = 0; o.q = d_sino;
    LK(TNLM_KCLASS_PROJECT, launch_project(g, base, base + nR, o, st), "project");
    return TNLM_OK;
}

tnlm_status tnlm_backproject(const tnlm_geometry* gc, const float* d_sino, float* d_img, void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(gc) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    if (!d_img || !d_sino) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_img) || !aligned16(d_sino)) return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    tnlm_geometry* g = const_cast<tnlm_geometry*>(gc);
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    tnlm_status s = ensure_ws(g, g->ws.base ? g->ws.rho : 0, g->ws.base ? g->ws.kcap : 1, st);
    if (s != TNLM_OK) return s;
    LK(TNLM_KCLASS_BACKPROJECT, launch_backproject(g, d_sino, d_img, nullptr, g->ws.bps, st), "backproject");
    return TNLM_OK;
}

tnlm_status tnlm_fbp(const tnlm_geometry* gc, const float* d_y, float* d_img, void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(gc) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    if (!d_y || !d_img) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_y) || !aligned16(d_img)) return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    tnlm_geometry* g = const_cast<tnlm_geometry*>(gc);
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    tnlm_status s = ensure_ws(g, g->ws.base ? g->ws.rho : 0, g->ws.base ? g->ws.kcap : 1, st);
    if (s != TNLM_OK) return s;
    LK(TNLM_KCLASS_PREP, launch_fbp(g, d_y, g->ws.t, d_img, st), "fbp");
    return TNLM_OK;
}

tnlm_status tnlm_fbp_phases(const tnlm_geometry* gc, const float* d_y, float* d_img, void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(gc) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    if (!d_y || !d_img) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_y) || !aligned16(d_img)) return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    tnlm_geometry* g = const_cast<tnlm_geometry*>(gc);
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    tnlm_status s = ensure_ws(g, g->ws.base ? g->ws.rho : 0, g->ws.base ? g->ws.kcap : 1, st);
    if (s != TNLM_OK) return s;
    LK(TNLM_KCLASS_PREP, launch_fbp_phases(g, d_y, g->ws.t, d_img, st), "fbp per phase");
    return TNLM_OK;
}

tnlm_status tnlm_weights_size(const tnlm_geometry* g, const tnlm_params* p, size_t* dist_bytes,
                              size_t* norm_bytes) {
    g_err[0] = 0;
    if (check_geom_handle(g) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    tnlm_status s = check_params(p);
    if (s != TNLM_OK) return s;
    const size_t npx = (size_t)g->nx * g->ny * g->N;
    if (dist_bytes) *dist_bytes = 4 * npx * p->window * p->window;
    if (norm_bytes) *norm_bytes = 4 * 4 * npx;
    return TNLM_OK;
}

tnlm_status tnlm_workspace_bytes(const tnlm_geometry* g, const tnlm_params* p, size_t* bytes) {
    g_err[0] = 0;
    if (check_geom_handle(g) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    tnlm_status s = check_params(p);
    if (s != TNLM_OK) return s;
    if (!bytes) return fail(TNLM_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = ws_layout(g, (p->window - 1) / 2, p->k_outer < 1 ? 1 : p->k_outer).total;
    return TNLM_OK;
}

tnlm_status tnlm_weights(const tnlm_geometry* gc, const tnlm_params* p, const float* d_g,
                         float* d_dist, float* d_norm, void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(gc) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    tnlm_status s = check_params(p);
    if (s != TNLM_OK) return s;
    if (!d_g || !d_dist || !d_norm) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_g) || !aligned16(d_dist) || !aligned16(d_norm))
        return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    tnlm_geometry* g = const_cast<tnlm_geometry*>(gc);
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    s = ensure_ws(g, (p->window - 1) / 2, g->ws.base ? g->ws.kcap : 1, st);
    if (s != TNLM_OK) return s;
    if (p->precision == TNLM_PREC_MIXED)
        LK(TNLM_KCLASS_WEIGHTS, launch_weights_tc(g, g->ws, p->patch, p->window, d_g, st), "weights (tensor cores)");
    else
        LK(TNLM_KCLASS_WEIGHTS, launch_weights(g, g->ws, p->patch, p->window, d_g, st), "weights");
    LK(TNLM_KCLASS_WEIGHTS, launch_weights_norm(g, g->ws, p->window, p->h, st), "weights normalisers");
    LK(TNLM_KCLASS_WEIGHTS, launch_weights_export(g, g->ws, p->window, d_dist, d_norm, st), "weights export");
    return TNLM_OK;
}

tnlm_status tnlm_reconstruct(const tnlm_geometry* gc, const tnlm_params* p, const float* d_y,
                             const float* d_winv, float* d_f, tnlm_report* rep, void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(gc) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    tnlm_status s = check_params(p);
    if (s != TNLM_OK) return s;
    if (!d_y || !d_winv || !d_f) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_y) || !aligned16(d_winv) || !aligned16(d_f))
        return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    tnlm_geometry* g = const_cast<tnlm_geometry*>(gc);
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    s = ensure_ws(g, (p->window - 1) / 2, p->k_outer < 1 ? 1 : p->k_outer, st);
    if (s != TNLM_OK) return s;
    Workspace& ws = g->ws;
    const size_t nsg = (size_t)g->N * g->V * g->B;
    CK(cudaMemsetAsync(ws.st.iter, 0, sizeof(int), st), "reset");
    LK(TNLM_KCLASS_PREP, launch_sqrt(d_winv, ws.sw, nsg, ws.st.err, st), "sqrt");
    const bool sync = rep != nullptr || p->tol > 0.0;
    int done = 0;
    // replay a captured iteration unless kernels are being timed individually
    const bool graphs = g->prof_mask == 0 && p->k_outer > 1;
    if (graphs) {
        s = ensure_graph(g, p, d_y, d_f);
        if (s != TNLM_OK) return s;
    }
    for (int k = 0; k < p->k_outer; ++k) {
        if (graphs) {
            GraphState* G = (GraphState*)g->graph;
            CK(cudaGraphLaunch(G->exec, st), "graph launch");
            for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) g->launches[c] += G->launches[c];
        } else {
            s = outer_iteration(g, p, d_y, d_f, st);
            if (s != TNLM_OK) return s;
        }
        done = k + 1;
        if (p->tol > 0.0 && (done % p->tol_check_every == 0 || done == p->k_outer)) {
            double rel = 0.0;
            CK(cudaMemcpyAsync(&rel, ws.st.hist_rel + k, sizeof(double), cudaMemcpyDeviceToHost, st),
               "readback");
            CK(cudaStreamSynchronize(st), "sync");
            if (rel < p->tol) break;
        }
    }
    if (p->monitor && done > 0) {
        s = final_data_term(g, d_y, d_f, st);
        if (s != TNLM_OK) return s;
    }
    if (sync) return read_report(g, p, done, rep, st);
    return TNLM_OK;
}

tnlm_status tnlm_autotune(tnlm_geometry* g, const tnlm_params* p, const float* d_y,
                          const float* d_winv, const float* d_f0, int* bp_groups, int* gj_tiles,
                          int* gj_split, void* stream) {
    g_err[0] = 0;
    if (check_geom_handle(g) != TNLM_OK) return TNLM_ERR_INVALID_ARG;
    tnlm_status s = check_params(p);
    if (s != TNLM_OK) return s;
    if (!d_y || !d_winv || !d_f0) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer");
    if (!aligned16(d_y) || !aligned16(d_winv) || !aligned16(d_f0))
        return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    DeviceGuard dg(g->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    s = autotune(g, p, d_y, d_winv, d_f0, (cudaStream_t)stream);
    if (s != TNLM_OK) return s;
    if (bp_groups) *bp_groups = g->tune_bp_groups;
    if (gj_tiles) *gj_tiles = g->tune_gj_tpb;
    if (gj_split) *gj_split = g->tune_gj_split;
    return TNLM_OK;
}

int tnlm_batch_last_was_loop(void) { return g_last_batch_loop; }

tnlm_status tnlm_reconstruct_batch(tnlm_geometry* const* geoms, const tnlm_params* params,
                                   int count, const float* const* d_y, const float* const* d_winv,
                                   float* const* d_f, tnlm_report* reports, int autotune_shapes,
                                   void* stream) {
    g_err[0] = 0;
    if (count < 1 || count > 4096) return fail(TNLM_ERR_INVALID_ARG, "count must be in [1, 4096]");
    if (!geoms || !params || !d_y || !d_winv || !d_f) return fail(TNLM_ERR_INVALID_ARG, "NULL array");
    int dev = -1, kmax = 0;
    for (int i = 0; i < count; ++i) {
        if (!geoms[i]) return fail(TNLM_ERR_INVALID_ARG, "geometry %d is NULL", i);
        tnlm_status s = check_params(&params[i]);
        if (s != TNLM_OK) return s;
        if (!d_y[i] || !d_winv[i] || !d_f[i]) return fail(TNLM_ERR_INVALID_ARG, "NULL buffer of slice %d", i);
        if (!aligned16(d_y[i]) || !aligned16(d_winv[i]) || !aligned16(d_f[i]))
            return fail(TNLM_ERR_INVALID_ARG, "buffers must be 16-byte aligned (slice %d)", i);
        if (dev < 0) dev = geoms[i]->device;
        if (geoms[i]->device != dev) return fail(TNLM_ERR_INVALID_ARG, "all slices must be on one device");
        for (int j = 0; j < i; ++j)
            if (geoms[j] == geoms[i]) return fail(TNLM_ERR_INVALID_ARG, "slice %d repeats a handle", i);
        kmax = params[i].k_outer > kmax ? params[i].k_outer : kmax;
    }
    DeviceGuard dg(dev);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> done(count, 0);
    for (int i = 0; i < count; ++i) {
        tnlm_geometry* g = geoms[i];
        const tnlm_params* p = &params[i];
        if (autotune_shapes && g->tune_gen == 0) {
            tnlm_status s = autotune(g, p, d_y[i], d_winv[i], d_f[i], st);
            if (s != TNLM_OK) return s;
        }
        tnlm_status s = ensure_ws(g, (p->window - 1) / 2, p->k_outer < 1 ? 1 : p->k_outer, st);
        if (s != TNLM_OK) return s;
        const size_t nsg = (size_t)g->N * g->V * g->B;
        CK(cudaMemsetAsync(g->ws.st.iter, 0, sizeof(int), st), "reset");
        LK(TNLM_KCLASS_PREP, launch_sqrt(d_winv[i], g->ws.sw, nsg, g->ws.st.err, st), "sqrt");
    }
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        BatchState*& B = g_batch[dev];
        if (!B) B = new BatchState();
        std::vector<tnlm_geometry*> gs;
        std::vector<const tnlm_params*> ps;
        std::vector<const float*> ys;
        std::vector<float*> fs;
        g_last_batch_loop = 0;
        for (int i = 0; i < count; ++i) {
            gs.push_back(geoms[i]); ps.push_back(&params[i]); ys.push_back(d_y[i]); fs.push_back(d_f[i]);
        }
        bool built = false;
        tnlm_status s = kmax > 0 ? loop_graph(B, gs, ps, ys, fs, &built) : TNLM_OK;
        if (s != TNLM_OK) return s;
        if (built) {
            std::vector<GateSlice> gh(count);
            for (int i = 0; i < count; ++i)
                gh[i] = {geoms[i]->ws.st.iter, geoms[i]->ws.st.hist_rel, params[i].tol, params[i].k_outer,
                         params[i].tol > 0.0 ? params[i].tol_check_every : 1};
            CK(cudaMemcpyAsync(B->gate, gh.data(), sizeof(GateSlice) * count, cudaMemcpyHostToDevice, st),
               "batch gate upload");
            CK(cudaMemcpyAsync(B->gate_h, B->handles.data(), sizeof(cudaGraphConditionalHandle) * count,
                               cudaMemcpyHostToDevice, st), "batch gate upload");
            CK(cudaGraphLaunch(B->loop_exec, st), "batch loop graph launch");
            for (int i = 0; i < count; ++i)
                CK(cudaMemcpyAsync(&done[i], geoms[i]->ws.st.iter, sizeof(int), cudaMemcpyDeviceToHost, st),
                   "readback");
            CK(cudaStreamSynchronize(st), "sync");
            for (int i = 0; i < count; ++i)
                for (int c = 0; c < TNLM_KCLASS_COUNT; ++c)
                    geoms[i]->launches[c] += (long long)done[i] * B->loop_launches[i][c];
            kmax = 0;     // done: skip the per-iteration replays below
            g_last_batch_loop = 1;
        }
        // replays of the single-iteration graph; slices leave it at their
        // k_outer or once their stopping rule holds (checked on the host)
        std::vector<char> live(count, 1);
        for (int k = 0; k < kmax; ++k) {
            gs.clear(); ps.clear(); ys.clear(); fs.clear();
            std::vector<int> idx;
            for (int i = 0; i < count; ++i)
                if (live[i] && k < params[i].k_outer) {
                    idx.push_back(i);
                    gs.push_back(geoms[i]); ps.push_back(&params[i]); ys.push_back(d_y[i]); fs.push_back(d_f[i]);
                }
            if (idx.empty()) break;
            s = batch_graph(B, gs, ps, ys, fs);
            if (s != TNLM_OK) return s;
            CK(cudaGraphLaunch(B->exec, st), "batch graph launch");
            for (size_t j = 0; j < gs.size(); ++j)
                for (int c = 0; c < TNLM_KCLASS_COUNT; ++c) gs[j]->launches[c] += B->launches[j][c];
            std::vector<int> chk;
            for (int i : idx) {
                done[i] = k + 1;
                if (params[i].tol > 0.0 && done[i] % params[i].tol_check_every == 0 && done[i] < params[i].k_outer)
                    chk.push_back(i);
            }
            if (!chk.empty()) {
                std::vector<double> rel(chk.size());
                for (size_t j = 0; j < chk.size(); ++j)
                    CK(cudaMemcpyAsync(&rel[j], geoms[chk[j]]->ws.st.hist_rel + k, sizeof(double),
                                       cudaMemcpyDeviceToHost, st), "readback");
                CK(cudaStreamSynchronize(st), "sync");
                for (size_t j = 0; j < chk.size(); ++j)
                    if (rel[j] < params[chk[j]].tol) live[chk[j]] = 0;
            }
        }
    }
    tnlm_status first = TNLM_OK;
    for (int i = 0; i < count; ++i) {
        if (params[i].monitor && done[i] > 0) {
            tnlm_status s = final_data_term(geoms[i], d_y[i], d_f[i], st);
            if (s != TNLM_OK) return s;
        }
    }
    for (int i = 0; i < count; ++i) {
        tnlm_status s = read_report(geoms[i], &params[i], done[i], reports ? &reports[i] : nullptr, st);
        if (s != TNLM_OK && first == TNLM_OK) first = s;
    }
    return first;
}

}  // extern "C"
