// Mixed-precision patch distances of Eq. 8 on the tensor cores (tcgen05).
//
// The distance between the patch of g_i at x and the patch of g_j at y is
//   D(x, y) = |P_i(x)|^2 + |P_j(y)|^2 - 2 <P_i(x), P_j(y)>.
// For a 16 x 8 tile of pixels x (the 128 rows M of a matrix product) and the
// (16 + 2 rho) x (8 + 2 rho) candidate pixels y its windows reach (the
// columns N), the cross terms of all pairs form one product A B^T with K =
// the d*d patch elements (zero padded to 32 or 64).  Up to 480 candidates
// (384 at K = 64) are one pass; more (e.g. 30 x 22 for a 15 x 15 window)
// are taken in two passes of whole candidate rows through the same
// accumulator.  The self-norms are summed exactly in FP32.  The cross term
// is taken in FP16 with an error-free split: v = 2^10 g is written as
// hi + lo with hi = fp16(v), lo = fp16(v - hi), and
//   <a, b> ~ a_hi.b_hi + a_lo.b_hi + a_hi.b_lo        (FP32 accumulation),
// which leaves out only a_lo.b_lo, ~2^-22 of the product; every FP16
// product is exact in the FP32 accumulator.  Distances carry an absolute
// error of a few 1e-9 against |P|^2 ~ 1e-2, far below h^2.
//
// One CTA per SM, persistent over (pair, tile) items.  Per item: the g tiles
// are staged in shared memory, each thread builds whole operand rows
// (canonical K-major layout, 8 x 16-byte core matrices, no swizzle), one
// thread issues, per pass, two N halves x three hi/lo products x K/16 K
// steps of tcgen05.mma into a 128 x (at most 512) FP32 accumulator in tensor
// memory and commits them to an mbarrier.  The epilogue warps read their 32 rows
// (tcgen05.ld), stage each 32-column chunk in shared memory to pick every
// pixel's own window, and store D (+inf where x + s leaves the image), the
// forward row minima and, through shared integer atomic minima, the
// backward minima -- the same outputs as the FP32 weights kernel.
#include "internal.cuh"
#include "tcgen05.cuh"

#include <cuda_fp16.h>

namespace tnlm {

constexpr int kTcTW = 16, kTcTH = 8;      // pixel tile (M = 128)
constexpr int kTcThreads = 512;
constexpr int kTcWG = kTcThreads / 128;   // warpgroups; each reads all 128 accumulator lanes
constexpr int kTcMinSmem = 117 * 1024;    // at least this much shared memory: one CTA per SM,
                                          // which keeps all 512 tensor-memory columns free
constexpr float kTcScale = 1024.f;

// Per (patch radius R, window radius RHO): tile and operand geometry and the
// shared-memory layout (bytes from a 1024-aligned base).
template <int R, int RHO>
struct TcGeo {
    static constexpr int d = 2 * R + 1, W = 2 * RHO + 1, D2 = d * d;
    static constexpr int KB = D2 <= 32 ? 32 : 64;        // K of one hi or lo block (zero padded)
    static constexpr int GIW = kTcTW + 2 * R, GIH = kTcTH + 2 * R;   // g_i tile
    static constexpr int CW = kTcTW + 2 * RHO, CH = kTcTH + 2 * RHO; // candidates
    static constexpr int GJW = CW + 2 * R, GJH = CH + 2 * R;        // g_j region
    static constexpr int NC = CW * CH;
    // candidates beyond what one pass holds (the accumulator's columns, and
    // the B operands' shared memory at K = 64) are taken in two passes of
    // whole candidate rows
    static constexpr int MaxN = KB == 64 ? 384 : 480;
    static constexpr int NPASS = NC <= MaxN ? 1 : 2;
    static constexpr int RP = (CH + NPASS - 1) / NPASS;            // candidate rows per pass
    static constexpr int NP = RP * CW;                             // candidates per pass
    static constexpr int NH = ((NP + 1) / 2 + 15) / 16 * 16;       // N of each of two MMAs
    static constexpr int ROWB = KB * 2;                            // bytes of one operand row
    static constexpr int SBO = (KB / 8) * 128;                     // step between 8-row groups
    static constexpr int a16(int v) { return (v + 15) / 16 * 16; }
    static constexpr int Ahi = 0;
    static constexpr int Alo = Ahi + 128 * ROWB;
    static constexpr int Bhi = Alo + 128 * ROWB;
    static constexpr int Blo = Bhi + 2 * NH * ROWB;
    static constexpr int Stage = Blo + 2 * NH * ROWB;              // per warp 32 x 32 floats
    static constexpr int Gi = Stage + (kTcThreads / 32) * 32 * 32 * 4;
    static constexpr int Gj = Gi + a16(GIW * GIH * 4);
    static constexpr int HiLo = Gj + a16(GJW * GJH * 4);           // FP16 hi, then lo
    static constexpr int Na = HiLo + a16(2 * (GIW * GIH + GJW * GJH) * 2);
    static constexpr int Nb = Na + 128 * 4;
    static constexpr int BM = Nb + a16(NC * 4);                    // backward minima
    static constexpr int Mf = BM + a16(NC * 4);                    // forward minima per warpgroup
    static constexpr int Bar = Mf + kTcWG * 128 * 4;
    static constexpr int Bytes = Bar + 16;
    static_assert(CW <= 32, "one tcgen05.ld chunk holds a candidate row");
    static_assert(2 * NH <= 512 && NH <= 256, "accumulator columns");
    static_assert(D2 <= 64, "patch elements");
    static_assert(Bytes + 2048 <= 227 * 1024, "shared memory (with the alignment slack and static part)");
};

struct TcArgs {
    const float* g;
    float* D;
    float* mins;
    float* U0;
    int* err;
    PadPlane pp;
    int nx, ny, N, tilesx, tilesy;
};

// byte offset of (row, k) in an operand block (K-major core matrices)
template <int SBO>
__device__ __forceinline__ int op_off(int row, int k) {
    return (row >> 3) * SBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Builds operand row r of a block whose patches are read from G (pitch P,
// FP16 halves at hb in Hi / Lo) around (cx, cy): K-major, zero padded to KB,
// 8 elements (one 16-byte chunk) at a time; returns the FP32 self-norm.
template <int KB, int SBO, int d>
__device__ __forceinline__ float build_row(unsigned char* ph, unsigned char* pl, int r, bool live,
                                           const float* G, int P, const __half* Hi, const __half* Lo,
                                           int hb, int cx, int cy) {
    constexpr int D2 = d * d;
    float nrm = 0.f;
#pragma unroll
    for (int c = 0; c < KB / 8; ++c) {
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t h2 = 0u, l2 = 0u;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = 8 * c + 2 * j + u;
                if (e < D2 && live) {
                    const int o = (cy + e / d) * P + cx + e % d;
                    const float v = G[o];
                    nrm = fmaf(v, v, nrm);
                    h2 |= (uint32_t)__half_as_ushort(Hi[hb + o]) << (16 * u);
                    l2 |= (uint32_t)__half_as_ushort(Lo[hb + o]) << (16 * u);
                }
            }
            hv[j] = h2;
            lv[j] = l2;
        }
        *(uint4*)(ph + op_off<SBO>(r, 8 * c)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *(uint4*)(pl + op_off<SBO>(r, 8 * c)) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
    return nrm;
}

template <int R, int RHO>
__global__ void __launch_bounds__(kTcThreads, 1) k_weights_tc(TcArgs a) {
    using T = TcGeo<R, RHO>;
    constexpr int d = T::d, W = T::W, CW = T::CW, CH = T::CH, NC = T::NC;
    constexpr int GIW = T::GIW, GIH = T::GIH, GJW = T::GJW, GJH = T::GJH;
    constexpr int NGI = GIW * GIH, NGJ = GJW * GJH;
    constexpr uint32_t IDESC = idesc_f16(128, T::NH, false);
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    float* stage = (float*)(sm + T::Stage);
    float* Gi = (float*)(sm + T::Gi);
    float* Gj = (float*)(sm + T::Gj);
    __half* Hi = (__half*)(sm + T::HiLo);             // hi of g_i tile, then of g_j region
    __half* Lo = Hi + NGI + NGJ;
    float* na = (float*)(sm + T::Na);
    float* nb = (float*)(sm + T::Nb);
    float* BM = (float*)(sm + T::BM);
    float* mfp = (float*)(sm + T::Mf);
    uint64_t* bar = (uint64_t*)(sm + T::Bar);
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = a.nx, ny = a.ny;
    const size_t npx = (size_t)nx * ny;
    if (warp == 0) {
        tmem_alloc512(&s_taddr);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    const uint32_t sbase = smem_u32(sm);
    const int per_pair = a.tilesx * a.tilesy;
    const int items = per_pair * a.N;
    // epilogue role: TMEM lanes 32q..32q+31 = pixels m; warpgroup wg takes
    // part of the candidate rows this warp's two pixel rows reach
    const int q = warp & 3, wg = warp >> 2;
    const int m = 32 * q + lane, px = m & 15, py = m >> 4;
    constexpr int NROW = 2 * RHO + 2;
    constexpr int RPW = (NROW + kTcWG - 1) / kTcWG;    // candidate rows per warpgroup
    const int cr0 = 2 * q + min(NROW, wg * RPW), cr1 = 2 * q + min(NROW, (wg + 1) * RPW);
    float* stg = stage + warp * 32 * 32;
    unsigned phase = 0;

    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int p = it / per_pair, t = it - p * per_pair;
        const int qj = (p + 1) % a.N;
        const int X0 = (t % a.tilesx) * kTcTW, Y0 = (t / a.tilesx) * kTcTH;
        const float* gp = a.g + p * npx;
        const float* gq = a.g + qj * npx;
        // (1) g tiles (zero outside the image), FP16 hi/lo of 2^10 g
        for (int e = tid; e < NGI + NGJ; e += kTcThreads) {
            float v;
            if (e < NGI) {
                const int x = X0 - R + e % GIW, y = Y0 - R + e / GIW;
                v = (x >= 0 && x < nx && y >= 0 && y < ny) ? gp[(size_t)y * nx + x] : 0.f;
                Gi[e] = v;
            } else {
                const int f = e - NGI;
                const int x = X0 - RHO - R + f % GJW, y = Y0 - RHO - R + f / GJW;
                v = (x >= 0 && x < nx && y >= 0 && y < ny) ? gq[(size_t)y * nx + x] : 0.f;
                Gj[f] = v;
            }
            const float s = v * kTcScale;
            const __half h = __float2half_rn(s);
            Hi[e] = h;
            Lo[e] = __float2half_rn(s - __half2float(h));
        }
        for (int e = tid; e < NC; e += kTcThreads) BM[e] = INFINITY;
        __syncthreads();
        // (2) A operand rows (the tile's patches) and their FP32 self-norms
        if (tid < 128)
            na[tid] = build_row<T::KB, T::SBO, d>(sm + T::Ahi, sm + T::Alo, tid, true, Gi, GIW, Hi, Lo, 0,
                                                 tid & 15, tid >> 4);
        if (a.U0) {  // padded copy of g_p: u^(0) of the Gauss-Jacobi sweeps
            for (int e = tid; e < kTcTW * kTcTH; e += kTcThreads) {
                const int x = X0 + (e & 15), y = Y0 + (e >> 4);
                if (x < nx && y < ny)
                    a.U0[p * a.pp.plane + (size_t)(y + a.pp.oy) * a.pp.px + x + a.pp.ox] =
                        Gi[((e >> 4) + R) * GIW + (e & 15) + R];
            }
        }
        float mf = INFINITY;
        const int x = X0 + px, y = Y0 + py;
        const bool pin = x < nx && y < ny;
        float* Dp = a.D + (size_t)p * (W * W) * a.pp.plane + (size_t)(y + a.pp.oy) * a.pp.px + x + a.pp.ox;
        bool stop = false;
        for (int pass = 0; pass < T::NPASS && !stop; ++pass) {
            const int crp = pass * T::RP;                              // first candidate row
            const int ncr = min(T::RP, CH - crp);
            // (3) B operand rows (this pass's candidates) and their self-norms
            for (int r = tid; r < 2 * T::NH; r += kTcThreads) {
                const bool live = r < ncr * CW;
                const int cx = r % CW, cy = crp + r / CW;
                const float nrm = build_row<T::KB, T::SBO, d>(sm + T::Bhi, sm + T::Blo, r, live, Gj, GJW, Hi,
                                                              Lo, NGI, cx, cy);
                if (live) nb[cy * CW + cx] = nrm;
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            // (4) the cross terms: 2 N halves x (hi.hi + lo.hi + hi.lo) x KB/16 K steps
            if (tid == 0) {
                tc_fence_after();
                const uint32_t Ah = sbase + T::Ahi, Al = sbase + T::Alo, Bh = sbase + T::Bhi, Bl = sbase + T::Blo;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t dt = taddr + (uint32_t)(h * T::NH);
                    const uint32_t bo = (uint32_t)(h * (T::NH / 8) * T::SBO);
                    int acc = 0;
#pragma unroll
                    for (int prod = 0; prod < 3; ++prod) {
                        const uint32_t A = prod == 1 ? Al : Ah;
                        const uint32_t Bm = prod == 2 ? Bl : Bh;
#pragma unroll
                        for (int ks = 0; ks < T::KB / 16; ++ks) {
                            umma_f16(dt, smem_desc(A + ks * 256, 128, T::SBO),
                                     smem_desc(Bm + bo + ks * 256, 128, T::SBO), IDESC, acc);
                            acc = 1;
                        }
                    }
                }
                umma_commit(bar);
            }
            if (!mbar_wait_bounded(bar, phase)) {
                s_abort = 1;
                atomicOr(a.err, 16);
                mbar_wait_bounded(bar, phase);    // let the products drain before leaving
            }
            phase ^= 1u;
            __syncthreads();                      // every thread takes the same exit decision
            tc_fence_after();
            if (s_abort) {
                stop = true;
                break;
            }
            // (5) epilogue of this pass's candidate rows
            const float nam = na[m];
            const int lo_r = max(cr0, crp), hi_r = min(cr1, crp + ncr);
            for (int cr = lo_r; cr < hi_r; ++cr) {
                uint32_t v[32];
                __syncwarp();
                tmem_ld32(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)((cr - crp) * CW), v);
#pragma unroll
                for (int c = 0; c < CW; ++c) stg[c * 32 + lane] = __uint_as_float(v[c]);
                const int sy = cr - py;            // window row of this pixel's shift
                if (sy < 0 || sy > 2 * RHO) continue;
                const int yy = y + sy - RHO;
                const bool rowok = pin && yy >= 0 && yy < ny;
#pragma unroll
                for (int sx = 0; sx < W; ++sx) {
                    const int c = px + sx;
                    const float cross = stg[c * 32 + lane];
                    const float dv = fmaxf(fmaf(-2.f / (kTcScale * kTcScale), cross, nam + nb[cr * CW + c]), 0.f);
                    const int xx = x + sx - RHO;
                    const bool ok = rowok && xx >= 0 && xx < nx;
                    const float val = ok ? dv : INFINITY;
                    if (pin) Dp[(size_t)(sy * W + sx) * a.pp.plane] = val;
                    mf = fminf(mf, val);
                    if (ok) atomicMin((int*)&BM[cr * CW + c], __float_as_int(val));
                }
            }
            tc_fence_before();
            __syncthreads();                      // TMEM and the B operands are free again
        }
        if (stop) break;
        mfp[wg * 128 + m] = mf;
        __syncthreads();
        // forward minima of the tile's pixels, backward minima of its reach
        if (tid < 128) {
            const int xm = X0 + (tid & 15), ym = Y0 + (tid >> 4);
            float v = mfp[tid];
#pragma unroll
            for (int w2 = 1; w2 < kTcWG; ++w2) v = fminf(v, mfp[w2 * 128 + tid]);
            if (xm < nx && ym < ny) {
                a.mins[p * npx + (size_t)ym * nx + xm] = v;
                if (!(v < INFINITY)) atomicOr(a.err, 4);
            }
        }
        int* mprev = (int*)(a.mins + (size_t)(a.N + qj) * npx);
        for (int e = tid; e < NC; e += kTcThreads) {
            const int xx = X0 - RHO + e % CW, yy = Y0 - RHO + e / CW;
            const float v = BM[e];
            if (xx >= 0 && xx < nx && yy >= 0 && yy < ny && v < INFINITY)
                atomicMin(mprev + (size_t)yy * nx + xx, __float_as_int(v));
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc512(taddr);
}

template <int R, int RHO>
static size_t tc_smem() {
    const size_t b = (size_t)TcGeo<R, RHO>::Bytes + 1024;
    return b > (size_t)kTcMinSmem ? b : (size_t)kTcMinSmem;
}

bool weights_tc_supported(int patch, int window) {
    return (patch == 1 || patch == 3 || patch == 5 || patch == 7) && (window & 1) && window >= 3 &&
           window <= 15;
}

template <int R, int RHO>
static cudaError_t launch_tc_rw(const TcArgs& a, int sms, cudaStream_t st) {
    const int items = a.tilesx * a.tilesy * a.N;
    const int grid = items < sms ? items : sms;
    k_weights_tc<R, RHO><<<grid, kTcThreads, tc_smem<R, RHO>(), st>>>(a);
    return cudaGetLastError();
}

template <int R>
static cudaError_t launch_tc_r(const TcArgs& a, int rho, int sms, cudaStream_t st) {
    switch (rho) {
        case 1: return launch_tc_rw<R, 1>(a, sms, st);
        case 2: return launch_tc_rw<R, 2>(a, sms, st);
        case 3: return launch_tc_rw<R, 3>(a, sms, st);
        case 4: return launch_tc_rw<R, 4>(a, sms, st);
        case 5: return launch_tc_rw<R, 5>(a, sms, st);
        case 6: return launch_tc_rw<R, 6>(a, sms, st);
        case 7: return launch_tc_rw<R, 7>(a, sms, st);
        default: return cudaErrorInvalidValue;
    }
}

#define TNLM_TC_ROW(X, R) X(R, 1) X(R, 2) X(R, 3) X(R, 4) X(R, 5) X(R, 6) X(R, 7)
#define TNLM_TC_ALL(X) TNLM_TC_ROW(X, 0) TNLM_TC_ROW(X, 1) TNLM_TC_ROW(X, 2) TNLM_TC_ROW(X, 3)

// Opt the tensor-core variants into their shared memory (geometry creation).
cudaError_t prepare_weights_tc() {
    cudaError_t e = cudaSuccess;
#define TNLM_TC_PREP(R, RHO)                                                                       \
    if (e == cudaSuccess)                                                                          \
        e = cudaFuncSetAttribute(k_weights_tc<R, RHO>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)tc_smem<R, RHO>());
    TNLM_TC_ALL(TNLM_TC_PREP)
#undef TNLM_TC_PREP
    return e;
}

cudaError_t launch_weights_tc(const tnlm_geometry* g, const Workspace& ws, int patch, int window,
                              const float* gimg, cudaStream_t st) {
    if (!weights_tc_supported(patch, window)) return cudaErrorInvalidValue;
    TcArgs a;
    a.g = gimg; a.D = ws.D; a.mins = ws.mins; a.U0 = ws.U0; a.err = ws.st.err; a.pp = ws.pp;
    a.nx = g->nx; a.ny = g->ny; a.N = g->N;
    a.tilesx = (g->nx + kTcTW - 1) / kTcTW;
    a.tilesy = (g->ny + kTcTH - 1) / kTcTH;
    const size_t npx = (size_t)g->nx * g->ny;
    cudaError_t e = cudaMemsetAsync(ws.mins + (size_t)g->N * npx, 0x7f, sizeof(float) * g->N * npx, st);
    if (e != cudaSuccess) return e;
    const int sms = g->num_sms > 0 ? g->num_sms : 1;
    switch ((patch - 1) / 2) {
        case 0: return launch_tc_r<0>(a, (window - 1) / 2, sms, st);
        case 1: return launch_tc_r<1>(a, (window - 1) / 2, sms, st);
        case 2: return launch_tc_r<2>(a, (window - 1) / 2, sms, st);
        case 3: return launch_tc_r<3>(a, (window - 1) / 2, sms, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnlm
