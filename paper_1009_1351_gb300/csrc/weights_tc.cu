// Mixed-precision patch distances of Eq. 8 on the tensor cores (tcgen05).
//
// The distance between the patch of g_i at x and the patch of g_j at y is
//   D(x, y) = |P_i(x)|^2 + |P_j(y)|^2 - 2 <P_i(x), P_j(y)>.
// For a 16 x 8 tile of pixels x (the 128 rows M of a matrix product) and the
// (16 + 2 rho) x (8 + 2 rho) candidate pixels y its windows reach (the
// columns N, at most 480), the cross terms of all pairs form one product
// A B^T with K = the d*d patch elements.  The self-norms are summed exactly
// in FP32.  The cross term is taken in FP16 with an error-free split:
// v = 2^10 g is written as hi + lo with hi = fp16(v), lo = fp16(v - hi), and
//   <a, b> ~ a_hi.b_hi + a_lo.b_hi + a_hi.b_lo        (FP32 accumulation),
// which leaves out only a_lo.b_lo, ~2^-22 of the product; every FP16
// product is exact in the FP32 accumulator.  Distances carry an absolute
// error of a few 1e-9 against |P|^2 ~ 1e-2, far below h^2.
//
// One CTA per SM, persistent over (pair, tile) items.  Per item: the g tiles
// are staged in shared memory, each thread builds whole operand rows
// (canonical K-major layout, 8 x 16-byte core matrices, no swizzle), one
// thread issues 12 tcgen05.mma (two N halves of 240, three hi/lo products,
// two K steps of 16) into a 128 x 480 FP32 accumulator in tensor memory and
// commits them to an mbarrier.  The epilogue warps read their 32 rows
// (tcgen05.ld), stage each 32-column chunk in shared memory to pick every
// pixel's own window, and store D (+inf where x + s leaves the image), the
// forward row minima and, through shared integer atomic minima, the
// backward minima -- the same outputs as the FP32 weights kernel.
#include "internal.cuh"
#include "tcgen05.cuh"

#include <cuda_fp16.h>

namespace tnlm {

constexpr int kTcTW = 16, kTcTH = 8;      // pixel tile (M = 128)
constexpr int kTcNHalf = 240;              // N of one MMA; two of them
constexpr int kTcN = 2 * kTcNHalf;
constexpr int kTcKB = 32;                  // K of one hi or lo operand block (d*d <= 25, zero padded)
constexpr int kTcThreads = 512;
constexpr int kTcWG = kTcThreads / 128;      // warpgroups; each reads all 128 accumulator lanes
constexpr int kTcRowBytes = kTcKB * 2;     // one operand row of a block: 64 bytes
constexpr int kTcSBO = (kTcKB / 8) * 128;  // byte step between 8-row groups (4 core matrices of 128 B)
constexpr float kTcScale = 1024.f;

// shared-memory layout (bytes from a 1024-aligned base)
constexpr int kTcAhi = 0;
constexpr int kTcAlo = kTcAhi + 128 * kTcRowBytes;           // 8 KB each
constexpr int kTcBhi = kTcAlo + 128 * kTcRowBytes;
constexpr int kTcBlo = kTcBhi + kTcN * kTcRowBytes;           // 30 KB each
constexpr int kTcStage = kTcBlo + kTcN * kTcRowBytes;         // per warp 32 x 32 floats
constexpr int kTcGi = kTcStage + (kTcThreads / 32) * 32 * 32 * 4;  // FP32 tile of g_i (<= 20 x 12)
constexpr int kTcGj = kTcGi + 256 * 4;                        // FP32 region of g_j (<= 30 x 22)
constexpr int kTcHiLo = kTcGj + 672 * 4;                      // FP16 hi / lo of both (2 x (256 + 672))
constexpr int kTcNa = kTcHiLo + 2 * (256 + 672) * 2;
constexpr int kTcNb = kTcNa + 128 * 4;
constexpr int kTcBM = kTcNb + kTcN * 4;                       // backward minima (<= 26 x 18)
constexpr int kTcMf = kTcBM + 480 * 4;                        // forward minima of each warpgroup
constexpr int kTcBar = kTcMf + kTcWG * 128 * 4;
constexpr int kTcBytes = kTcBar + 16;
static_assert(kTcBytes + 1024 > 116 * 1024, "one CTA per SM keeps all of tensor memory free");

struct TcArgs {
    const float* g;
    float* D;
    float* mins;
    float* U0;
    int* err;
    PadPlane pp;
    int nx, ny, N, tilesx, tilesy;
};

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// FP16 A and B (bits 7-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at 24.
constexpr uint32_t kTcIdesc = idesc_f16(128, kTcNHalf, false);

// byte offset of (row, k) in an operand block (K-major core matrices)
__device__ __forceinline__ int op_off(int row, int k) {
    return (row >> 3) * kTcSBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

template <int R, int RHO>
__global__ void __launch_bounds__(kTcThreads, 1) k_weights_tc(TcArgs a) {
    constexpr int d = 2 * R + 1, W = 2 * RHO + 1, D2 = d * d;
    constexpr int GIW = kTcTW + 2 * R, GIH = kTcTH + 2 * R;                   // g_i tile
    constexpr int CW = kTcTW + 2 * RHO, CH = kTcTH + 2 * RHO;                // candidates
    constexpr int GJW = CW + 2 * R, GJH = CH + 2 * R;                         // g_j region
    constexpr int NC = CW * CH;                                              // candidates used
    static_assert(NC <= kTcN && GIW * GIH <= 256 && GJW * GJH <= 672 && D2 <= kTcKB, "tile sizes");
    static_assert(CW <= 32, "one tcgen05.ld chunk holds a candidate row");
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    float* stage = (float*)(sm + kTcStage);
    float* Gi = (float*)(sm + kTcGi);
    float* Gj = (float*)(sm + kTcGj);
    __half* Hi = (__half*)(sm + kTcHiLo);             // hi of g_i tile, then of g_j region
    __half* Lo = Hi + 256 + 672;
    float* na = (float*)(sm + kTcNa);
    float* nb = (float*)(sm + kTcNb);
    float* BM = (float*)(sm + kTcBM);
    float* mfp = (float*)(sm + kTcMf);
    uint64_t* bar = (uint64_t*)(sm + kTcBar);
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
    // half of the candidate rows this warp's two pixel rows reach
    const int q = warp & 3, wg = warp >> 2;
    const int m = 32 * q + lane, px = m & 15, py = m >> 4;
    constexpr int NROW = 2 * RHO + 2;
    constexpr int RPW = (NROW + kTcWG - 1) / kTcWG;    // candidate rows per warpgroup
    const int cr0 = 2 * q + min(NROW, wg * RPW), cr1 = 2 * q + min(NROW, (wg + 1) * RPW);
    float* stg = stage + warp * 32 * 32;
    unsigned phase = 0;

    for (int it = blockIdx.x; it < items; it += gridDim.x, phase ^= 1u) {
        const int p = it / per_pair, t = it - p * per_pair;
        const int qj = (p + 1) % a.N;
        const int X0 = (t % a.tilesx) * kTcTW, Y0 = (t / a.tilesx) * kTcTH;
        const float* gp = a.g + p * npx;
        const float* gq = a.g + qj * npx;
        // (1) g tiles (zero outside the image), FP16 hi/lo of 2^10 g
        for (int e = tid; e < GIW * GIH + GJW * GJH; e += kTcThreads) {
            float v;
            if (e < GIW * GIH) {
                const int x = X0 - R + e % GIW, y = Y0 - R + e / GIW;
                v = (x >= 0 && x < nx && y >= 0 && y < ny) ? gp[(size_t)y * nx + x] : 0.f;
                Gi[e] = v;
            } else {
                const int f = e - GIW * GIH;
                const int x = X0 - RHO - R + f % GJW, y = Y0 - RHO - R + f / GJW;
                v = (x >= 0 && x < nx && y >= 0 && y < ny) ? gq[(size_t)y * nx + x] : 0.f;
                Gj[f] = v;
            }
            const float s = v * kTcScale;
            const __half h = __float2half_rn(s);
            const int o = e < GIW * GIH ? e : 256 + (e - GIW * GIH);
            Hi[o] = h;
            Lo[o] = __float2half_rn(s - __half2float(h));
        }
        for (int e = tid; e < NC; e += kTcThreads) BM[e] = INFINITY;
        __syncthreads();
        // (2) operand rows and FP32 self-norms: rows 0..127 of A, 0..479 of B
        for (int row = tid; row < 128 + kTcN; row += kTcThreads) {
            const bool isA = row < 128;
            const int r = isA ? row : row - 128;
            uint32_t hv[kTcKB / 2], lv[kTcKB / 2];   // pairs of FP16, element 2j in the low half
            float nrm = 0.f;
            const bool live = isA || r < NC;
            const int cx = isA ? (r & 15) : r % CW, cy = isA ? (r >> 4) : r / CW;
            const float* G = isA ? Gi : Gj;
            const int P = isA ? GIW : GJW;
            const int hb = isA ? 0 : 256;
#pragma unroll
            for (int j = 0; j < kTcKB / 2; ++j) {
                uint32_t h2 = 0u, l2 = 0u;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = 2 * j + u;
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
            unsigned char* ph = sm + (isA ? kTcAhi : kTcBhi);
            unsigned char* pl = sm + (isA ? kTcAlo : kTcBlo);
#pragma unroll
            for (int c = 0; c < kTcKB / 8; ++c) {
                *(uint4*)(ph + op_off(r, 8 * c)) = make_uint4(hv[4 * c], hv[4 * c + 1], hv[4 * c + 2], hv[4 * c + 3]);
                *(uint4*)(pl + op_off(r, 8 * c)) = make_uint4(lv[4 * c], lv[4 * c + 1], lv[4 * c + 2], lv[4 * c + 3]);
            }
            if (isA) na[r] = nrm;
            else nb[r] = nrm;
        }
        if (a.U0) {  // padded copy of g_p: u^(0) of the Gauss-Jacobi sweeps
            for (int e = tid; e < kTcTW * kTcTH; e += kTcThreads) {
                const int x = X0 + (e & 15), y = Y0 + (e >> 4);
                if (x < nx && y < ny)
                    a.U0[p * a.pp.plane + (size_t)(y + a.pp.oy) * a.pp.px + x + a.pp.ox] =
                        Gi[((e >> 4) + R) * GIW + (e & 15) + R];
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        // (3) the cross terms: 2 N halves x (hi.hi + lo.hi + hi.lo) x 2 K steps
        if (tid == 0) {
            tc_fence_after();
            const uint32_t Ah = sbase + kTcAhi, Al = sbase + kTcAlo, Bh = sbase + kTcBhi, Bl = sbase + kTcBlo;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t dt = taddr + (uint32_t)(h * kTcNHalf);
                const uint32_t bo = (uint32_t)(h * (kTcNHalf / 8) * kTcSBO);
                int acc = 0;
#pragma unroll
                for (int prod = 0; prod < 3; ++prod) {
                    const uint32_t A = prod == 1 ? Al : Ah;
                    const uint32_t Bm = prod == 2 ? Bl : Bh;
#pragma unroll
                    for (int ks = 0; ks < kTcKB / 16; ++ks) {
                        umma_f16(dt, smem_desc(A + ks * 256, 128, kTcSBO),
                                 smem_desc(Bm + bo + ks * 256, 128, kTcSBO), kTcIdesc, acc);
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
        __syncthreads();                      // every thread takes the same exit decision
        tc_fence_after();
        if (s_abort) break;
        // (4) epilogue
        float mf = INFINITY;
        const int x = X0 + px, y = Y0 + py;
        const bool pin = x < nx && y < ny;
        const float nam = na[m];
        float* Dp = a.D + (size_t)p * (W * W) * a.pp.plane + (size_t)(y + a.pp.oy) * a.pp.px + x + a.pp.ox;
        for (int cr = cr0; cr < cr1; ++cr) {
            uint32_t v[32];
            __syncwarp();
            tmem_ld32(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(cr * CW), v);
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
        mfp[wg * 128 + m] = mf;
        tc_fence_before();
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

static size_t tc_smem() { return (size_t)kTcBytes + 1024; }

bool weights_tc_supported(int patch, int window) {
    return (patch == 1 || patch == 3 || patch == 5) && window >= 3 && window <= 11;
}

template <int R, int RHO>
static cudaError_t launch_tc_rw(const TcArgs& a, int sms, cudaStream_t st) {
    const int items = a.tilesx * a.tilesy * a.N;
    const int grid = items < sms ? items : sms;
    k_weights_tc<R, RHO><<<grid, kTcThreads, tc_smem(), st>>>(a);
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
        default: return cudaErrorInvalidValue;
    }
}

#define TNLM_TC_ALL(X) \
    X(0, 1) X(0, 2) X(0, 3) X(0, 4) X(0, 5) X(1, 1) X(1, 2) X(1, 3) X(1, 4) X(1, 5) X(2, 1) X(2, 2) X(2, 3) X(2, 4) X(2, 5)

// Opt the tensor-core variants into their shared memory (geometry creation).
cudaError_t prepare_weights_tc() {
    cudaError_t e = cudaSuccess;
#define TNLM_TC_PREP(R, RHO)                                                                       \
    if (e == cudaSuccess)                                                                          \
        e = cudaFuncSetAttribute(k_weights_tc<R, RHO>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)tc_smem());
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
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnlm
