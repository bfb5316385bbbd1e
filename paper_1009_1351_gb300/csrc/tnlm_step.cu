// TNLM step (Sec. 2.2-2.3): Eq. 8 weights from g^(k), then M2 Gauss-Jacobi
// sweeps of Eq. 7, then the positivity truncation.
//
// K4 (k_weights) computes, for each cyclic pair (i, i+1) and every pixel x
// and shift s of the W x W window, the patch distance
//   D_i(x, s) = sum_{|p|<=r} (g_i(x+p) - g_{i+1}(x+s+p))^2   (zero outside the image)
// once, and stores it in a single array that both directions read (the
// symmetric reuse of Sec. 2.3: omega_{i,i+1}(x, x+s) and omega_{i+1,i}(x+s, x)
// share exp(-D/h^2) before normalisation).  Eq. 8 is evaluated as a stable
// softmax, exp(-(D - m)/h^2) / Z with m the row minimum; K4 also produces m
// for both directions:
//   m_next_i(x)     = min_s D_i(x, s)            (row x of phase i toward i+1)
//   m_prev_{i+1}(y) = min_s D_i(y - s, s)        (row y of phase i+1 toward i)
// A block owns a 64 x TY tile T of one pair (TY = 32 - 2r rounded down to a
// multiple of 4).  For each shift, pass 1 forms 32 rows of horizontal patch
// sums (8 adjacent sums per thread from a register window of squared
// differences) into one of two shared buffers while pass 2 sums the other
// buffer vertically (one column, TY/4 rows per thread), stores the forward
// distances, keeps the forward row minima in registers and folds each
// distance into a shared array of backward minima at x + s; one barrier per
// shift.  The backward minima of T's rho-neighbourhood are combined across
// blocks with an integer atomic min at the end.
//
// K5 (k_gj) is one Gauss-Jacobi sweep, one thread per pixel of one phase.  It
// streams the two distance planes that touch phase i (pair i forward at x,
// pair i-1 backward at x - s) and forms both normalisers on the fly:
//   u_i^+(x) = g_i(x)/(mu+1) + mu/(2mu+2) [ sum_s e_p u_{i-1}(x-s) / sum_s e_p
//                                         + sum_s e_n u_{i+1}(x+s) / sum_s e_n ]
// with e = 2^(log2(e) (m - D) / h^2).  Blocks are ordered tile-major, phase-
// minor, so the two reads of a distance plane (by phase i and phase i+1)
// happen close together in time and the second is served from L2.
#include "internal.cuh"

#include <math.h>

namespace tnlm {

struct WArgs {
    const float* g;
    float* D;
    float* mins;
    float* U0;
    int* err;
    PadPlane pp;
    int nx, ny, N, rho, W;
};

// Shared-memory geometry of k_weights.  The output tile is 64 columns by
// TY rows, TY = 4 floor((32 - 2R) / 4), so that the TY + 2R rows of
// horizontal sums fit one 32-row pass.
template <int R>
struct WGeo {
    static constexpr int TX = 64;
    static constexpr int TY = (32 - 2 * R) / 4 * 4;
    static constexpr int HR = TY + 2 * R;       // rows of horizontal sums (<= 32)
    static constexpr int RPT = TY / 4;          // output rows per thread
    static constexpr int NQ = 8 + 2 * R;        // taps of 8 adjacent horizontal sums
    static constexpr int NQ4 = (NQ + 3) / 4;    // float4 loads of a g_i row segment
    // g_i tile: TY + 2R rows, pitch a multiple of 4 with pitch/4 odd (float4
    // loads of two consecutive rows fall in distinct bank groups)
    static constexpr int GIW0 = (TX + 2 * R + 3) / 4 * 4;
    static constexpr int GIW = ((GIW0 / 4) & 1) ? GIW0 : GIW0 + 4;
    static constexpr int GIH = TY + 2 * R;
    static constexpr int HP = 68;               // horizontal-sum pitch (68 / 4 odd)
    static constexpr int BMW = TX + 2 * ((kMaxWindow - 1) / 2);   // backward-minimum pitch
    int GJW, GJH, GJS, BMH;
    __host__ __device__ explicit WGeo(int rho) {
        GJW = (TX + 2 * rho + 2 * R) | 1;       // odd: rows of a warp hit distinct banks
        GJH = TY + 2 * rho + 2 * R;
        GJS = (GJW * GJH + 3) / 4 * 4;          // keeps the next buffer 16-byte aligned
        BMH = TY + 2 * rho;
    }
    __host__ __device__ size_t floats() const {
        return (size_t)GIW * GIH + (size_t)GJS + 2 * 32 * (size_t)HP + (size_t)BMW * BMH;
    }
};

// SLIDE (patch <= 7, window <= 15): pass 1 keeps the task's g_p segment in
// registers for the whole kernel and, along a row of shifts (sy fixed, sx
// rising), a sliding register window of the g_q segment that takes one new
// value per shift; the shift loop is unrolled over sx so every window index
// is static.  Otherwise pass 1 reloads both segments from shared memory for
// every shift.
template <int R, bool SLIDE>
__global__ void __launch_bounds__(256, 4) k_weights(WArgs a) {
    using G = WGeo<R>;
    extern __shared__ __align__(16) float sm[];
    const int rho = a.rho, W = a.W;
    const G L(rho);
    float* Gi = sm;                                  // g_p at rows Y0-R.., columns X0-R..
    float* Gj = Gi + G::GIW * G::GIH;                // g_q at rows Y0-rho-R.., columns X0-rho-R..
    float* H = Gj + L.GJS;                           // two buffers of 32 x HP
    float* BM = H + 2 * 32 * G::HP;                  // backward minima at rows Y0-rho.., columns X0-rho..
    const int p = blockIdx.z, q = (p + 1) % a.N;
    const int X0 = blockIdx.x * G::TX, Y0 = blockIdx.y * G::TY;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = a.nx, ny = a.ny;
    const size_t npx = (size_t)nx * ny;
    const float* gp = a.g + p * npx;
    const float* gq = a.g + q * npx;
    for (int r = warp; r < G::GIH; r += 8)
        for (int c = lane; c < G::GIW; c += 32) {
            const int x = X0 - R + c, y = Y0 - R + r;
            Gi[r * G::GIW + c] = (x >= 0 && x < nx && y >= 0 && y < ny) ? gp[(size_t)y * nx + x] : 0.f;
        }
    for (int r = warp; r < L.GJH; r += 8)
        for (int c = lane; c < L.GJW; c += 32) {
            const int x = X0 - rho - R + c, y = Y0 - rho - R + r;
            Gj[r * L.GJW + c] = (x >= 0 && x < nx && y >= 0 && y < ny) ? gq[(size_t)y * nx + x] : 0.f;
        }
    for (int e = tid; e < G::BMW * L.BMH; e += 256) BM[e] = INFINITY;
    __syncthreads();
    if (a.U0) {  // padded copy of g_p: u^(0) of the Gauss-Jacobi sweeps
        for (int r = warp; r < G::TY; r += 8)
            for (int c = lane; c < G::TX; c += 32) {
                const int x = X0 + c, y = Y0 + r;
                if (x < nx && y < ny)
                    a.U0[p * a.pp.plane + (size_t)(y + a.pp.oy) * a.pp.px + x + a.pp.ox] =
                        Gi[(r + R) * G::GIW + c + R];
            }
    }

    // pass-1 task: H row hr, 8 adjacent columns from 8 g
    const int g8 = 8 * ((warp & 1) * 4 + (lane & 3));
    const int hr = (warp >> 1) * 8 + (lane >> 2);
    // pass-2 task: output column c2, output rows r2 .. r2 + RPT - 1
    const int c2 = (warp & 1) * 32 + lane;
    const int r2 = (warp >> 1) * G::RPT;
    const int x2 = X0 + c2;
    const bool xin = x2 < nx;

    // (1) horizontal patch sums of shift (sx, sy) into buffer b:
    //     H(hr, c) = sum_{t=0..2R} d2(c + t - R, hr - R),  d2 = (g_p(x) - g_q(x + s))^2
    auto horizontal = [&](int sx, int sy, float* Hb) {
        if (hr >= G::HR) return;
        float d2[4 * G::NQ4];
        const float* pi = Gi + hr * G::GIW + g8;
        const float* pj = Gj + (hr + sy + rho) * L.GJW + g8 + sx + rho;
#pragma unroll
        for (int t = 0; t < G::NQ4; ++t) {
            const float4 v = *(const float4*)(pi + 4 * t);
            const float vi[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (4 * t + u < G::NQ) {
                    const float d = vi[u] - pj[4 * t + u];
                    d2[4 * t + u] = d * d;
                }
            }
        }
        float h[8];
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
            float m = 0.f;
#pragma unroll
            for (int t = 1; t <= 2 * R; ++t) m = (t == 1) ? d2[c + 1] : m + d2[c + t];
            h[c] = (R == 0) ? d2[c] : d2[c] + m;
            h[c + 1] = (R == 0) ? d2[c + 1] : m + d2[c + 2 * R + 1];
        }
        float* o = Hb + hr * G::HP + g8;
        *(float4*)o = make_float4(h[0], h[1], h[2], h[3]);
        *(float4*)(o + 4) = make_float4(h[4], h[5], h[6], h[7]);
    };

    float mf[G::RPT];
#pragma unroll
    for (int r = 0; r < G::RPT; ++r) mf[r] = INFINITY;
    const size_t plane = a.pp.plane;
    const bool store = a.D != nullptr;            // NULL: row minima (and u^(0)) only
    float* Dbase = store ? a.D + (size_t)p * W * W * plane + (size_t)(Y0 + r2 + a.pp.oy) * a.pp.px + x2 + a.pp.ox
                         : nullptr;

    // (2) vertical sums of the shift with index k = (sy + rho) W + sx + rho
    //     from buffer Hk, the stores and both minima
    auto vertical = [&](int k, int sx, int sy, const float* Hk) {
        // D(c2, r) = sum_{t=0..2R} H(r + t, c2)
        {
            const float* Hb = Hk + r2 * G::HP + c2;
            float hv[G::RPT + 2 * R];
#pragma unroll
            for (int t = 0; t < G::RPT + 2 * R; ++t) hv[t] = Hb[t * G::HP];
            float dv[G::RPT];
#pragma unroll
            for (int r = 0; r < G::RPT; r += 2) {
                float m = 0.f;
#pragma unroll
                for (int t = 1; t <= 2 * R; ++t) m = (t == 1) ? hv[r + 1] : m + hv[r + t];
                dv[r] = (R == 0) ? hv[r] : hv[r] + m;
                if (r + 1 < G::RPT) dv[r + 1] = (R == 0) ? hv[r + 1] : m + hv[r + 2 * R + 1];
            }
            // (3) store the forward distance (+inf where x + s leaves the image),
            //     track the forward row minimum and the backward minimum at x + s
            const bool colok = xin && (unsigned)(x2 + sx) < (unsigned)nx;
            float* Dk = store ? Dbase + (size_t)k * plane : nullptr;
            float* bm = BM + (r2 + sy + rho) * G::BMW + c2 + sx + rho;
            const int y0 = Y0 + r2;
            if (y0 + G::RPT <= ny && y0 + sy >= 0 && y0 + G::RPT - 1 + sy < ny) {
                // every row of this warp and its shifted row lie in the image
#pragma unroll
                for (int r = 0; r < G::RPT; ++r) {
                    const float val = colok ? dv[r] : INFINITY;
                    if (xin && store) Dk[(size_t)r * a.pp.px] = val;
                    mf[r] = fminf(mf[r], val);
                    bm[r * G::BMW] = fminf(bm[r * G::BMW], val);
                }
            } else {
#pragma unroll
                for (int r = 0; r < G::RPT; ++r) {
                    const int y = y0 + r;
                    const bool yin = y < ny;
                    const bool vf = colok && yin && (unsigned)(y + sy) < (unsigned)ny;
                    const float val = vf ? dv[r] : INFINITY;
                    if (xin && yin && store) Dk[(size_t)r * a.pp.px] = val;
                    mf[r] = fminf(mf[r], val);
                    bm[r * G::BMW] = fminf(bm[r * G::BMW], val);
                }
            }
        }
    };

    const int W2 = W * W;
    if constexpr (SLIDE) {
        // g_p segment of the pass-1 task, for every shift
        const bool hact = hr < G::HR;
        float gi[4 * G::NQ4];
#pragma unroll
        for (int t = 0; t < G::NQ4; ++t) {
            const float4 v = hact ? *(const float4*)(Gi + hr * G::GIW + g8 + 4 * t)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            gi[4 * t] = v.x; gi[4 * t + 1] = v.y; gi[4 * t + 2] = v.z; gi[4 * t + 3] = v.w;
        }
        float gw[G::NQ];   // g_q(row, g8 + sx + rho + t) in slot (sx + rho + t) % NQ
        int k = 0;
        for (int sy = -rho; sy <= rho; ++sy) {
            const float* prow = Gj + (hr + sy + rho) * L.GJW + g8;
#pragma unroll
            for (int j = 0; j < 15; ++j) {   // 15 = the largest window of this path
                if (j >= W) break;
                if (hact) {
                    if (j == 0) {
#pragma unroll
                        for (int t = 0; t < G::NQ - 1; ++t) gw[t] = prow[t];
                    }
                    gw[(j + G::NQ - 1) % G::NQ] = prow[j + G::NQ - 1];
                    float d2[G::NQ];
#pragma unroll
                    for (int t = 0; t < G::NQ; ++t) {
                        const float d = gi[t] - gw[(j + t) % G::NQ];
                        d2[t] = d * d;
                    }
                    float h[8];
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        float m = 0.f;
#pragma unroll
                        for (int t = 1; t <= 2 * R; ++t) m = (t == 1) ? d2[c + 1] : m + d2[c + t];
                        h[c] = (R == 0) ? d2[c] : d2[c] + m;
                        h[c + 1] = (R == 0) ? d2[c + 1] : m + d2[c + 2 * R + 1];
                    }
                    float* o = H + (k & 1) * 32 * G::HP + hr * G::HP + g8;
                    *(float4*)o = make_float4(h[0], h[1], h[2], h[3]);
                    *(float4*)(o + 4) = make_float4(h[4], h[5], h[6], h[7]);
                }
                if (k > 0) {
                    // the previous shift: (j - 1, sy), or the end of the previous row
                    const int psx = j > 0 ? j - 1 - rho : rho;
                    const int psy = j > 0 ? sy : sy - 1;
                    vertical(k - 1, psx, psy, H + ((k - 1) & 1) * 32 * G::HP);
                }
                __syncthreads();
                ++k;
            }
        }
        vertical(W2 - 1, rho, rho, H + ((W2 - 1) & 1) * 32 * G::HP);
        __syncthreads();
    } else {
        horizontal(-rho, -rho, H);
        __syncthreads();
        int sx = -rho, sy = -rho;
        for (int k = 0; k < W2; ++k) {
            if (k + 1 < W2) {
                const int nx1 = (sx == rho) ? -rho : sx + 1;
                const int ny1 = (sx == rho) ? sy + 1 : sy;
                horizontal(nx1, ny1, H + ((k + 1) & 1) * 32 * G::HP);
            }
            vertical(k, sx, sy, H + (k & 1) * 32 * G::HP);
            __syncthreads();
            if (sx == rho) { sx = -rho; ++sy; } else { ++sx; }
        }
    }
    // forward minima: owned by this thread
#pragma unroll
    for (int r = 0; r < G::RPT; ++r) {
        const int y = Y0 + r2 + r;
        if (xin && y < ny) {
            a.mins[p * npx + (size_t)y * nx + x2] = mf[r];
            if (!(mf[r] < INFINITY)) atomicOr(a.err, 4);
        }
    }
    // backward minima of phase q toward p: a pixel receives from every block
    // whose tile lies within rho of it; combine with an integer atomic min
    // (the order of non-negative floats is that of their bit patterns)
    int* mprev = (int*)(a.mins + (size_t)(a.N + q) * npx);
    for (int r = warp; r < L.BMH; r += 8)
        for (int c = lane; c < G::TX + 2 * rho; c += 32) {
            const int x = X0 - rho + c, y = Y0 - rho + r;
            const float v = BM[r * G::BMW + c];
            if (x >= 0 && x < nx && y >= 0 && y < ny && v < INFINITY)
                atomicMin(mprev + (size_t)y * nx + x, __float_as_int(v));
        }
}

template <int R>
static size_t weights_smem(int rho) { return sizeof(float) * WGeo<R>(rho).floats(); }

// Shapes of the sliding-window pass 1: patch <= 7, window <= 15.
constexpr int kSlideMaxR = 3;
constexpr int kSlideMaxRho = 7;

static cudaError_t prepare_gj_tma(int* slots);

// Opt every weight-kernel variant into the largest dynamic shared memory any
// window can need (called at geometry creation, outside any stream capture).
cudaError_t prepare_weights(int* gj_slots) {
    cudaError_t e = cudaSuccess;
#define TNLM_PREP_W(R, SLIDE, RHO)                                                      \
    if (e == cudaSuccess)                                                               \
        e = cudaFuncSetAttribute(k_weights<R, SLIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)weights_smem<R>(RHO));
    TNLM_PREP_W(0, false, (kMaxWindow - 1) / 2) TNLM_PREP_W(1, false, (kMaxWindow - 1) / 2)
    TNLM_PREP_W(2, false, (kMaxWindow - 1) / 2) TNLM_PREP_W(3, false, (kMaxWindow - 1) / 2)
    TNLM_PREP_W(4, false, (kMaxWindow - 1) / 2) TNLM_PREP_W(5, false, (kMaxWindow - 1) / 2)
    TNLM_PREP_W(6, false, (kMaxWindow - 1) / 2) TNLM_PREP_W(7, false, (kMaxWindow - 1) / 2)
    TNLM_PREP_W(0, true, kSlideMaxRho) TNLM_PREP_W(1, true, kSlideMaxRho)
    TNLM_PREP_W(2, true, kSlideMaxRho) TNLM_PREP_W(3, true, kSlideMaxRho)
#undef TNLM_PREP_W
    return e == cudaSuccess ? prepare_gj_tma(gj_slots) : e;
}

template <int R>
static cudaError_t launch_weights_r(const WArgs& a, cudaStream_t st) {
    using G = WGeo<R>;
    const size_t smem = weights_smem<R>(a.rho);
    dim3 grid((a.nx + G::TX - 1) / G::TX, (a.ny + G::TY - 1) / G::TY, a.N);
    if constexpr (R <= kSlideMaxR) {
        if (a.rho <= kSlideMaxRho) {
            k_weights<R, true><<<grid, 256, smem, st>>>(a);
            return cudaGetLastError();
        }
    }
    k_weights<R, false><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_weights(const tnlm_geometry* g, const Workspace& ws, int patch, int window,
                           const float* gimg, cudaStream_t st, bool store) {
    WArgs a;
    a.g = gimg; a.D = store ? ws.D : nullptr; a.mins = ws.mins; a.U0 = ws.U0; a.err = ws.st.err; a.pp = ws.pp;
    a.nx = g->nx; a.ny = g->ny; a.N = g->N; a.rho = (window - 1) / 2; a.W = window;
    // backward minima start above every distance (0x7f7f7f7f = 3.4e38)
    const size_t npx = (size_t)g->nx * g->ny;
    cudaError_t e = cudaMemsetAsync(ws.mins + (size_t)g->N * npx, 0x7f, sizeof(float) * g->N * npx, st);
    if (e != cudaSuccess) return e;
    switch ((patch - 1) / 2) {
        case 0: return launch_weights_r<0>(a, st);
        case 1: return launch_weights_r<1>(a, st);
        case 2: return launch_weights_r<2>(a, st);
        case 3: return launch_weights_r<3>(a, st);
        case 4: return launch_weights_r<4>(a, st);
        case 5: return launch_weights_r<5>(a, st);
        case 6: return launch_weights_r<6>(a, st);
        case 7: return launch_weights_r<7>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// K5
// ---------------------------------------------------------------------------
// Partial slots per block of the last sweep: squared change, squared norm,
// clamped pixels.
constexpr int kPart = 3;

struct GjArgs {
    const float* D;
    const float* mins;
    const float* g;
    const float* uin;
    float* uout;
    float* fout;
    float* zn;
    double* part;
    int* err;
    PadPlane pp;
    int nx, ny, N, rho, W, clamp;
    float k2, c1, c2;
};

// MODE 0: intermediate sweep (uout, padded); 1: last sweep, clamp, write f and
// the relative-change partials; 2: write the normalisers Z (public weights).
template <int MODE>
__global__ void __launch_bounds__(kGjTileX * kGjTileY) k_gj(GjArgs a) {
    const int N = a.N, nx = a.nx, ny = a.ny;
    const int tile = blockIdx.x / N, i = blockIdx.x % N;
    const int tilesx = (nx + kGjTileX - 1) / kGjTileX;
    const int tid = threadIdx.x;
    const int x = (tile % tilesx) * kGjTileX + (tid & 31);
    const int y = (tile / tilesx) * kGjTileY + (tid >> 5);
    const bool in = x < nx && y < ny;
    const size_t npx = (size_t)nx * ny;
    const int ip = (i + N - 1) % N, inx = (i + 1) % N;
    float af = 0.f, zf = 0.f, ab = 0.f, zb = 0.f;
    const size_t pix = (size_t)y * nx + x;
    if (in) {
        const int rho = a.rho, W = a.W, px = a.pp.px;
        const size_t plane = a.pp.plane, W2 = (size_t)W * W;
        const float k2 = a.k2;
        const float mfk = a.mins[i * npx + pix] * k2;
        const float mbk = a.mins[(N + i) * npx + pix] * k2;
        const size_t cpos = (size_t)(y + a.pp.oy) * px + x + a.pp.ox;
        const float* dn = a.D + (size_t)i * W2 * plane + cpos;
        const float* dp = a.D + (size_t)ip * W2 * plane + cpos + (size_t)rho * px + rho;
        const float* un = a.uin + inx * plane + cpos - (size_t)rho * px - rho;
        const float* up = a.uin + ip * plane + cpos + (size_t)rho * px + rho;
        for (int sy = 0; sy < W; ++sy) {
            const float* dnr = dn + (size_t)sy * W * plane;
            const float* dpr = dp + (size_t)sy * W * plane - (size_t)sy * px;
            const float* unr = un + (size_t)sy * px;
            const float* upr = up - (size_t)sy * px;
#pragma unroll 4
            for (int sx = 0; sx < W; ++sx) {
                const float Df = __ldg(dnr + (size_t)sx * plane);
                const float Db = __ldg(dpr + (size_t)sx * plane - sx);
                const float ef = ex2_approx(fmaf(-Df, k2, mfk));
                const float eb = ex2_approx(fmaf(-Db, k2, mbk));
                if (MODE != 2) {
                    af = fmaf(ef, __ldg(unr + sx), af);
                    ab = fmaf(eb, __ldg(upr - sx), ab);
                }
                zf += ef;
                zb += eb;
            }
        }
        // the row minimum contributes 2^(rounding error of m*k2) ~ 1, so a
        // normaliser below 1/2 (or NaN) means a non-finite distance or image
        if (!(zf >= 0.5f) || !(zb >= 0.5f)) atomicOr(a.err, 8);
    }
    if (MODE == 2) {
        if (in) {
            a.zn[i * npx + pix] = zf;
            a.zn[(N + i) * npx + pix] = zb;
        }
        return;
    }
    const float unew = in ? fmaf(a.g[i * npx + pix], a.c1, a.c2 * (af / zf + ab / zb)) : 0.f;
    if (MODE == 0) {
        if (in) a.uout[i * a.pp.plane + (size_t)(y + a.pp.oy) * a.pp.px + x + a.pp.ox] = unew;
        return;
    }
    float fnew = 0.f, dif = 0.f, ncl = 0.f;
    if (in) {
        fnew = a.clamp ? fmaxf(unew, 0.f) : unew;
        ncl = (a.clamp && unew < 0.f) ? 1.f : 0.f;
        const float fold = a.fout[i * npx + pix];
        a.fout[i * npx + pix] = fnew;
        dif = fnew - fold;
    }
    __shared__ double sh[kGjTileX * kGjTileY / 32];
    const double d2 = block_sum<kGjTileX * kGjTileY>(dif * dif, sh, tid);
    const double n2 = block_sum<kGjTileX * kGjTileY>(fnew * fnew, sh, tid);
    const double c2 = block_sum<kGjTileX * kGjTileY>(ncl, sh, tid);
    if (tid == 0) {
        a.part[kPart * (size_t)blockIdx.x] = d2;
        a.part[kPart * (size_t)blockIdx.x + 1] = n2;
        a.part[kPart * (size_t)blockIdx.x + 2] = c2;
    }
}

// Vectorised sweep for W in {3, 5, ..., 15}: a thread owns 4 consecutive
// pixels of one row.  Per window row it loads the neighbour-phase values it
// needs as aligned float4 windows into registers; per shift it loads the
// forward distances as one float4 and the backward ones from an aligned
// 8-float window at a compile-time offset.  Requires the padded layout with
// ox >= align4(rho) + 4 and px a multiple of 4 (see the workspace layout).
constexpr int kGjvPx = 4;              // pixels per thread
constexpr int kGjvTx = 16, kGjvTy = 16;  // threads per block in x (64 px) and y

template <int W, int MODE>
__global__ void __launch_bounds__(kGjvTx * kGjvTy) k_gj_vec(GjArgs a) {
    constexpr int RHO = (W - 1) / 2;
    constexpr int UOFF = 4 * ((RHO + 3) / 4);
    constexpr int UW = 4 + 2 * UOFF;
    const int N = a.N, nx = a.nx, ny = a.ny;
    const int tile = blockIdx.x / N, i = blockIdx.x % N;
    const int tilesx = (nx + kGjvTx * kGjvPx - 1) / (kGjvTx * kGjvPx);
    const int tid = threadIdx.x;
    const int x0 = (tile % tilesx) * (kGjvTx * kGjvPx) + kGjvPx * (tid % kGjvTx);
    const int y = (tile / tilesx) * kGjvTy + tid / kGjvTx;
    const bool rowin = x0 < nx && y < ny;
    const size_t npx = (size_t)nx * ny;
    const int ip = (i + N - 1) % N, inx = (i + 1) % N;
    const int px = a.pp.px;
    const int plane = (int)a.pp.plane;
    float af[4] = {0.f, 0.f, 0.f, 0.f}, zf[4] = {0.f, 0.f, 0.f, 0.f};
    float ab[4] = {0.f, 0.f, 0.f, 0.f}, zb[4] = {0.f, 0.f, 0.f, 0.f};
    const float k2 = a.k2;
    if (rowin) {
        float mfk[4], mbk[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const bool in = x0 + p < nx;
            const size_t pix = (size_t)y * nx + x0 + p;
            mfk[p] = in ? a.mins[i * npx + pix] * k2 : 0.f;
            mbk[p] = in ? a.mins[(N + i) * npx + pix] * k2 : 0.f;
        }
        const int c0 = x0 + a.pp.ox;                    // padded column of pixel x0
        const float* Dn = a.D + (size_t)i * (W * W) * a.pp.plane + (size_t)(y + a.pp.oy) * px + c0;
        const float* Dp = a.D + (size_t)ip * (W * W) * a.pp.plane + (size_t)(y + a.pp.oy) * px + c0;
        const float* Un = a.uin + (size_t)inx * a.pp.plane + (size_t)(y + a.pp.oy) * px + c0 - UOFF;
        const float* Up = a.uin + (size_t)ip * a.pp.plane + (size_t)(y + a.pp.oy) * px + c0 - UOFF;
        for (int sy = 0; sy < W; ++sy) {
            const int dy = sy - RHO;
            float un[UW], up[UW];
#pragma unroll
            for (int q = 0; q < UW / 4; ++q) {
                const float4 vn = __ldg((const float4*)(Un + dy * px) + q);
                const float4 vp = __ldg((const float4*)(Up - dy * px) + q);
                un[4 * q] = vn.x; un[4 * q + 1] = vn.y; un[4 * q + 2] = vn.z; un[4 * q + 3] = vn.w;
                up[4 * q] = vp.x; up[4 * q + 1] = vp.y; up[4 * q + 2] = vp.z; up[4 * q + 3] = vp.w;
            }
#pragma unroll
            for (int sx = 0; sx < W; ++sx) {
                const int dx = sx - RHO;
                const int k = sy * W + sx;
                const float4 f4 = __ldg((const float4*)(Dn + k * plane));
                const float df[4] = {f4.x, f4.y, f4.z, f4.w};
                // backward distances at columns x0 - dx .. x0 - dx + 3, row y - dy
                const int off = -dx;
                const int base = off >= 0 ? (off / 4) * 4 : -(((-off) + 3) / 4) * 4;
                const int sh = off - base;
                const float* pb = Dp + k * plane - dy * px + base;
                const float4 b0 = __ldg((const float4*)pb);
                float w8[8] = {b0.x, b0.y, b0.z, b0.w, 0.f, 0.f, 0.f, 0.f};
                if (sh != 0) {
                    const float4 b1 = __ldg((const float4*)pb + 1);
                    w8[4] = b1.x; w8[5] = b1.y; w8[6] = b1.z; w8[7] = b1.w;
                }
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float ef = ex2_approx(fmaf(-df[p], k2, mfk[p]));
                    const float eb = ex2_approx(fmaf(-w8[sh + p], k2, mbk[p]));
                    if (MODE != 2) {
                        af[p] = fmaf(ef, un[UOFF + p + dx], af[p]);
                        ab[p] = fmaf(eb, up[UOFF + p - dx], ab[p]);
                    }
                    zf[p] += ef;
                    zb[p] += eb;
                }
            }
        }
    }
    float dsq = 0.f, nsq = 0.f, ncl = 0.f;
    bool bad = false;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int x = x0 + p;
        if (!rowin || x >= nx) continue;
        bad |= !(zf[p] >= 0.5f) || !(zb[p] >= 0.5f);
        const size_t pix = (size_t)y * nx + x;
        if (MODE == 2) {
            a.zn[i * npx + pix] = zf[p];
            a.zn[(N + i) * npx + pix] = zb[p];
            continue;
        }
        const float unew = fmaf(a.g[i * npx + pix], a.c1, a.c2 * (af[p] / zf[p] + ab[p] / zb[p]));
        if (MODE == 0) {
            a.uout[i * a.pp.plane + (size_t)(y + a.pp.oy) * px + x + a.pp.ox] = unew;
        } else {
            const float fnew = a.clamp ? fmaxf(unew, 0.f) : unew;
            if (a.clamp && unew < 0.f) ncl += 1.f;
            const float fold = a.fout[i * npx + pix];
            a.fout[i * npx + pix] = fnew;
            dsq = fmaf(fnew - fold, fnew - fold, dsq);
            nsq = fmaf(fnew, fnew, nsq);
        }
    }
    if (bad) atomicOr(a.err, 8);
    if (MODE == 1) {
        __shared__ double sh[kGjvTx * kGjvTy / 32];
        const double d2 = block_sum<kGjvTx * kGjvTy>(dsq, sh, tid);
        const double n2 = block_sum<kGjvTx * kGjvTy>(nsq, sh, tid);
        const double c2 = block_sum<kGjvTx * kGjvTy>(ncl, sh, tid);
        if (tid == 0) {
            a.part[kPart * (size_t)blockIdx.x] = d2;
            a.part[kPart * (size_t)blockIdx.x + 1] = n2;
            a.part[kPart * (size_t)blockIdx.x + 2] = c2;
        }
    }
}

// ---------------------------------------------------------------------------
// TMA-pipelined sweep (W in {3, 5, ..., 15}).  A block owns a 64 x 16 pixel
// tile of one phase: 8 consumer warps (a thread owns 4 consecutive pixels of
// one row) and one producer warp.  For every window shift the producer
// loads two boxes of the distance planes with tensor-map copies
// (cp.async.bulk.tensor): the 64 x 16 forward box of pair i at the tile and
// the 68 x 16 backward box of pair i-1 at the tile shifted by -s (x rounded
// down to a 16-byte boundary), into a ring of stages.  Each stage has a
// "full" mbarrier (expected bytes) and an "empty" one (one arrival per
// consumer warp); every wait is bounded and a timeout ends the block with an
// error flag after draining its copies.
//
// Work units.  With split = 2 a (tile, phase) is two units, each taking half
// of the window rows (rows [0, (W+1)/2) and the rest), so that the number of
// units fills the resident CTA slots in whole waves where (tile, phase)
// alone would leave a partial last wave.  Each half stores its four partial
// sums per pixel in a scratch slot; the half that arrives second (a counter
// per tile, no waiting) adds the other's sums to its own -- one FP32
// addition, which is commutative, so the result does not depend on the
// arrival order -- and finishes the pixels.  The relative-change partials
// are written per (tile, phase), so they do not depend on split or on the
// tiles per CTA either.
// ---------------------------------------------------------------------------
// Tile width 64 (64 x 16 tiles) or 128 (128 x 8, rows of 512 contiguous
// bytes per box): measured at 512^2, W = 15, 0.554 against 0.549 ms per
// sweep, 0.1016 against 0.1018 ms at 256^2 -- within noise, so the box
// rows' DRAM locality is not what limits the sweep; 64 is kept.
#ifndef TNLM_GJ_TW
#define TNLM_GJ_TW 64
#endif
constexpr int kTmaTW = TNLM_GJ_TW, kTmaTH = 1024 / kTmaTW;   // 1024 pixels, 4 per consumer thread
static_assert(kTmaTW == 64 || kTmaTW == 128, "sweep tile width");
constexpr int kTmaBW = kTmaTW + 4;
constexpr int kTmaConsumers = 256;
constexpr int kTmaThreads = kTmaConsumers + 32;
constexpr int kTmaStageFloats = kTmaTH * (kTmaTW + kTmaBW);   // 2112 floats = 66 x 128 B
#ifndef TNLM_GJ_STAGES
#define TNLM_GJ_STAGES 6
#endif
constexpr int kTmaStages = TNLM_GJ_STAGES;
constexpr int kTmaUBufs = 1;      // neighbour-iterate tile buffers (2 lets a multi-tile CTA load the next tile early)
// neighbour-phase tile: the 64 x 16 pixels widened by 8 columns and 7 rows
// on each side (every window up to 15 x 15), loaded once per block
constexpr int kTmaUW = kTmaTW + 16, kTmaUH = kTmaTH + 14;
constexpr int kTmaUFloats = kTmaUW * kTmaUH;    // 2400 floats = 75 x 128 B

struct TmaMaps {
    CUtensorMap F, B, U;     // forward / backward distance boxes, iterate tile box
};

__device__ __forceinline__ float f4get(const float4& v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Barrier 1 of the consumer warps only (the producer warp never joins it).
// Every consumer thread reaches each of these barriers the same number of
// times: a wait that timed out does not leave the unit loop on its own, the
// consumers leave it together after consumer_sync_or agrees to stop.
__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kTmaConsumers) : "memory");
}
__device__ __forceinline__ bool consumer_sync_or(bool v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v), "n"(kTmaConsumers)
        : "memory");
    return r != 0;
}

template <int W, int MODE>
__global__ void __launch_bounds__(kTmaThreads, 3) k_gj_tma(GjArgs a, const __grid_constant__ CUtensorMap tmF,
                                                        const __grid_constant__ CUtensorMap tmB,
                                                        const __grid_constant__ CUtensorMap tmU,
                                                        int tpb, int split, float4* __restrict__ hsum,
                                                        int* __restrict__ hcnt, long wlim) {
    constexpr int RHO = (W - 1) / 2;
    constexpr int UOFF = 4 * ((RHO + 3) / 4);
    constexpr int NCH = (2 * UOFF + 4) / 4;     // float4 chunks of a window row
    constexpr int NK = W * W;
    extern __shared__ __align__(128) float tma_sm_raw[];
    // tensor-copy destinations must be 128-byte aligned: round the base up
    float* stages = (float*)(((uintptr_t)tma_sm_raw + 127) & ~(uintptr_t)127);
    float* utile = stages + kTmaStages * kTmaStageFloats;     // [2 buffers][2 phases][UH][UW]
    uint64_t* full = (uint64_t*)(utile + 2 * kTmaUBufs * kTmaUFloats);
    uint64_t* empty = full + kTmaStages;
    uint64_t* ufull = empty + kTmaStages;                      // [2]
    uint64_t* uempty = ufull + 2;                              // [2]
    __shared__ int s_abort, s_issued, s_uissued, s_second;
    __shared__ double wsum[3][kTmaConsumers / 32];
    const int N = a.N, nx = a.nx, ny = a.ny;
    const int tilesx = (nx + kTmaTW - 1) / kTmaTW;
    const int nunits = tilesx * ((ny + kTmaTH - 1) / kTmaTH) * N * split;
    // units blockIdx.x, + gridDim.x, ...: the units in flight at any moment
    // stay a contiguous run of the tile-major, phase-minor order, so the
    // second read of each distance plane is served by L2
    const int t0 = blockIdx.x, tstep = gridDim.x, t1 = min(nunits, t0 + tpb * tstep);
    constexpr int RMID = (W + 1) / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int px = a.pp.px;
    const size_t plane = a.pp.plane;
    if (tid == 0) {
        for (int st = 0; st < kTmaStages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], kTmaConsumers / 32);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ufull[b], 1);
            mbar_init(&uempty[b], kTmaConsumers / 32);
        }
        s_abort = 0;
        s_issued = 0;
        s_uissued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kTmaConsumers / 32) {
        if (lane == 0) {   // producer: runs ahead across the block's tiles
            int kk = 0, nu = 0;
            bool ok = true;
            for (int q = t0, u = 0; q < t1 && ok; q += tstep, ++u) {
                const int ub = u % kTmaUBufs;
                const int t = q / split, half = q - t * split;
                const int k0 = half ? RMID * W : 0, k1 = (split == 1 || half) ? NK : RMID * W;
                const int tile = t / N, i = t % N;
                const int X0 = (tile % tilesx) * kTmaTW, Y0 = (tile / tilesx) * kTmaTH;
                const int ip = (i + N - 1) % N, inx = (i + 1) % N;
                // iterate tiles of both neighbour phases (rows/columns outside the plane read 0)
                if (u >= kTmaUBufs &&
                    !mbar_wait_bounded(&uempty[ub], (unsigned)(((u - kTmaUBufs) / kTmaUBufs) & 1), wlim)) {
                    ok = false;
                    break;
                }
                float* ut = utile + ub * 2 * kTmaUFloats;
                mbar_arrive_expect_tx(&ufull[ub], 8u * kTmaUFloats);
                tma_load_3d(ut, &tmU, X0 + a.pp.ox - 8, Y0 + a.pp.oy - 7, inx, &ufull[ub]);
                tma_load_3d(ut + kTmaUFloats, &tmU, X0 + a.pp.ox - 8, Y0 + a.pp.oy - 7, ip, &ufull[ub]);
                nu = u + 1;
                for (int k = k0; k < k1; ++k) {
                    const int slot = kk % kTmaStages;
                    if (kk >= kTmaStages &&
                        !mbar_wait_bounded(&empty[slot], (unsigned)((kk / kTmaStages - 1) & 1), wlim)) {
                        ok = false;
                        break;
                    }
                    if (*(volatile int*)&s_abort) {
                        ok = false;
                        break;
                    }
                    const int dy = k / W - RHO, dx = k % W - RHO;
                    const int off = -dx;
                    const int base = off >= 0 ? (off / 4) * 4 : -(((-off) + 3) / 4) * 4;
                    float* stg = stages + slot * kTmaStageFloats;
                    mbar_arrive_expect_tx(&full[slot], 4u * kTmaStageFloats);
                    tma_load_3d(stg, &tmF, X0 + a.pp.ox, Y0 + a.pp.oy, i * NK + k, &full[slot]);
                    tma_load_3d(stg + kTmaTH * kTmaTW, &tmB, X0 + a.pp.ox + base, Y0 + a.pp.oy - dy,
                                ip * NK + k, &full[slot]);
                    ++kk;
                }
            }
            if (!ok) s_abort = 1;
            s_issued = kk;
            s_uissued = nu;
        }
    } else {
        const int tx = tid % (kTmaTW / 4), ty = tid / (kTmaTW / 4);
        const size_t npx = (size_t)nx * ny;
        const float k2 = a.k2;
        bool bad = false, ok = true;
        int kk = 0;
        for (int q = t0, u = 0; q < t1 && ok; q += tstep, ++u) {
            const int ub = u % kTmaUBufs;
            const int t = q / split, half = q - t * split;
            const int r0 = half ? RMID : 0, r1 = (split == 1 || half) ? W : RMID;
            const int tile = t / N, i = t % N;
            const int x0 = (tile % tilesx) * kTmaTW + 4 * tx, y = (tile / tilesx) * kTmaTH + ty;
            const bool rowin = x0 < nx && y < ny;
            float af[4] = {0.f, 0.f, 0.f, 0.f}, zf[4] = {0.f, 0.f, 0.f, 0.f};
            float ab[4] = {0.f, 0.f, 0.f, 0.f}, zb[4] = {0.f, 0.f, 0.f, 0.f};
            float mfk[4], mbk[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const bool in = rowin && x0 + p < nx;
                const size_t pix = (size_t)y * nx + x0 + p;
                mfk[p] = in ? a.mins[i * npx + pix] * k2 : 0.f;
                mbk[p] = in ? a.mins[(N + i) * npx + pix] * k2 : 0.f;
            }
            // window rows of this thread inside the neighbour tiles
            const float* Un = utile + ub * 2 * kTmaUFloats + (ty + 7) * kTmaUW + 4 * tx + 8 - UOFF;
            const float* Up = Un + kTmaUFloats;
            const bool uok = mbar_wait_bounded(&ufull[ub], (unsigned)((u / kTmaUBufs) & 1), wlim);
            if (!uok) {
                s_abort = 1;
                ok = false;     // skips the window loop; the unit ends at the vote below
            }
            for (int sy = r0; sy < r1 && ok; ++sy) {
                const int dy = sy - RHO;
                // window rows as float4 chunks, loaded when the sliding window
                // first reaches them (forward slides right, backward left), so
                // only two or three chunks of each are live at a time
                const float4* rn = (const float4*)(Un + dy * kTmaUW);
                const float4* rp = (const float4*)(Up - dy * kTmaUW);
                float4 cn[NCH], cp[NCH];
#pragma unroll
                for (int sx = 0; sx < W; ++sx, ++kk) {
                    const int dx = sx - RHO;
                    const int slot = kk % kTmaStages;
                    if (!mbar_wait_bounded(&full[slot], (unsigned)((kk / kTmaStages) & 1), wlim)) {
                        s_abort = 1;
                        ok = false;
                        break;
                    }
                    {
                        const int flo = (UOFF + dx) >> 2, fhi = (UOFF + dx + 3) >> 2;
                        const int blo = (UOFF - dx) >> 2, bhi = (UOFF - dx + 3) >> 2;
                        const int pfhi = (UOFF + dx + 2) >> 2, pblo = (UOFF - dx + 1) >> 2;
#pragma unroll
                        for (int j = 0; j < NCH; ++j) {
                            if ((sx == 0 && j >= flo && j <= fhi) || (sx > 0 && j == fhi && fhi != pfhi))
                                cn[j] = rn[j];
                            if ((sx == 0 && j >= blo && j <= bhi) || (sx > 0 && j == blo && blo != pblo))
                                cp[j] = rp[j];
                        }
                    }
                    const float* stg = stages + slot * kTmaStageFloats;
                    const float4 f4 = *(const float4*)(stg + ty * kTmaTW + 4 * tx);
                    const int off = -dx;
                    const int base = off >= 0 ? (off / 4) * 4 : -(((-off) + 3) / 4) * 4;
                    const int sh = off - base;
                    const float* pb = stg + kTmaTH * kTmaTW + ty * kTmaBW + 4 * tx;
                    const float4 b0 = *(const float4*)pb;
                    const float4 b1 = *(const float4*)(pb + 4);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[slot]);   // this warp is done with the stage
                    const float df[4] = {f4.x, f4.y, f4.z, f4.w};
                    const float w8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const float ef = ex2_approx(fmaf(-df[p], k2, mfk[p]));
                        const float eb = ex2_approx(fmaf(-w8[sh + p], k2, mbk[p]));
                        af[p] = fmaf(ef, f4get(cn[(UOFF + p + dx) >> 2], (UOFF + p + dx) & 3), af[p]);
                        ab[p] = fmaf(eb, f4get(cp[(UOFF + p - dx) >> 2], (UOFF + p - dx) & 3), ab[p]);
                        zf[p] += ef;
                        zb[p] += eb;
                    }
                }
            }
            __syncwarp();
            // this warp is done with the tile's windows (a buffer whose load
            // was never seen complete is not handed back to the producer)
            if (lane == 0 && uok) mbar_arrive(&uempty[ub]);
            if (consumer_sync_or(!ok || *(volatile int*)&s_abort)) break;   // all consumers stop together
            if (split > 1) {
                float4* mine = hsum + ((size_t)t * 2 + half) * 4 * kTmaConsumers + tid;
                mine[0] = make_float4(af[0], af[1], af[2], af[3]);
                mine[kTmaConsumers] = make_float4(zf[0], zf[1], zf[2], zf[3]);
                mine[2 * kTmaConsumers] = make_float4(ab[0], ab[1], ab[2], ab[3]);
                mine[3 * kTmaConsumers] = make_float4(zb[0], zb[1], zb[2], zb[3]);
                __threadfence();
                consumer_sync();
                if (tid == 0) s_second = atomicAdd(&hcnt[t], 1);
                consumer_sync();
                if (s_second == 0) continue;      // the other half finishes this tile
                __threadfence();
                const float4* oth = hsum + ((size_t)t * 2 + (1 - half)) * 4 * kTmaConsumers + tid;
                const float4 o0 = __ldcg(oth), o1 = __ldcg(oth + kTmaConsumers);
                const float4 o2 = __ldcg(oth + 2 * kTmaConsumers), o3 = __ldcg(oth + 3 * kTmaConsumers);
                af[0] += o0.x; af[1] += o0.y; af[2] += o0.z; af[3] += o0.w;
                zf[0] += o1.x; zf[1] += o1.y; zf[2] += o1.z; zf[3] += o1.w;
                ab[0] += o2.x; ab[1] += o2.y; ab[2] += o2.z; ab[3] += o2.w;
                zb[0] += o3.x; zb[1] += o3.y; zb[2] += o3.z; zb[3] += o3.w;
                if (tid == 0) hcnt[t] = 0;        // ready for the next sweep
            }
            float dsq = 0.f, nsq = 0.f, ncl = 0.f;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int x = x0 + p;
                if (!rowin || x >= nx) continue;
                bad |= !(zf[p] >= 0.5f) || !(zb[p] >= 0.5f);
                const size_t pix = (size_t)y * nx + x;
                const float unew = fmaf(a.g[i * npx + pix], a.c1, a.c2 * (af[p] / zf[p] + ab[p] / zb[p]));
                if (MODE == 0) {
                    a.uout[i * plane + (size_t)(y + a.pp.oy) * px + x + a.pp.ox] = unew;
                } else {
                    const float fnew = a.clamp ? fmaxf(unew, 0.f) : unew;
                    if (a.clamp && unew < 0.f) ncl += 1.f;
                    const float fold = a.fout[i * npx + pix];
                    a.fout[i * npx + pix] = fnew;
                    dsq = fmaf(fnew - fold, fnew - fold, dsq);
                    nsq = fmaf(fnew, fnew, nsq);
                }
            }
            if (MODE == 1) {     // relative-change and clamp-count partials of this (tile, phase)
                const float d = warp_sum(dsq), n = warp_sum(nsq), c = warp_sum(ncl);
                if (lane == 0) {
                    wsum[0][warp] = (double)d;
                    wsum[1][warp] = (double)n;
                    wsum[2][warp] = (double)c;
                }
                consumer_sync();
                if (tid == 0) {
                    double d2 = 0.0, n2 = 0.0, c2 = 0.0;
                    for (int w = 0; w < kTmaConsumers / 32; ++w) {
                        d2 += wsum[0][w];
                        n2 += wsum[1][w];
                        c2 += wsum[2][w];
                    }
                    a.part[kPart * (size_t)t] = d2;
                    a.part[kPart * (size_t)t + 1] = n2;
                    a.part[kPart * (size_t)t + 2] = c2;
                }
                consumer_sync();
            }
        }
        if (bad) atomicOr(a.err, 8);
    }
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            atomicOr(a.err, 16);
            // drain the block's copies in flight: the last use of each iterate
            // buffer and the last kTmaStages stage loads
            for (int u = max(0, s_uissued - kTmaUBufs); u < s_uissued; ++u)
                mbar_wait_bounded(&ufull[u % kTmaUBufs], (unsigned)((u / kTmaUBufs) & 1));
            for (int kk = s_issued - kTmaStages; kk < s_issued; ++kk)
                if (kk >= 0) mbar_wait_bounded(&full[kk % kTmaStages], (unsigned)((kk / kTmaStages) & 1));
        }
        __syncthreads();
        return;
    }
}

static size_t tma_smem() {
    return 128 + sizeof(float) * (kTmaStages * kTmaStageFloats + 2 * kTmaUBufs * kTmaUFloats) +
           8 * (2 * kTmaStages + 4);
}

// Opt the TMA sweeps into their dynamic shared memory and count the CTAs the
// device holds at once (geometry creation).
static cudaError_t prepare_gj_tma(int* slots) {
    const int sm = (int)tma_smem();
    cudaError_t e = cudaSuccess;
#define TNLM_PREP_GJ(W)                                                                     \
    if (e == cudaSuccess)                                                                   \
        e = cudaFuncSetAttribute(k_gj_tma<W, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); \
    if (e == cudaSuccess)                                                                   \
        e = cudaFuncSetAttribute(k_gj_tma<W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    TNLM_PREP_GJ(3) TNLM_PREP_GJ(5) TNLM_PREP_GJ(7) TNLM_PREP_GJ(9) TNLM_PREP_GJ(11)
    TNLM_PREP_GJ(13) TNLM_PREP_GJ(15)
#undef TNLM_PREP_GJ
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_tma<15, 1>, kTmaThreads,
                                                           tma_smem())) != cudaSuccess)
        return e;
    *slots = (sms > 0 && per_sm > 0) ? sms * per_sm : 1;
    return cudaSuccess;
}

long g_gj_wait_limit = kSpinLimit;

// Tiles per CTA of the TMA sweep: one unless the autotuner measured more to
// be faster on this device and shape.
static int gj_tma_tpb(const tnlm_geometry* g) { return g->tune_gj_tpb > 0 ? g->tune_gj_tpb : 1; }
static int gj_tma_tiles(const tnlm_geometry* g) {
    return ((g->nx + kTmaTW - 1) / kTmaTW) * ((g->ny + kTmaTH - 1) / kTmaTH) * g->N;
}
// Halves of the window per (tile, phase): 2 when that fills the device's
// resident CTA slots in whole waves clearly better (fraction of the last
// wave that is busy), e.g. 640 (tile, phase) pairs on 456 slots.
int gj_tma_split(const tnlm_geometry* g) {
    if (g->tune_gj_split > 0) return g->tune_gj_split;
    const double slots = g->cta_slots_gj > 0 ? g->cta_slots_gj : 1;
    auto fill = [&](double units) { return units / (slots * ceil(units / slots)); };
    const double t = gj_tma_tiles(g);
    return fill(2 * t) > fill(t) + 0.1 ? 2 : 1;
}
static int gj_tma_blocks(const tnlm_geometry* g) {
    const int units = gj_tma_tiles(g) * gj_tma_split(g);
    const int tpb = gj_tma_tpb(g);
    return (units + tpb - 1) / tpb;
}
size_t gj_split_floats(const tnlm_geometry* g) {
    return (size_t)gj_tma_tiles(g) * 2 * 4 * kTmaConsumers * 4;
}

template <int MODE>
static bool launch_gj_tma(const tnlm_geometry* g, const GjArgs& a, const Workspace& ws, int window,
                          cudaStream_t st) {
    const size_t sm = tma_smem();
    const CUtensorMap* U = a.uin == ws.U0 ? &ws.tmU0 : (a.uin == ws.U1 ? &ws.tmU1 : nullptr);
    if (!U) return false;
    const int nb = gj_tma_blocks(g), tpb = gj_tma_tpb(g), sp = gj_tma_split(g);
    float4* hs = (float4*)ws.gjsum;
    switch (window) {
        case 3: k_gj_tma<3, MODE><<<nb, kTmaThreads, sm, st>>>(a, ws.tmF, ws.tmB, *U, tpb, sp, hs, ws.gjcnt, g_gj_wait_limit); return true;
        case 5: k_gj_tma<5, MODE><<<nb, kTmaThreads, sm, st>>>(a, ws.tmF, ws.tmB, *U, tpb, sp, hs, ws.gjcnt, g_gj_wait_limit); return true;
        case 7: k_gj_tma<7, MODE><<<nb, kTmaThreads, sm, st>>>(a, ws.tmF, ws.tmB, *U, tpb, sp, hs, ws.gjcnt, g_gj_wait_limit); return true;
        case 9: k_gj_tma<9, MODE><<<nb, kTmaThreads, sm, st>>>(a, ws.tmF, ws.tmB, *U, tpb, sp, hs, ws.gjcnt, g_gj_wait_limit); return true;
        case 11: k_gj_tma<11, MODE><<<nb, kTmaThreads, sm, st>>>(a, ws.tmF, ws.tmB, *U, tpb, sp, hs, ws.gjcnt, g_gj_wait_limit); return true;
        case 13: k_gj_tma<13, MODE><<<nb, kTmaThreads, sm, st>>>(a, ws.tmF, ws.tmB, *U, tpb, sp, hs, ws.gjcnt, g_gj_wait_limit); return true;
        case 15: k_gj_tma<15, MODE><<<nb, kTmaThreads, sm, st>>>(a, ws.tmF, ws.tmB, *U, tpb, sp, hs, ws.gjcnt, g_gj_wait_limit); return true;
        default: return false;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_distance_maps(Workspace& ws, int N) {
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    if (!fn || !ws.D || !ws.U0 || !ws.U1) return false;
    const int W2 = (2 * ws.rho + 1) * (2 * ws.rho + 1);
    const cuuint64_t dims[3] = {(cuuint64_t)ws.pp.px, (cuuint64_t)ws.pp.py, (cuuint64_t)N * W2};
    const cuuint64_t strides[2] = {(cuuint64_t)ws.pp.px * 4, (cuuint64_t)ws.pp.plane * 4};
    const cuuint32_t boxF[3] = {kTmaTW, kTmaTH, 1}, boxB[3] = {kTmaBW, kTmaTH, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    if (fn(&ws.tmF, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ws.D, dims, strides, boxF, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (fn(&ws.tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ws.D, dims, strides, boxB, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t udims[3] = {(cuuint64_t)ws.pp.px, (cuuint64_t)ws.pp.py, (cuuint64_t)N};
    const cuuint32_t boxU[3] = {kTmaUW, kTmaUH, 1};
    for (int b = 0; b < 2; ++b)
        if (fn(b ? &ws.tmU1 : &ws.tmU0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, b ? ws.U1 : ws.U0, udims,
               strides, boxU, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    return true;
}

static int gjv_blocks(const tnlm_geometry* g) {
    const int tx = (g->nx + kGjvTx * kGjvPx - 1) / (kGjvTx * kGjvPx);
    const int ty = (g->ny + kGjvTy - 1) / kGjvTy;
    return tx * ty * g->N;
}

template <int MODE>
static bool launch_gj_vec(const GjArgs& a, int window, int nb, cudaStream_t st) {
    const int th = kGjvTx * kGjvTy;
    switch (window) {
        case 3: k_gj_vec<3, MODE><<<nb, th, 0, st>>>(a); return true;
        case 5: k_gj_vec<5, MODE><<<nb, th, 0, st>>>(a); return true;
        case 7: k_gj_vec<7, MODE><<<nb, th, 0, st>>>(a); return true;
        case 9: k_gj_vec<9, MODE><<<nb, th, 0, st>>>(a); return true;
        case 11: k_gj_vec<11, MODE><<<nb, th, 0, st>>>(a); return true;
        case 13: k_gj_vec<13, MODE><<<nb, th, 0, st>>>(a); return true;
        case 15: k_gj_vec<15, MODE><<<nb, th, 0, st>>>(a); return true;
        default: return false;
    }
}

// Number of relative-change partial slots used by the sweep / finalisation.
static int gjs_blocks(const tnlm_geometry* g) {
    return ((g->nx + kGjTileX - 1) / kGjTileX) * ((g->ny + kGjTileY - 1) / kGjTileY) * g->N;
}
int gj_blocks(const tnlm_geometry* g) {
    const int a = gjs_blocks(g), b = gjv_blocks(g), c = gj_tma_tiles(g);
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

static GjArgs gj_args(const tnlm_geometry* g, const Workspace& ws, int window, double h,
                      double mu_hat) {
    GjArgs a;
    a.D = ws.D; a.mins = ws.mins; a.g = nullptr; a.uin = nullptr; a.uout = nullptr;
    a.fout = nullptr; a.zn = ws.zn; a.part = ws.part2; a.err = ws.st.err; a.pp = ws.pp;
    a.nx = g->nx; a.ny = g->ny; a.N = g->N; a.rho = (window - 1) / 2; a.W = window; a.clamp = 0;
    a.k2 = (float)(1.4426950408889634 / (h * h));
    a.c1 = (float)(1.0 / (mu_hat + 1.0));
    a.c2 = (float)(mu_hat / (2.0 * mu_hat + 2.0));
    return a;
}

cudaError_t launch_gj_sweep(const tnlm_geometry* g, const Workspace& ws, int window, double h,
                            double mu_hat, const float* gimg, const float* uin, float* uout,
                            float* fout, int clamp, cudaStream_t st) {
    GjArgs a = gj_args(g, ws, window, h, mu_hat);
    a.g = gimg; a.uin = uin; a.uout = uout; a.fout = fout; a.clamp = clamp;
    // the partial slots not written by this launch must read as zero
    const int nv = gjv_blocks(g), ns = gjs_blocks(g);
    const int tw = kGjvTx * kGjvPx;
    const int tx64 = (g->nx + tw - 1) / tw * tw, ty16 = (g->ny + kGjvTy - 1) / kGjvTy * kGjvTy;
    const bool layout_ok = ws.pp.ox >= ((a.rho + 3) / 4) * 4 + 4 && ws.pp.oy >= a.rho &&
                           (ws.pp.px % 4) == 0 && ws.pp.px >= tx64 + 2 * ws.pp.ox &&
                           ws.pp.py >= ty16 + 2 * ws.pp.oy;
    if (layout_ok && ws.tm_ok &&
        (fout ? launch_gj_tma<1>(g, a, ws, window, st) : launch_gj_tma<0>(g, a, ws, window, st))) {
        const int nt = gj_tma_tiles(g), nmax = ns > nv ? ns : nv;
        if (fout && nmax > nt)
            return cudaMemsetAsync(ws.part2 + kPart * (size_t)nt, 0, 8 * kPart * (size_t)(nmax - nt), st);
        return cudaGetLastError();
    }
    if (ws.pp.ox >= ((a.rho + 3) / 4) * 4 + 4 && ws.pp.oy >= a.rho && (ws.pp.px % 4) == 0 &&
        ws.pp.px >= tx64 + 2 * ws.pp.ox && ws.pp.py >= ty16 + 2 * ws.pp.oy &&
        (fout ? launch_gj_vec<1>(a, window, nv, st) : launch_gj_vec<0>(a, window, nv, st))) {
        if (fout && ns > nv)
            return cudaMemsetAsync(ws.part2 + kPart * (size_t)nv, 0, 8 * kPart * (size_t)(ns - nv), st);
        return cudaGetLastError();
    }
    if (fout)
        k_gj<1><<<ns, kGjTileX * kGjTileY, 0, st>>>(a);
    else
        k_gj<0><<<ns, kGjTileX * kGjTileY, 0, st>>>(a);
    if (fout && nv > ns)
        return cudaMemsetAsync(ws.part2 + kPart * (size_t)ns, 0, 8 * kPart * (size_t)(nv - ns), st);
    return cudaGetLastError();
}

cudaError_t launch_weights_norm(const tnlm_geometry* g, const Workspace& ws, int window, double h,
                                cudaStream_t st) {
    GjArgs a = gj_args(g, ws, window, h, 0.0);
    a.uin = ws.U0;
    k_gj<2><<<gjs_blocks(g), kGjTileX * kGjTileY, 0, st>>>(a);
    return cudaGetLastError();
}

// M2 = 0: f = max(g, 0) (or g), with the relative-change partials.
__global__ void __launch_bounds__(256) k_finalize_nogj(const float* __restrict__ gimg,
                                                       float* __restrict__ fout, double* part,
                                                       int nx, int ny, int N, int clamp) {
    const int tile = blockIdx.x / N, i = blockIdx.x % N;
    const int tilesx = (nx + kGjTileX - 1) / kGjTileX;
    const int tid = threadIdx.x;
    const int x = (tile % tilesx) * kGjTileX + (tid & 31);
    const int y = (tile / tilesx) * kGjTileY + (tid >> 5);
    const size_t npx = (size_t)nx * ny;
    float fnew = 0.f, dif = 0.f, ncl = 0.f;
    if (x < nx && y < ny) {
        const size_t k = i * npx + (size_t)y * nx + x;
        const float v = gimg[k];
        fnew = clamp ? fmaxf(v, 0.f) : v;
        ncl = (clamp && v < 0.f) ? 1.f : 0.f;
        dif = fnew - fout[k];
        fout[k] = fnew;
    }
    __shared__ double sh[8];
    const double d2 = block_sum<256>(dif * dif, sh, tid);
    const double n2 = block_sum<256>(fnew * fnew, sh, tid);
    const double c2 = block_sum<256>(ncl, sh, tid);
    if (tid == 0) {
        part[kPart * (size_t)blockIdx.x] = d2;
        part[kPart * (size_t)blockIdx.x + 1] = n2;
        part[kPart * (size_t)blockIdx.x + 2] = c2;
    }
}

cudaError_t launch_finalize_nogj(const tnlm_geometry* g, const Workspace& ws, const float* gimg,
                                 float* fout, int clamp, cudaStream_t st) {
    const int ns = gjs_blocks(g), nv = gjv_blocks(g);
    k_finalize_nogj<<<ns, 256, 0, st>>>(gimg, fout, ws.part2, g->nx, g->ny, g->N, clamp);
    if (nv > ns) return cudaMemsetAsync(ws.part2 + kPart * (size_t)ns, 0, 8 * kPart * (size_t)(nv - ns), st);
    return cudaGetLastError();
}

// Per-iteration monitors: relative change, data term of f^(k-1), clamped
// pixels and (monitor on) the TNLM term of Eq. 1.  256 threads so that each
// reads only a few partials (the loads, not the FP64 adds, set the time); a
// fixed-order tree keeps the sums deterministic.
constexpr int kScalThreads = 256;
__global__ void __launch_bounds__(kScalThreads) k_iter_scalars(const double* part, int nblocks,
                                                               const double* part3, int n3,
                                                               const double* res0, int N, DevState st,
                                                               int kcap) {
    __shared__ double sd[kScalThreads], sn[kScalThreads], sc[kScalThreads], sj[kScalThreads];
    double d = 0.0, n = 0.0, c = 0.0, j = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += kScalThreads) {
        d += part[kPart * (size_t)k];
        n += part[kPart * (size_t)k + 1];
        c += part[kPart * (size_t)k + 2];
    }
    for (int k = threadIdx.x; k < n3; k += kScalThreads) j += part3[k];
    sd[threadIdx.x] = d;
    sn[threadIdx.x] = n;
    sc[threadIdx.x] = c;
    sj[threadIdx.x] = j;
    __syncthreads();
    for (int h = kScalThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sd[threadIdx.x] += sd[threadIdx.x + h];
            sn[threadIdx.x] += sn[threadIdx.x + h];
            sc[threadIdx.x] += sc[threadIdx.x + h];
            sj[threadIdx.x] += sj[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d = sd[0];
        n = sn[0];
        double r = 0.0;
        for (int i = 0; i < N; ++i) r += res0[i];
        const int it = *st.iter;
        if (it < kcap) {
            st.hist_rel[it] = n > 0.0 ? sqrt(d / n) : 0.0;
            st.hist_res[it] = r;
            st.hist_clamp[it] = sc[0];
            st.hist_tnlm[it] = n3 > 0 ? sj[0] : 0.0;
        }
        *st.iter = it + 1;
    }
}

cudaError_t launch_iter_scalars(const tnlm_geometry* g, const Workspace& ws, int nblocks, bool monitor,
                                cudaStream_t st) {
    k_iter_scalars<<<1, kScalThreads, 0, st>>>(ws.part2, nblocks, ws.part3, monitor ? gjs_blocks(g) : 0,
                                               ws.st.res0, g->N, ws.st, ws.kcap);
    return cudaGetLastError();
}

// TNLM term of Eq. 1 for the monitor: per pixel x of phase i,
//   J_i(x) = sum_s omega_{i,i+1}(x, x+s) (f_i(x) - f_{i+1}(x+s))^2
//          + sum_s omega_{i,i-1}(x, x-s) (f_i(x) - f_{i-1}(x-s))^2
// (Eq. 2 for both neighbours, the weights of this outer iteration: the
// stored distances and row minima, normalisers formed on the fly as in the
// sweep), summed per block in FP64; candidates outside the image carry no
// weight.  f is the unpadded result of the iteration.
__global__ void __launch_bounds__(kGjTileX * kGjTileY) k_tnlm_energy(GjArgs a, const float* __restrict__ f,
                                                                    double* __restrict__ part3) {
    const int N = a.N, nx = a.nx, ny = a.ny;
    const int tile = blockIdx.x / N, i = blockIdx.x % N;
    const int tilesx = (nx + kGjTileX - 1) / kGjTileX;
    const int tid = threadIdx.x;
    const int x = (tile % tilesx) * kGjTileX + (tid & 31);
    const int y = (tile / tilesx) * kGjTileY + (tid >> 5);
    const bool in = x < nx && y < ny;
    const size_t npx = (size_t)nx * ny;
    const int ip = (i + N - 1) % N, inx = (i + 1) % N;
    float jt = 0.f;
    if (in) {
        const int rho = a.rho, W = a.W, px = a.pp.px;
        const size_t plane = a.pp.plane, W2 = (size_t)W * W;
        const float k2 = a.k2;
        const size_t pix = (size_t)y * nx + x;
        const float mfk = a.mins[i * npx + pix] * k2;
        const float mbk = a.mins[(N + i) * npx + pix] * k2;
        const float fi = f[i * npx + pix];
        const float* fn = f + inx * npx;
        const float* fp = f + ip * npx;
        const size_t cpos = (size_t)(y + a.pp.oy) * px + x + a.pp.ox;
        const float* dn = a.D + (size_t)i * W2 * plane + cpos;
        const float* dp = a.D + (size_t)ip * W2 * plane + cpos + (size_t)rho * px + rho;
        float jf = 0.f, zf = 0.f, jb = 0.f, zb = 0.f;
        for (int sy = 0; sy < W; ++sy) {
            const int yn = y + sy - rho, yp = y - sy + rho;
            const float* dnr = dn + (size_t)sy * W * plane;
            const float* dpr = dp + (size_t)sy * W * plane - (size_t)sy * px;
            for (int sx = 0; sx < W; ++sx) {
                const int xn = x + sx - rho, xp = x - sx + rho;
                const float ef = ex2_approx(fmaf(-__ldg(dnr + (size_t)sx * plane), k2, mfk));
                const float eb = ex2_approx(fmaf(-__ldg(dpr + (size_t)sx * plane - sx), k2, mbk));
                zf += ef;
                zb += eb;
                if ((unsigned)xn < (unsigned)nx && (unsigned)yn < (unsigned)ny) {
                    const float dv = fi - fn[(size_t)yn * nx + xn];
                    jf = fmaf(ef, dv * dv, jf);
                }
                if ((unsigned)xp < (unsigned)nx && (unsigned)yp < (unsigned)ny) {
                    const float dv = fi - fp[(size_t)yp * nx + xp];
                    jb = fmaf(eb, dv * dv, jb);
                }
            }
        }
        jt = jf / zf + jb / zb;
    }
    __shared__ double sh[kGjTileX * kGjTileY / 32];
    const double tot = block_sum<kGjTileX * kGjTileY>(jt, sh, tid);
    if (tid == 0) part3[blockIdx.x] = tot;
}

int tnlm_energy_blocks(const tnlm_geometry* g) { return gjs_blocks(g); }

cudaError_t launch_tnlm_energy(const tnlm_geometry* g, const Workspace& ws, int window, double h,
                               const float* f, cudaStream_t st) {
    GjArgs a = gj_args(g, ws, window, h, 0.0);
    k_tnlm_energy<<<gjs_blocks(g), kGjTileX * kGjTileY, 0, st>>>(a, f, ws.part3);
    return cudaGetLastError();
}

// Data term of the final image (monitor): the FP64 sum of the projector's
// per-(phase, view, chunk) partials of ||sqrt(w)(y - P f)||^2.
__global__ void __launch_bounds__(kScalThreads) k_sum_partials(const double* part, int n, double* out) {
    __shared__ double sh[kScalThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += kScalThreads) s += part[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = kScalThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t st) {
    k_sum_partials<<<1, kScalThreads, 0, st>>>(part, n, out);
    return cudaGetLastError();
}

// Public weights output: D to [N][W*W][ny][nx], (m, Z) to [4][N][ny][nx].
__global__ void __launch_bounds__(256) k_weights_export(const float* __restrict__ D,
                                                        const float* __restrict__ mins,
                                                        const float* __restrict__ zn,
                                                        float* __restrict__ dist,
                                                        float* __restrict__ norm, PadPlane pp,
                                                        int nx, int ny, int N, int W2) {
    const size_t npx = (size_t)nx * ny;
    const size_t nd = npx * N * W2;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nd + 4 * npx * N;
         k += stride) {
        if (k < nd) {
            const size_t pl = k / npx, pix = k % npx;
            const int y = (int)(pix / nx), x = (int)(pix % nx);
            dist[k] = D[pl * pp.plane + (size_t)(y + pp.oy) * pp.px + x + pp.ox];
        } else {
            const size_t q = k - nd;
            const int c = (int)(q / (npx * N));
            const size_t r = q % (npx * N);
            // c: 0 m_next, 1 Z_next, 2 m_prev, 3 Z_prev
            norm[q] = (c & 1) ? zn[(size_t)(c >> 1) * npx * N + r] : mins[(size_t)(c >> 1) * npx * N + r];
        }
    }
}

cudaError_t launch_weights_export(const tnlm_geometry* g, const Workspace& ws, int window,
                                  float* d_dist, float* d_norm, cudaStream_t st) {
    const size_t n = (size_t)g->nx * g->ny * g->N * (window * window + 4);
    size_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    k_weights_export<<<(int)b, 256, 0, st>>>(ws.D, ws.mins, ws.zn, d_dist, d_norm, ws.pp, g->nx,
                                             g->ny, g->N, window * window);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Gauss-Jacobi sweep with the patch distances recomputed (the alternative to
// storing them: no distance array is read).  A block owns a 64 x TY tile of
// one phase i, the tiles of K4 (k_weights).  It stages g_i with the patch
// halo, g_{i+1} and g_{i-1} with the window and patch halo and the two
// neighbour iterates u_{i+1}, u_{i-1} with the window halo; for every shift
// s it forms, exactly as K4 does (horizontal running sums of the squared
// differences into one of two buffers, vertical sums of the other, one
// barrier per shift), the forward distance D_i(x, s) = |P_i(x) - P_{i+1}(x+s)|^2
// and the backward one D_{i-1}(x-s, s) = |P_{i-1}(x-s) - P_i(x)|^2 of the
// thread's pixels, weights them with the stored row minima,
//   e = 2^(log2(e) (m - D) / h^2),
// and accumulates both directions' sums and normalisers in registers.  The
// backward distance is summed around x rather than around x - s, so its FP32
// association can differ from K4's in the last bit.
// ---------------------------------------------------------------------------
struct FArgs {
    const float* g;       // g^(k) [N][ny][nx]
    const float* mins;    // [2][N][ny][nx] row minima (toward i+1, toward i-1)
    const float* uin;     // padded iterate planes [N][py][px], zero outside the image
    float* uout;          // padded (intermediate sweeps)
    float* fout;          // unpadded result (last sweep)
    double* part;         // last sweep: kPart partials per block
    int* err;
    PadPlane pp;
    int nx, ny, N, rho, W, clamp;
    float k2, c1, c2;
};

template <int R>
struct FGeo {
    using G = WGeo<R>;
    int GJW, GJH, GJS, UW, UH, US;
    __host__ __device__ explicit FGeo(int rho) {
        GJW = (G::TX + 2 * rho + 2 * R) | 1;
        GJH = G::TY + 2 * rho + 2 * R;
        GJS = (GJW * GJH + 3) / 4 * 4;
        UW = G::TX + 2 * rho;
        UH = G::TY + 2 * rho;
        US = (UW * UH + 3) / 4 * 4;
    }
    __host__ __device__ size_t floats() const {
        return (size_t)G::GIW * G::GIH + 2 * (size_t)GJS + 4 * 32 * (size_t)G::HP + 2 * (size_t)US;
    }
};

template <int R, int MODE>
__global__ void __launch_bounds__(256, 2) k_gj_fused(FArgs a) {
    using G = WGeo<R>;
    extern __shared__ __align__(16) float sm[];
    const int rho = a.rho, W = a.W, N = a.N, nx = a.nx, ny = a.ny;
    const FGeo<R> L(rho);
    float* Gi = sm;                                  // g_i at rows Y0-R.., columns X0-R..
    float* Gn = Gi + G::GIW * G::GIH;                // g_{i+1} at rows Y0-rho-R.., columns X0-rho-R..
    float* Gp = Gn + L.GJS;                          // g_{i-1}, same region
    float* H = Gp + L.GJS;                           // [buffer][direction][32][HP]
    float* Un = H + 4 * 32 * G::HP;                  // u_{i+1} at rows Y0-rho.., columns X0-rho..
    float* Up = Un + L.US;                           // u_{i-1}, same region
    const int i = blockIdx.z, inx = (i + 1) % N, ip = (i + N - 1) % N;
    const int X0 = blockIdx.x * G::TX, Y0 = blockIdx.y * G::TY;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t npx = (size_t)nx * ny;
    const float* gi = a.g + i * npx;
    const float* gn = a.g + inx * npx;
    const float* gp = a.g + ip * npx;
    for (int r = warp; r < G::GIH; r += 8)
        for (int c = lane; c < G::GIW; c += 32) {
            const int x = X0 - R + c, y = Y0 - R + r;
            Gi[r * G::GIW + c] = (x >= 0 && x < nx && y >= 0 && y < ny) ? gi[(size_t)y * nx + x] : 0.f;
        }
    for (int r = warp; r < L.GJH; r += 8)
        for (int c = lane; c < L.GJW; c += 32) {
            const int x = X0 - rho - R + c, y = Y0 - rho - R + r;
            const bool in = x >= 0 && x < nx && y >= 0 && y < ny;
            Gn[r * L.GJW + c] = in ? gn[(size_t)y * nx + x] : 0.f;
            Gp[r * L.GJW + c] = in ? gp[(size_t)y * nx + x] : 0.f;
        }
    const size_t plane = a.pp.plane;
    for (int r = warp; r < L.UH; r += 8)
        for (int c = lane; c < L.UW; c += 32) {
            const int x = X0 - rho + c, y = Y0 - rho + r;
            const bool in = x >= 0 && x < nx && y >= 0 && y < ny;
            const size_t o = (size_t)(y + a.pp.oy) * a.pp.px + x + a.pp.ox;
            Un[r * L.UW + c] = in ? a.uin[inx * plane + o] : 0.f;
            Up[r * L.UW + c] = in ? a.uin[ip * plane + o] : 0.f;
        }
    __syncthreads();

    // pass-1 task: H row hr, 8 adjacent columns from g8
    const int g8 = 8 * ((warp & 1) * 4 + (lane & 3));
    const int hr = (warp >> 1) * 8 + (lane >> 2);
    // pass-2 task: output column c2, output rows r2 .. r2 + RPT - 1
    const int c2 = (warp & 1) * 32 + lane;
    const int r2 = (warp >> 1) * G::RPT;
    const int x2 = X0 + c2;
    const bool xin = x2 < nx;

    // horizontal patch sums of direction dir (0: g_{i+1} at +s, 1: g_{i-1} at -s)
    auto horizontal = [&](const float* Gj, int sx, int sy, float* Hb) {
        if (hr >= G::HR) return;
        float d2[4 * G::NQ4];
        const float* pi = Gi + hr * G::GIW + g8;
        const float* pj = Gj + (hr + sy + rho) * L.GJW + g8 + sx + rho;
#pragma unroll
        for (int t = 0; t < G::NQ4; ++t) {
            const float4 v = *(const float4*)(pi + 4 * t);
            const float vi[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (4 * t + u < G::NQ) {
                    const float d = vi[u] - pj[4 * t + u];
                    d2[4 * t + u] = d * d;
                }
            }
        }
        float h[8];
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
            float m = 0.f;
#pragma unroll
            for (int t = 1; t <= 2 * R; ++t) m = (t == 1) ? d2[c + 1] : m + d2[c + t];
            h[c] = (R == 0) ? d2[c] : d2[c] + m;
            h[c + 1] = (R == 0) ? d2[c + 1] : m + d2[c + 2 * R + 1];
        }
        float* o = Hb + hr * G::HP + g8;
        *(float4*)o = make_float4(h[0], h[1], h[2], h[3]);
        *(float4*)(o + 4) = make_float4(h[4], h[5], h[6], h[7]);
    };
    // vertical sums of a buffer: this thread's RPT distances
    auto vertical = [&](const float* Hb, float* dv) {
        const float* hb = Hb + r2 * G::HP + c2;
        float hv[G::RPT + 2 * R];
#pragma unroll
        for (int t = 0; t < G::RPT + 2 * R; ++t) hv[t] = hb[t * G::HP];
#pragma unroll
        for (int r = 0; r < G::RPT; r += 2) {
            float m = 0.f;
#pragma unroll
            for (int t = 1; t <= 2 * R; ++t) m = (t == 1) ? hv[r + 1] : m + hv[r + t];
            dv[r] = (R == 0) ? hv[r] : hv[r] + m;
            if (r + 1 < G::RPT) dv[r + 1] = (R == 0) ? hv[r + 1] : m + hv[r + 2 * R + 1];
        }
    };

    const float k2 = a.k2;
    float mfk[G::RPT], mbk[G::RPT], af[G::RPT], zf[G::RPT], ab[G::RPT], zb[G::RPT];
#pragma unroll
    for (int r = 0; r < G::RPT; ++r) {
        const int y = Y0 + r2 + r;
        const bool in = xin && y < ny;
        const size_t pix = (size_t)y * nx + x2;
        mfk[r] = in ? a.mins[i * npx + pix] * k2 : 0.f;
        mbk[r] = in ? a.mins[(N + i) * npx + pix] * k2 : 0.f;
        af[r] = zf[r] = ab[r] = zb[r] = 0.f;
    }
    const int HB = 32 * G::HP;                       // one direction's buffer
    horizontal(Gn, -rho, -rho, H);
    horizontal(Gp, rho, rho, H + HB);
    __syncthreads();
    const int W2 = W * W;
    int sx = -rho, sy = -rho;
    for (int k = 0; k < W2; ++k) {
        if (k + 1 < W2) {
            const int nx1 = (sx == rho) ? -rho : sx + 1;
            const int ny1 = (sx == rho) ? sy + 1 : sy;
            float* Hn = H + ((k + 1) & 1) * 2 * HB;
            horizontal(Gn, nx1, ny1, Hn);
            horizontal(Gp, -nx1, -ny1, Hn + HB);
        }
        float df[G::RPT], db[G::RPT];
        const float* Hc = H + (k & 1) * 2 * HB;
        vertical(Hc, df);
        vertical(Hc + HB, db);
        const bool fcol = xin && (unsigned)(x2 + sx) < (unsigned)nx;
        const bool bcol = xin && (unsigned)(x2 - sx) < (unsigned)nx;
        const float* un = Un + (r2 + sy + rho) * L.UW + c2 + sx + rho;
        const float* up = Up + (r2 - sy + rho) * L.UW + c2 - sx + rho;
#pragma unroll
        for (int r = 0; r < G::RPT; ++r) {
            const int y = Y0 + r2 + r;
            const bool yin = y < ny;
            if (fcol && yin && (unsigned)(y + sy) < (unsigned)ny) {
                const float e = ex2_approx(fmaf(-df[r], k2, mfk[r]));
                af[r] = fmaf(e, un[r * L.UW], af[r]);
                zf[r] += e;
            }
            if (bcol && yin && (unsigned)(y - sy) < (unsigned)ny) {
                const float e = ex2_approx(fmaf(-db[r], k2, mbk[r]));
                ab[r] = fmaf(e, up[r * L.UW], ab[r]);
                zb[r] += e;
            }
        }
        __syncthreads();
        if (sx == rho) { sx = -rho; ++sy; } else { ++sx; }
    }
    float dsq = 0.f, nsq = 0.f, ncl = 0.f;
    bool bad = false;
#pragma unroll
    for (int r = 0; r < G::RPT; ++r) {
        const int y = Y0 + r2 + r;
        if (!xin || y >= ny) continue;
        bad |= !(zf[r] >= 0.5f) || !(zb[r] >= 0.5f);
        const size_t pix = (size_t)y * nx + x2;
        const float unew = fmaf(a.g[i * npx + pix], a.c1, a.c2 * (af[r] / zf[r] + ab[r] / zb[r]));
        if (MODE == 0) {
            a.uout[i * plane + (size_t)(y + a.pp.oy) * a.pp.px + x2 + a.pp.ox] = unew;
        } else {
            const float fnew = a.clamp ? fmaxf(unew, 0.f) : unew;
            if (a.clamp && unew < 0.f) ncl += 1.f;
            const float fold = a.fout[i * npx + pix];
            a.fout[i * npx + pix] = fnew;
            dsq = fmaf(fnew - fold, fnew - fold, dsq);
            nsq = fmaf(fnew, fnew, nsq);
        }
    }
    if (bad) atomicOr(a.err, 8);
    if (MODE == 1) {
        __shared__ double sh[8];
        const double d2 = block_sum<256>(dsq, sh, tid);
        const double n2 = block_sum<256>(nsq, sh, tid);
        const double c3 = block_sum<256>(ncl, sh, tid);
        if (tid == 0) {
            const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            a.part[kPart * blk] = d2;
            a.part[kPart * blk + 1] = n2;
            a.part[kPart * blk + 2] = c3;
        }
    }
}

template <int R>
static size_t fused_smem(int rho) { return sizeof(float) * FGeo<R>(rho).floats(); }

cudaError_t prepare_gj_fused() {
    cudaError_t e = cudaSuccess;
#define TNLM_PREP_F(R)                                                                              \
    if (e == cudaSuccess)                                                                           \
        e = cudaFuncSetAttribute(k_gj_fused<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 (int)fused_smem<R>((kMaxWindow - 1) / 2));                         \
    if (e == cudaSuccess)                                                                           \
        e = cudaFuncSetAttribute(k_gj_fused<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 (int)fused_smem<R>((kMaxWindow - 1) / 2));
    TNLM_PREP_F(0) TNLM_PREP_F(1) TNLM_PREP_F(2) TNLM_PREP_F(3)
#undef TNLM_PREP_F
    return e;
}

template <int R>
static cudaError_t launch_fused_r(const tnlm_geometry* g, const FArgs& a, cudaStream_t st) {
    using G = WGeo<R>;
    dim3 grid((g->nx + G::TX - 1) / G::TX, (g->ny + G::TY - 1) / G::TY, g->N);
    const size_t sm = fused_smem<R>(a.rho);
    if (a.fout) k_gj_fused<R, 1><<<grid, 256, sm, st>>>(a);
    else k_gj_fused<R, 0><<<grid, 256, sm, st>>>(a);
    cudaError_t e = cudaGetLastError();
    // the partial slots this launch does not write must read as zero
    const size_t nb = (size_t)grid.x * grid.y * grid.z, nmax = (size_t)gj_blocks(g);
    if (e == cudaSuccess && a.fout && nmax > nb)
        e = cudaMemsetAsync(a.part + kPart * nb, 0, 8 * kPart * (nmax - nb), st);
    return e;
}

bool fused_supported(int patch, int window) {
    return patch >= 1 && patch <= 7 && (patch & 1) && window >= 1 && window <= 15 && (window & 1);
}

cudaError_t launch_gj_fused(const tnlm_geometry* g, const Workspace& ws, int patch, int window, double h,
                            double mu_hat, const float* gimg, const float* uin, float* uout, float* fout,
                            int clamp, cudaStream_t st) {
    if (!fused_supported(patch, window)) return cudaErrorInvalidValue;
    FArgs a;
    a.g = gimg; a.mins = ws.mins; a.uin = uin; a.uout = uout; a.fout = fout; a.part = ws.part2;
    a.err = ws.st.err; a.pp = ws.pp;
    a.nx = g->nx; a.ny = g->ny; a.N = g->N; a.rho = (window - 1) / 2; a.W = window; a.clamp = clamp;
    a.k2 = (float)(1.4426950408889634 / (h * h));
    a.c1 = (float)(1.0 / (mu_hat + 1.0));
    a.c2 = (float)(mu_hat / (2.0 * mu_hat + 2.0));
    switch ((patch - 1) / 2) {
        case 0: return launch_fused_r<0>(g, a, st);
        case 1: return launch_fused_r<1>(g, a, st);
        case 2: return launch_fused_r<2>(g, a, st);
        case 3: return launch_fused_r<3>(g, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnlm
