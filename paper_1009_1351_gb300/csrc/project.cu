// Projector P_i and its exact transpose (Eq. 1; the CGLS box and Eq. 4 use
// both).  Entry (ray, pixel) of the system matrix is the length of the ray
// inside the pixel square, the quantity Siddon's method traces (Sec. 3).
//
// K1 (k_project): one thread per ray.  A ray with |u_x| >= |u_y| marches over
// pixel columns: inside one column it spans less than one pixel in y, so it
// meets at most two rows, lo and lo+1, and the length in row lo is the
// column width times the fraction of the column where the ray is below row
// lo+1, divided by |u_x|.  Rays with |u_y| > |u_x| march over rows the same
// way.  The 32 rays of a warp are adjacent bins of one view, so at a given
// column they read adjacent rows: the column-marching class reads the
// column-major copy T and the row-marching class the row-major copy R,
// which makes both classes' loads consecutive across the warp.  All lanes
// of a warp walk the union of their column ranges in lock step.
//
// K2 (k_backproject): the transpose as an atomic-free gather.  A block owns
// a 32 x 32 pixel tile of one phase.  Four of its 8 warps deposit the
// column-marching rays and four the row-marching rays; the four warps of a
// class take every 4th view.  For a view, the rays that can touch the tile
// form one bin range (from the fan angles of the tile corners), cut to the
// bins of the warp's class (one run per view, tabulated at geometry
// creation).  All 32 lanes of a warp handle the same ray at once: for a
// column-marching ray lane c is tile column c and, with the very same
// floating-point steps as K1, finds the ray's rows lo, lo+1 in that column
// and adds frac * L * z and (1 - frac) * L * z to the warp's private
// accumulator tile; a row-marching ray is handled the same way with lane c
// as tile row c.  One class per warp means one private tile per warp, which
// keeps five blocks resident per SM.  The private tiles are summed in a
// fixed order at the end, so the result is bitwise reproducible, and every
// matrix entry is formed by the same FP32 operations on the same per-ray
// constants as in K1.
//
// Per-ray constants (built in FP64 on the host at geometry creation):
//   float4 (kk, alpha, ik, L): the position across the marching lines at the
//   start of line k is alpha + kk*k (pixel units), ik = 1/|kk|, and L > 0 is
//   the length per line (pixel / |u_x|) of a column-marching ray; L < 0 marks
//   a row-marching ray (length -L per row).
#include "internal.cuh"

#include <math.h>

#include <mutex>

namespace tnlm {

// ---------------------------------------------------------------------------
// Dual layout of pairs.  Along each line of the row-major copy R [N][ny][nx+4]
// and of the column-major copy T [N][nx][ny+4] (two pad positions on each
// side of the nx or ny interior ones, X[q] = 0 there), entry q holds the
// float2 (X[q] - X[q+1], X[q+1]): the two values a ray meets in a line, with
// the difference the projector's interpolation takes, so K1 reads one 8-byte
// pair per line and forms exactly the FP32 values it would form from X[q] and
// X[q+1].  Entries 1 .. n+1 depend on the image and are written here; the
// others stay zero from the workspace clear.
// ---------------------------------------------------------------------------
// MODE 0: R, T of img.  MODE 1: also a copy of img into cp (u^(0) = f).
// MODE 2: first the CGLS direction update cp = gr + b_i img (for phases
// whose CGLS is still active, else cp = img; the same FP32 operation as a
// separate update kernel would do), then R, T of the result.  img is never
// written: a block also updates the pixels of the row and column beyond its
// tile for their pairs, from the values of img before the update.
template <int MODE>
__global__ void __launch_bounds__(256) k_prep_dual(const float* __restrict__ img, float2* __restrict__ R,
                                                   float2* __restrict__ T, float* __restrict__ cp,
                                                   const float* __restrict__ gr,
                                                   const double* __restrict__ bcoef,
                                                   const int* __restrict__ active, int nx, int ny) {
    __shared__ float tile[33][33];   // [row][col]: the 32 x 32 tile and one more row and column
    const int i = blockIdx.z;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const size_t npx = (size_t)nx * ny;
    const float* src = img + i * npx;
    float2* Ri = R + (size_t)i * ny * (nx + 4);
    float2* Ti = T + (size_t)i * nx * (ny + 4);
    const bool upd = MODE == 2 && active[i];
    const float b = MODE == 2 ? (float)bcoef[i] : 0.f;
    for (int e = tid; e < 33 * 33; e += 256) {
        const int k = e / 33, c = e - k * 33;
        const int x = x0 + c, y = y0 + k;
        float v = 0.f;
        if (x < nx && y < ny) {
            const size_t idx = (size_t)y * nx + x;
            v = src[idx];
            if (upd) v = fmaf(b, v, gr[i * npx + idx]);
            if (MODE != 0 && k < 32 && c < 32) cp[i * npx + idx] = v;   // this block's own pixels
        }
        tile[k][c] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int x = x0 + tx, y = y0 + k;        // row pairs, lanes along the row
        if (x < nx && y < ny) {
            float2* line = Ri + (size_t)y * (nx + 4);
            const float v0 = tile[k][tx], v1 = tile[k][tx + 1];
            line[x + 2] = make_float2(v0 - v1, v1);
            if (x == 0) line[1] = make_float2(0.f - v0, v0);
        }
        const int xc = x0 + k, yc = y0 + tx;      // column pairs, lanes along the column
        if (xc < nx && yc < ny) {
            float2* line = Ti + (size_t)xc * (ny + 4);
            const float v0 = tile[tx][k], v1 = tile[tx + 1][k];
            line[yc + 2] = make_float2(v0 - v1, v1);
            if (yc == 0) line[1] = make_float2(0.f - v0, v0);
        }
    }
}

cudaError_t launch_prep_dual(const tnlm_geometry* g, const float* img, float* R, float* T,
                             cudaStream_t st) {
    dim3 grid((g->nx + 31) / 32, (g->ny + 31) / 32, g->N), blk(32, 8);
    k_prep_dual<0><<<grid, blk, 0, st>>>(img, (float2*)R, (float2*)T, nullptr,
                                         nullptr, nullptr, nullptr, g->nx, g->ny);
    return cudaGetLastError();
}

cudaError_t launch_prep_dual_copy(const tnlm_geometry* g, const float* img, float* cp, float* R,
                                  float* T, cudaStream_t st) {
    dim3 grid((g->nx + 31) / 32, (g->ny + 31) / 32, g->N), blk(32, 8);
    k_prep_dual<1><<<grid, blk, 0, st>>>(img, (float2*)R, (float2*)T, cp,
                                         nullptr, nullptr, nullptr, g->nx, g->ny);
    return cudaGetLastError();
}

cudaError_t launch_prep_dual_update(const tnlm_geometry* g, const float* s, float* s_new,
                                    const float* gr, const double* bcoef, const int* active,
                                    float* R, float* T, cudaStream_t st) {
    dim3 grid((g->nx + 31) / 32, (g->ny + 31) / 32, g->N), blk(32, 8);
    k_prep_dual<2><<<grid, blk, 0, st>>>(s, (float2*)R, (float2*)T, s_new, gr, bcoef, active,
                                         g->nx, g->ny);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K1
// ---------------------------------------------------------------------------
// A projector block holds kProjViews consecutive views of one phase, each
// with kProjWarpsPerView warps of 32 adjacent bins.  Consecutive views of a
// phase are a small rotation apart, so their rays march over nearly the same
// pixels at the same time and the block's warps share the gathered lines in
// L1.  In eager A/B runs at 512^2 (888 bins), 4 views in 128-thread blocks
// took 0.725 / 0.275 ms per launch at 360 / 90 views against 0.754 / 0.281
// with 256 threads and 0.823 / 0.298 with 512; in the graph-replayed
// benchmark the mean launch is within 1 % of one view per 256-thread block.
#ifndef TNLM_PROJ_VPB
#define TNLM_PROJ_VPB 4
#endif
constexpr int kProjViews = TNLM_PROJ_VPB;
static_assert(kProjViews == 1 || kProjViews == 2 || kProjViews == 4 || kProjViews == 8,
              "views per projector block");
constexpr int kProjWarpsPerView = kProjThreads / 32 / kProjViews;
static_assert(kProjWarpsPerView >= 1, "projector block smaller than its views");
constexpr int kProjBinsPerBlock = 32 * kProjWarpsPerView;

struct ProjArgs {
    const float2* R;
    const float2* T;
    const float4* ray;
    int nx, ny, V, B, nbc, nvg;   // bin chunks per view group, view groups per phase
    ProjOut o;
};

// Lower of the two across-line positions of a ray inside line k, its lower
// line index clamped into the zero pads [-1, nacross], and the fraction of
// the line's width where the ray lies in that line.  K1 and K2 both use this,
// so they form every matrix entry with identical FP32 operations.
struct Cut {
    float frac;
    int j;
};
__device__ __forceinline__ Cut line_cut(float kk, float am, float ik, float kf, float nacross_f) {
    const float mn = fmaf(kk, kf, am);
    const float fl = fminf(fmaxf(floorf(mn), -1.f), nacross_f);
    Cut c;
    c.frac = fminf(1.f, fmaf(fl - mn, ik, ik));
    // exact float -> int of a small integer-valued float
    c.j = __float_as_int(fl + 12582912.f) - 0x4B400000;
    return c;
}

// March one ray over 'lines' (columns of T or rows of R) lo..hi.  base points
// at the pair of the first interior element of line 0 of the phase; 'pitch'
// is the line stride in pairs; 'nacross' the interior length of a line.  The
// position across the line at the start of line k is alpha + kk*k (pixel
// units); am = alpha + min(kk, 0) is the lower end of the ray's span inside
// line 0.  With v0, v1 the values at the lower line index and the next, the
// pair holds (v0 - v1, v1) and the ray accumulates frac * (v0 - v1) + v1.
#ifndef TNLM_PROJ_UNROLL
#define TNLM_PROJ_UNROLL 4
#endif
constexpr int kProjUnroll = TNLM_PROJ_UNROLL;   // lines per unrolled step of a ray's march
__device__ __forceinline__ float march(const float2* __restrict__ base, int pitch, int nacross,
                                       float kk, float am, float ik, int lo, int hi, bool on) {
    float acc = 0.f;
    float kf = (float)lo;
    int koff = lo * pitch;
    const float na = (float)nacross;
#pragma unroll kProjUnroll
    for (int k = lo; k <= hi; ++k) {
        const Cut c = line_cut(kk, am, ik, kf, na);
        if (on) {
            const float2 pv = __ldg(base + (koff + c.j));
            acc = fmaf(c.frac, pv.x, acc + pv.y);
        }
        kf += 1.f;
        koff += pitch;
    }
    return acc;
}

// Conservative index range [lo, hi] of lines 0..nlines-1 where the ray's
// across-position alpha + kk*k lies within [-1, nacross+1].
__device__ __forceinline__ void line_range(float kk, float alpha, int nlines, int nacross,
                                           int* lo, int* hi) {
    float a = 0.f, b = (float)nlines;
    if (kk != 0.f) {
        const float xa = (-1.f - alpha) / kk, xb = ((float)nacross + 1.f - alpha) / kk;
        a = fmaxf(a, fminf(xa, xb) - 1.f);
        b = fminf(b, fmaxf(xa, xb) + 1.f);
    } else if (!(alpha >= -1.f && alpha <= (float)nacross + 1.f)) {
        a = 1.f;
        b = 0.f;
    }
    *lo = (int)floorf(a);
    *hi = min(nlines - 1, (int)ceilf(b));
    if (!(b >= a)) { *lo = 1; *hi = 0; }
}

template <int MODE>
__global__ void __launch_bounds__(kProjThreads) k_project(ProjArgs a) {
    const int pg = blockIdx.x / a.nbc;          // phase * nvg + view group
    const int chunk = blockIdx.x - pg * a.nbc;
    const int phase = pg / a.nvg;
    const int w = threadIdx.x >> 5;
    const int view = (pg - phase * a.nvg) * kProjViews + w / kProjWarpsPerView;
    const int b = chunk * kProjBinsPerBlock + (w % kProjWarpsPerView) * 32 + (threadIdx.x & 31);
    const bool valid = view < a.V && b < a.B;
    const int gv = phase * a.V + (view < a.V ? view : 0);
    const float4 rp = a.ray[(size_t)gv * a.B + (valid ? b : 0)];
    const bool colm = rp.w > 0.f;

    float q = 0.f;
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int cls = 0; cls < 2; ++cls) {
        // cls 0: column-marching rays read T; cls 1: row-marching rays read R
        const bool in = valid && (cls == 0 ? colm : !colm);
        const int nlines = cls == 0 ? a.nx : a.ny;
        const int nacross = cls == 0 ? a.ny : a.nx;
        int lo = 1, hi = 0;
        if (in) line_range(rp.x, rp.y, nlines, nacross, &lo, &hi);
        const bool any = in && hi >= lo;
        if (__ballot_sync(full, any)) {
            const int wl = __reduce_min_sync(full, any ? lo : 0x7fffffff);
            const int wh = __reduce_max_sync(full, any ? hi : -1);
            const float2* base = cls == 0 ? a.T + (size_t)phase * a.nx * (a.ny + 4) + 2
                                          : a.R + (size_t)phase * a.ny * (a.nx + 4) + 2;
            const float acc = march(base, nacross + 4, nacross, rp.x, rp.y + fminf(rp.x, 0.f), rp.z,
                                    wl, wh, in);
            if (in) q = acc * fabsf(rp.w);
        }
    }

    const size_t ray = (size_t)gv * a.B + b;
    float part = 0.f;
    if (MODE == 0) {
        if (valid) a.o.q[ray] = q;
    } else if (MODE == 1) {
        if (valid) {
            const float s = a.o.sw[ray];
            const float rr = s * (a.o.y[ray] - q);
            a.o.r[ray] = rr;
            a.o.z[ray] = s * rr;
            part = rr * rr;
        }
    } else {
        if (valid) {
            const float t = a.o.sw[ray] * q;
            a.o.q[ray] = t;
            part = t * t;
        }
    }
    if (MODE != 0) {
        __shared__ double sh[kProjThreads / 32];
        const double tot = block_sum<kProjThreads>(part, sh, threadIdx.x);
        if (threadIdx.x == 0) a.o.part[blockIdx.x] = tot;
    }
}

static int proj_bin_chunks(const tnlm_geometry* g) { return (g->B + kProjBinsPerBlock - 1) / kProjBinsPerBlock; }
static int proj_view_groups(const tnlm_geometry* g) { return (g->V + kProjViews - 1) / kProjViews; }
int proj_blocks_per_phase(const tnlm_geometry* g) { return proj_bin_chunks(g) * proj_view_groups(g); }

cudaError_t launch_project(const tnlm_geometry* g, const float* R, const float* T,
                           const ProjOut& o, cudaStream_t st) {
    ProjArgs a;
    a.R = (const float2*)R; a.T = (const float2*)T; a.ray = g->d_ray;
    a.nx = g->nx; a.ny = g->ny; a.V = g->V; a.B = g->B;
    a.nbc = proj_bin_chunks(g); a.nvg = proj_view_groups(g);
    a.o = o;
    dim3 grid(proj_blocks_per_phase(g) * g->N);
    switch (o.mode) {
        case 0: k_project<0><<<grid, kProjThreads, 0, st>>>(a); break;
        case 1: k_project<1><<<grid, kProjThreads, 0, st>>>(a); break;
        default: k_project<2><<<grid, kProjThreads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K2
// ---------------------------------------------------------------------------
constexpr int kBpT = 32;        // tile side
// Warps per backprojector block, half per ray class.  Measured per launch
// at 512^2 (360 / 90 views): 4 warps 1.313 / 0.362 ms, 8 warps 1.254 /
// 0.338 ms, 12 warps 1.261 / 0.352 ms; 8 is kept.
#ifndef TNLM_BP_WARPS
#define TNLM_BP_WARPS 8
#endif
constexpr int kBpWarps = TNLM_BP_WARPS;     // per block: kBpClassWarps per ray class
static_assert(kBpWarps % 2 == 0 && kBpWarps >= 2 && kBpWarps <= 16, "backprojector warps");
constexpr int kBpMinBlocks = 40 / kBpWarps > 0 ? 40 / kBpWarps : 1;   // about 40 resident warps per SM
constexpr int kBpClassWarps = kBpWarps / 2;
constexpr int kBpMaxGroups = 4;  // view groups per tile (CTAs per tile)

struct BpArgs {
    const float* sino;
    float* img;            // output when the tile's views are not split
    float* scratch;        // [G][N][ny][nx] partial images when they are
    double* part;          // nullable: per-tile partial sums of img^2
    const float2* view;
    const float4* ray;
    const int4* vcls;      // per view: bin ranges of the two ray classes
    int nx, ny, V, B, G;
    float sidp, inv_dg, half_b;
};

size_t bp_smem_bytes() {
    return sizeof(float) * (kBpWarps * kBpT * kBpT + kBpT * (kBpT + 1)) +
           sizeof(float4) * kBpWarps * 32;
}

// Add frac * Lz to line j and (1 - frac) * Lz to line j + 1 of a private
// accumulator column (tile-local index j relative to j0, n lines).
// The lower line index here is not clamped into [-1, nacross] as in K1: the
// two lines that receive a deposit lie inside the tile and the image, where
// that clamp leaves the index unchanged, so every deposited entry is the one
// K1 forms.
__device__ __forceinline__ void deposit(float* acc, float kk, float am, float ik, float Lz,
                                        float kf, int j0, unsigned n) {
    const float mn = fmaf(kk, kf, am);
    const float fl = floorf(mn);
    const float frac = fminf(1.f, fmaf(fl - mn, ik, ik));
    const int r0 = (__float_as_int(fl + 12582912.f) - 0x4B400000) - j0;
    if ((unsigned)r0 < n) acc[r0 * 32] += frac * Lz;
    if ((unsigned)(r0 + 1) < n) acc[(r0 + 1) * 32] += fmaf(-frac, Lz, Lz);
}

// The first kBpClassWarps warps deposit the column-marching rays (lane =
// tile column, private tile [row][col]), the others the row-marching rays
// (lane = tile row, private tile [col][row]); both layouts are conflict-free
// for their class, and each warp needs only one private tile.
// DIRECT: the block sees all views of its tile and writes the image (and the
// squared-norm partial); otherwise it writes its view group's partial image.
template <bool DIRECT, bool PART>
__global__ void __launch_bounds__(kBpWarps * 32, kBpMinBlocks) k_backproject(BpArgs a) {
    extern __shared__ float sm[];
    float* acc = sm;                                    // [warp][32][32]
    float* tsum = acc + kBpWarps * kBpT * kBpT;         // [row][col + 1]
    float4* stg = (float4*)(tsum + kBpT * (kBpT + 1));  // [warp][32]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const bool colw = w < kBpClassWarps;                // warp-uniform
    const int X0 = blockIdx.x * kBpT, Y0 = blockIdx.y * kBpT;
    const int phase = blockIdx.z / a.G, grp = blockIdx.z - phase * a.G;
    const int ncols = min(kBpT, a.nx - X0), nrows = min(kBpT, a.ny - Y0);
    for (int k = tid; k < kBpWarps * kBpT * kBpT; k += blockDim.x) sm[k] = 0.f;
    __syncthreads();
    float* my = acc + w * kBpT * kBpT + lane;
    float4* myS = stg + w * 32;
    // this lane's marching line (tile column or row), the origin and count of
    // the lines across it, and whether the lane's line lies in the image
    const float kf = colw ? (float)(X0 + lane) : (float)(Y0 + lane);
    const int j0 = colw ? Y0 : X0;
    const unsigned nacross = (unsigned)(colw ? nrows : ncols);
    const int nalong = colw ? ncols : nrows;
    const bool lane_on = lane < nalong;
    // tile corners (pixel units about the isocentre), clipped to the image
    const float xa = X0 - 0.5f * a.nx, xb = X0 + ncols - 0.5f * a.nx;
    const float ya = Y0 - 0.5f * a.ny, yb = Y0 + nrows - 0.5f * a.ny;
    const unsigned full = 0xffffffffu;
    const int S = kBpClassWarps * a.G;                      // view stride of a warp
    const int gw = grp * kBpClassWarps + (w % kBpClassWarps);  // first view of this warp
    const float4* rays = a.ray + (size_t)phase * a.V * a.B;
    const float* zs = a.sino + (size_t)phase * a.V * a.B;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    for (int m0 = 0; gw + S * m0 < a.V; m0 += 32) {
        // bin ranges of this warp's class in the next 32 views of this warp,
        // one view per lane
        const int vl = gw + S * (m0 + lane);
        int lo = 1, hi = 0;
        if (vl < a.V) {
            const float2 vt = a.view[(size_t)phase * a.V + vl];
            float bmin = 3e30f, bmax = -3e30f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float cx = (c & 1) ? xb : xa, cy = (c & 2) ? yb : ya;
                const float X = vt.y * cx - vt.x * cy;
                const float Y = a.sidp - (vt.x * cx + vt.y * cy);
                const float bc = fmaf(atanf(X / Y), a.inv_dg, a.half_b);
                bmin = fminf(bmin, bc);
                bmax = fmaxf(bmax, bc);
            }
            const int4 cr = a.vcls[(size_t)phase * a.V + vl];
            lo = max(max(0, (int)floorf(bmin) - 1), colw ? cr.x : cr.z);
            hi = min(min(a.B - 1, (int)ceilf(bmax) + 1), colw ? cr.y : cr.w);
        }
        const unsigned todo = __ballot_sync(full, lo <= hi);
        if (!todo) continue;
        // walk the (view, 32-ray chunk) pairs, prefetching the next chunk's
        // ray constants and sinogram values while the current one is deposited
        int vi = __ffs(todo) - 1;
        int b0 = __shfl_sync(full, lo, vi);
        int bh = __shfl_sync(full, hi, vi);
        int nb = min(32, bh - b0 + 1);
        size_t rb = (size_t)(gw + S * (m0 + vi)) * a.B + b0;
        float4 rp = lane < nb ? __ldg(rays + rb + lane) : zero4;
        float zz = lane < nb ? __ldg(zs + rb + lane) : 0.f;
        while (true) {
            int nvi = vi, nb0 = b0 + 32, nbh = bh;
            if (nb0 > bh) {
                const unsigned rest = todo & ~((2u << vi) - 1u);
                nvi = rest ? __ffs(rest) - 1 : -1;
                if (nvi >= 0) {
                    nb0 = __shfl_sync(full, lo, nvi);
                    nbh = __shfl_sync(full, hi, nvi);
                }
            }
            int nnb = 0;
            float4 nrp = zero4;
            float nzz = 0.f;
            if (nvi >= 0) {
                nnb = min(32, nbh - nb0 + 1);
                const size_t nrb = (size_t)(gw + S * (m0 + nvi)) * a.B + nb0;
                if (lane < nnb) {
                    nrp = __ldg(rays + nrb + lane);
                    nzz = __ldg(zs + nrb + lane);
                }
            }
            // bit t: staged ray t is of this warp's class
            const unsigned mine =
                __ballot_sync(full, lane < nb && (colw ? rp.w > 0.f : !(rp.w > 0.f)));
            __syncwarp();
            myS[lane] = make_float4(rp.x, rp.y + fminf(rp.x, 0.f), rp.z, fabsf(rp.w) * zz);
            __syncwarp();
            const unsigned staged = nb >= 32 ? full : (1u << nb) - 1u;
            if (mine == staged && nalong == kBpT) {
                // the usual case: every staged ray is of this class and the
                // tile side is full -- no per-ray class or lane test
#pragma unroll 4
                for (int t = 0; t < nb; ++t) {
                    const float4 r = myS[t];
                    deposit(my, r.x, r.y, r.z, r.w, kf, j0, nacross);
                }
            } else {
#pragma unroll 2
                for (int t = 0; t < nb; ++t) {
                    const float4 r = myS[t];
                    if (((mine >> t) & 1u) && lane_on) deposit(my, r.x, r.y, r.z, r.w, kf, j0, nacross);
                }
            }
            if (nvi < 0) break;
            vi = nvi; b0 = nb0; bh = nbh; nb = nnb; rp = nrp; zz = nzz;
        }
    }
    __syncthreads();
    // fixed-order reduction of the private tiles
    for (int k = tid; k < kBpT * kBpT; k += blockDim.x) {
        const int r = k >> 5, c = k & 31;
        float s = 0.f;
#pragma unroll
        for (int ww = 0; ww < kBpClassWarps; ++ww) s += acc[(ww * kBpT + r) * kBpT + c];
        tsum[r * (kBpT + 1) + c] = s;
    }
    __syncthreads();
    for (int k = tid; k < kBpT * kBpT; k += blockDim.x) {
        const int c = k >> 5, r = k & 31;
        float s = tsum[r * (kBpT + 1) + c];
#pragma unroll
        for (int ww = kBpClassWarps; ww < kBpWarps; ++ww) s += acc[(ww * kBpT + c) * kBpT + r];
        tsum[r * (kBpT + 1) + c] = s;
    }
    __syncthreads();
    float sq = 0.f;
    const int nph = gridDim.z / a.G;
    float* out = DIRECT ? a.img : a.scratch + (size_t)grp * nph * a.ny * a.nx;
    for (int k = tid; k < kBpT * kBpT; k += blockDim.x) {
        const int r = k >> 5, c = k & 31;
        if (r < nrows && c < ncols) {
            const float v = tsum[r * (kBpT + 1) + c];
            out[((size_t)phase * a.ny + Y0 + r) * a.nx + X0 + c] = v;
            sq = fmaf(v, v, sq);
        }
    }
    if (DIRECT && PART) {
        __shared__ double sh[kBpWarps];
        const double tot = block_sum<kBpWarps * 32>(sq, sh, tid);
        if (tid == 0)
            a.part[(size_t)phase * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
}

// Sum of the G partial images in a fixed order (and the per-tile partials).
template <bool PART>
__global__ void __launch_bounds__(256) k_bp_combine(const float* __restrict__ scratch,
                                                    float* __restrict__ img, double* part,
                                                    int nx, int ny, int N, int G) {
    const int X0 = blockIdx.x * kBpT, Y0 = blockIdx.y * kBpT, phase = blockIdx.z;
    const size_t stride = (size_t)N * nx * ny;
    float sq = 0.f;
    for (int k = threadIdx.x; k < kBpT * kBpT; k += blockDim.x) {
        const int r = k >> 5, c = k & 31;
        if (Y0 + r < ny && X0 + c < nx) {
            const size_t idx = ((size_t)phase * ny + Y0 + r) * nx + X0 + c;
            float v = 0.f;
            for (int g = 0; g < G; ++g) v += scratch[g * stride + idx];
            img[idx] = v;
            sq = fmaf(v, v, sq);
        }
    }
    if (PART) {
        __shared__ double sh[8];
        const double tot = block_sum<256>(sq, sh, threadIdx.x);
        if (threadIdx.x == 0)
            part[(size_t)phase * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
}

int bp_blocks_per_phase(const tnlm_geometry* g) {
    return ((g->nx + kBpT - 1) / kBpT) * ((g->ny + kBpT - 1) / kBpT);
}

// Opt the backprojector variants into their dynamic shared memory and
// count the CTA slots of the current device (called at geometry creation,
// outside any stream capture).
cudaError_t prepare_backproject(int* slots) {
    const int smem = (int)bp_smem_bytes();
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_backproject<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_backproject<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_backproject<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backproject<false, false>,
                                                           kBpWarps * 32, bp_smem_bytes())) != cudaSuccess)
        return e;
    *slots = (sms > 0 && per_sm > 0) ? sms * per_sm : 1;
    return cudaSuccess;
}

int bp_max_groups(const tnlm_geometry* g) {
    const int m = (g->V + kBpClassWarps - 1) / kBpClassWarps;
    return m < kBpMaxGroups ? m : kBpMaxGroups;
}

// View groups per tile (CTAs per tile).  Tiles differ in cost (rays per
// tile fall off towards the edge of the field of view), so the grid should
// span about three waves of resident CTAs for the block scheduler to even
// out: the smallest G that reaches three waves, else the largest G that
// still leaves each warp at least 4 views (measured on 256^2 slices: with
// 360 views one group per tile took 0.69 ms per call, four groups 0.55 ms).
static int bp_groups(const tnlm_geometry* g) {
    if (g->tune_bp_groups > 0) return min(g->tune_bp_groups, bp_max_groups(g));
    const long long slots = g->cta_slots_bp > 0 ? g->cta_slots_bp : 1;
    const long long tiles = (long long)bp_blocks_per_phase(g) * g->N;
    int G = 1;
    while (G < bp_max_groups(g) && tiles * G < 3 * slots &&
           g->V >= 4 * kBpClassWarps * (G + 1))
        ++G;
    return G;
}

size_t bp_scratch_floats(const tnlm_geometry* g) {
    return (size_t)kBpMaxGroups * g->N * g->nx * g->ny;
}

template <bool DIRECT, bool PART>
static cudaError_t launch_bp(const BpArgs& a, dim3 grid, cudaStream_t st) {
    k_backproject<DIRECT, PART><<<grid, kBpWarps * 32, bp_smem_bytes(), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const tnlm_geometry* g, const float* sino, float* img,
                               double* part, float* scratch, cudaStream_t st) {
    BpArgs a;
    a.sino = sino; a.img = img; a.part = part; a.scratch = scratch;
    a.view = g->d_view; a.ray = g->d_ray; a.vcls = g->d_vcls;
    a.nx = g->nx; a.ny = g->ny; a.V = g->V; a.B = g->B;
    a.G = scratch ? bp_groups(g) : 1;
    a.sidp = (float)(g->sid / g->pixel);
    a.inv_dg = (float)(g->sdd / g->bin_mm);
    a.half_b = 0.5f * (float)(g->B - 1);
    const dim3 tiles((g->nx + kBpT - 1) / kBpT, (g->ny + kBpT - 1) / kBpT, g->N);
    const dim3 grid(tiles.x, tiles.y, g->N * a.G);
    cudaError_t e;
    if (a.G == 1)
        return part ? launch_bp<true, true>(a, grid, st) : launch_bp<true, false>(a, grid, st);
    e = launch_bp<false, false>(a, grid, st);
    if (e != cudaSuccess) return e;
    if (part)
        k_bp_combine<true><<<tiles, 256, 0, st>>>(scratch, img, part, g->nx, g->ny, g->N, a.G);
    else
        k_bp_combine<false><<<tiles, 256, 0, st>>>(scratch, img, part, g->nx, g->ny, g->N, a.G);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free projection: the dual-layout scratch of K1 lives in a
// file-scope device array instead of the handle's workspace.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchFloats = (size_t)12 << 20;  // 48 MiB per device
static __device__ __align__(256) float g_proj_scratch[kStaticScratchFloats];

size_t static_scratch_floats() { return kStaticScratchFloats; }

// Device address of the array on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached.
cudaError_t static_scratch_ptr(float** out) {
    static std::mutex mu;
    static float* ptrs[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_proj_scratch);
        if (e != cudaSuccess) return e;
        ptrs[dev] = (float*)p;
    }
    *out = ptrs[dev];
    return cudaSuccess;
}

}  // namespace tnlm
