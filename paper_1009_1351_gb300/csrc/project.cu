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
// K2 (k_backproject): one thread per pixel, a gather over views -- no
// atomics, so results are bitwise reproducible.  For a view, the bins whose
// rays can touch the pixel lie within +-(1/sqrt 2)/dist of the pixel
// centre's fan angle; for each, the exact chord of the line through the
// square follows from the line's signed distance e to the pixel centre:
// with a = |u_x|, b = |u_y|, chord = clamp(((a+b)/2 - |e|) / min(a,b), 0, 1) /
// max(a,b) (a trapezoid in e whose area is the pixel area).  This is the
// same matrix entry K1 accumulates, so K2 is the transpose of K1 up to FP32
// rounding.
#include "internal.cuh"

#include <math.h>

namespace tnlm {

// ---------------------------------------------------------------------------
// Dual layout: R[i][iy][ix+2] (row-major, two zero columns each side) and
// T[i][ix][iy+2] (column-major, two zero rows each side).  Pads are zeroed
// once when the workspace is created and never written.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_prep_dual(const float* __restrict__ img,
                                                   float* __restrict__ R, float* __restrict__ T,
                                                   int nx, int ny) {
    __shared__ float tile[32][33];
    const int i = blockIdx.z;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const size_t npx = (size_t)nx * ny;
    const float* src = img + i * npx;
    float* Ri = R + (size_t)i * ny * (nx + 4);
    float* Ti = T + (size_t)i * nx * (ny + 4);
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int x = x0 + threadIdx.x, y = y0 + k;
        float v = 0.f;
        if (x < nx && y < ny) {
            v = src[(size_t)y * nx + x];
            Ri[(size_t)y * (nx + 4) + x + 2] = v;
        }
        tile[k][threadIdx.x] = v;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int y = y0 + threadIdx.x, x = x0 + k;
        if (x < nx && y < ny) Ti[(size_t)x * (ny + 4) + y + 2] = tile[threadIdx.x][k];
    }
}

cudaError_t launch_prep_dual(const tnlm_geometry* g, const float* img, float* R, float* T,
                             cudaStream_t st) {
    dim3 grid((g->nx + 31) / 32, (g->ny + 31) / 32, g->N), blk(32, 8);
    k_prep_dual<<<grid, blk, 0, st>>>(img, R, T, g->nx, g->ny);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K1
// ---------------------------------------------------------------------------
struct ProjArgs {
    const float* R;
    const float* T;
    const float2* view;
    const float2* bin;
    int nx, ny, V, B, nchunk;
    float sidp;      // sid / pixel
    float pixel;
    ProjOut o;
};

// March one ray over 'lines' (columns of T or rows of R) lo..hi.  base points
// at the first interior element of line 0 of the phase; 'pitch' is the line
// stride; 'nacross' the interior length of a line.  The position across the
// line at the start of line k is alpha + kk*k (pixel units).
__device__ __forceinline__ float march(const float* __restrict__ base, int pitch, int nacross,
                                       float kk, float alpha, float ik, int lo, int hi, bool on) {
    float acc = 0.f;
#pragma unroll 2
    for (int k = lo; k <= hi; ++k) {
        const float c0 = fmaf(kk, (float)k, alpha);
        const float mn = fminf(c0, c0 + kk);
        // clamp the lower line index into the zero pads [-1, nacross]; the
        // fraction is taken w.r.t. the clamped index, so a ray entirely
        // below (above) the image puts all (no) weight on pad line -1
        // (lines nacross, nacross+1), i.e. contributes zero.
        const float fl = fminf(fmaxf(floorf(mn), -1.f), (float)nacross);
        const float frac = fminf(1.f, (fl + 1.f - mn) * ik);
        const int j = (int)fl;
        if (on) {
            const float* p = base + (size_t)k * pitch + j;
            const float v0 = __ldg(p), v1 = __ldg(p + 1);
            acc = fmaf(frac, v0 - v1, acc + v1);
        }
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
    const int gv = blockIdx.x / a.nchunk;      // phase * V + view
    const int chunk = blockIdx.x - gv * a.nchunk;
    const int phase = gv / a.V;
    const int b = chunk * kProjThreads + threadIdx.x;
    const bool valid = b < a.B;
    const float2 vt = a.view[gv];
    const float2 bt = a.bin[valid ? b : 0];
    // ray direction u = -(cos(t+g), sin(t+g)); line: u_x*Y - u_y*X = c0 in
    // pixel units about the isocentre, c0 = sid*sin(g)/pixel.
    const float ux = -(vt.x * bt.x - vt.y * bt.y);
    const float uy = -(vt.y * bt.x + vt.x * bt.y);
    const float c0 = a.sidp * bt.y;
    const bool colm = fabsf(ux) >= fabsf(uy);
    const float hx = 0.5f * a.nx, hy = 0.5f * a.ny;

    float q = 0.f;
    const unsigned full = 0xffffffffu;
    // --- column-marching class (reads T) ---
    {
        const bool in = valid && colm;
        const float kk = uy / ux;
        const float alpha = c0 / ux - kk * hx + hy;   // row coordinate at column 0
        const float ik = fabsf(ux / uy);
        int lo = 1, hi = 0;
        if (in) line_range(kk, alpha, a.nx, a.ny, &lo, &hi);
        const unsigned m = __ballot_sync(full, in && hi >= lo);
        if (m) {
            const int wl = __reduce_min_sync(full, (in && hi >= lo) ? lo : 0x7fffffff);
            const int wh = __reduce_max_sync(full, (in && hi >= lo) ? hi : -1);
            const float* base = a.T + (size_t)phase * a.nx * (a.ny + 4) + 2;
            const float acc = march(base, a.ny + 4, a.ny, kk, alpha, ik, wl, wh, in);
            if (in) q = acc * (a.pixel / fabsf(ux));
        }
    }
    // --- row-marching class (reads R) ---
    {
        const bool in = valid && !colm;
        const float kk = ux / uy;
        const float alpha = -c0 / uy - kk * hy + hx;  // column coordinate at row 0
        const float ik = fabsf(uy / ux);
        int lo = 1, hi = 0;
        if (in) line_range(kk, alpha, a.ny, a.nx, &lo, &hi);
        const unsigned m = __ballot_sync(full, in && hi >= lo);
        if (m) {
            const int wl = __reduce_min_sync(full, (in && hi >= lo) ? lo : 0x7fffffff);
            const int wh = __reduce_max_sync(full, (in && hi >= lo) ? hi : -1);
            const float* base = a.R + (size_t)phase * a.ny * (a.nx + 4) + 2;
            const float acc = march(base, a.nx + 4, a.nx, kk, alpha, ik, wl, wh, in);
            if (in) q = acc * (a.pixel / fabsf(uy));
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

int proj_chunks(const tnlm_geometry* g) { return (g->B + kProjThreads - 1) / kProjThreads; }

cudaError_t launch_project(const tnlm_geometry* g, const float* R, const float* T,
                           const ProjOut& o, cudaStream_t st) {
    ProjArgs a;
    a.R = R; a.T = T; a.view = g->d_view; a.bin = g->d_bin;
    a.nx = g->nx; a.ny = g->ny; a.V = g->V; a.B = g->B; a.nchunk = proj_chunks(g);
    a.sidp = (float)(g->sid / g->pixel);
    a.pixel = (float)g->pixel;
    a.o = o;
    dim3 grid(a.nchunk * g->N * g->V);
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
struct BpArgs {
    const float* sino;
    float* img;
    double* part;          // nullable: per-block partial sums of img^2
    const float2* view;
    const float2* bin;
    const float4* ray;
    int nx, ny, V, B;
    float sidp, pixel, inv_dg, half_b;
};

template <bool PART>
__global__ void __launch_bounds__(kBpTile * kBpTile) k_backproject(BpArgs a) {
    extern __shared__ float2 s_bin[];          // [B] (cos g, sin g)
    const int tid = threadIdx.x;
    for (int k = tid; k < a.B; k += blockDim.x) s_bin[k] = a.bin[k];
    __syncthreads();
    // 8 warps, each an 8 x 4 pixel sub-tile (compact footprint on the detector)
    const int w = tid >> 5, l = tid & 31;
    const int lx = (l & 7) + 8 * (w & 1);
    const int ly = (l >> 3) + 4 * (w >> 1);
    const int ix = blockIdx.x * kBpTile + lx, iy = blockIdx.y * kBpTile + ly;
    const int phase = blockIdx.z;
    const bool inside = ix < a.nx && iy < a.ny;
    const float cx = (float)ix - 0.5f * (a.nx - 1);
    const float cy = (float)iy - 0.5f * (a.ny - 1);
    const float hwk = 0.70711f * 1.0001f * a.inv_dg;

    float acc = 0.f;
    if (inside) {
        const float2* vtab = a.view + (size_t)phase * a.V;
        for (int v = 0; v < a.V; ++v) {
            const float2 vt = vtab[v];
            // X = cross(c_dir, c - S), Y = dot(c_dir, c - S), c_dir = -(cos t, sin t)
            const float X = vt.y * cx - vt.x * cy;
            const float Y = a.sidp - (vt.x * cx + vt.y * cy);
            const float gc = atanf(X / Y);
            const float bc = fmaf(gc, a.inv_dg, a.half_b);
            const float hw = hwk / Y + 1e-3f;
            const int b0 = max(0, (int)ceilf(bc - hw));
            const int b1 = min(a.B - 1, (int)floorf(bc + hw));
            const size_t rbase = ((size_t)phase * a.V + v) * a.B;
            for (int b = b0; b <= b1; ++b) {
                const float2 gb = s_bin[b];
                const float4 rp = __ldg(a.ray + rbase + b);
                const float e = gb.x * X - gb.y * Y;           // signed distance (pixels)
                const float frac = __saturatef((rp.x - fabsf(e)) * rp.y);
                acc = fmaf(frac * rp.z, __ldg(a.sino + rbase + b), acc);
            }
        }
        acc *= a.pixel;
        a.img[((size_t)phase * a.ny + iy) * a.nx + ix] = acc;
    }
    if (PART) {
        __shared__ double sh[kBpTile * kBpTile / 32];
        const double tot = block_sum<kBpTile * kBpTile>(inside ? acc * acc : 0.f, sh, tid);
        if (tid == 0)
            a.part[(size_t)phase * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
}

int bp_blocks_per_phase(const tnlm_geometry* g) {
    return ((g->nx + kBpTile - 1) / kBpTile) * ((g->ny + kBpTile - 1) / kBpTile);
}

cudaError_t launch_backproject(const tnlm_geometry* g, const float* sino, float* img,
                               double* part, cudaStream_t st) {
    BpArgs a;
    a.sino = sino; a.img = img; a.part = part;
    a.view = g->d_view; a.bin = g->d_bin; a.ray = g->d_ray;
    a.nx = g->nx; a.ny = g->ny; a.V = g->V; a.B = g->B;
    a.sidp = (float)(g->sid / g->pixel);
    a.pixel = (float)g->pixel;
    a.inv_dg = (float)(g->sdd / g->bin_mm);
    a.half_b = 0.5f * (float)(g->B - 1);
    dim3 grid((g->nx + kBpTile - 1) / kBpTile, (g->ny + kBpTile - 1) / kBpTile, g->N);
    const size_t smem = sizeof(float2) * g->B;
    if (part)
        k_backproject<true><<<grid, kBpTile * kBpTile, smem, st>>>(a);
    else
        k_backproject<false><<<grid, kBpTile * kBpTile, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tnlm
