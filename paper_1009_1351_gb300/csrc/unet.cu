// Learned warm start: a 2D U-Net over the N phases of a slice as channels,
// with hand-written BF16-storage / FP32-accumulate training and inference
// kernels (forward, backward, Adam).  The network only supplies a start
// image; the TNLM iteration (Sec. 2.2) still runs to its own stopping rule.
//
// Architecture (all convolutions zero-padded, with bias; c_l = base 2^l):
//   encoder l = 0..L-1: x_0 = input, x_l = maxpool2(e_{l-1});
//                       e_l = relu(conv3(relu(conv3(x_l))))
//   decoder l = L-2..0: c = [upsample2(d_{l+1}), e_l] (d_{L-1} = e_{L-1});
//                       d_l = relu(conv3(relu(conv3(c))))
//   output = input + conv1(d_0); loss = mean squared error.
// Storage: input, convolution weights and every post-ReLU activation in
// BF16 (nearest even), accumulation, output, gradients, master weights and
// Adam moments in FP32.  Layout NCHW; every tensor is a view (pointer,
// batch stride) so that e_l is written straight into the channels of the
// decoder's concatenation buffer.  Max pooling sends the gradient to the
// first maximum of each 2x2 window in row-major order.  Reductions over
// pixels (weight and bias gradients, loss) are two-stage with a fixed
// order, so a training step is deterministic.
#include "internal.cuh"
#include "tcgen05.cuh"
#include "tnlm_unet.h"

#include <cuda_bf16.h>

#include <math.h>
#include <stdio.h>

#include <vector>

namespace tnlm {
namespace unet {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// conv3x3, forward and input-gradient (same kernel, different weights):
//   out[b][o][y][x] = bias[o] + sum_c sum_k W[o][c][k] * in[b][c][y+ky-1][x+kx-1]
// Block: 16 x 16 pixels x 16 output channels, 128 threads, each thread two
// vertically adjacent pixels x 16 outputs.  Input channels in chunks of 16
// staged in shared memory (with the 1-pixel halo), weights too.
// TIN: bf16 (activations) or float (gradients).  With mask != nullptr the
// input is multiplied by (mask > 0) on load (the ReLU of the layer whose
// gradient is being propagated).
// ---------------------------------------------------------------------------
constexpr int kCT = 16, kCO = 16, kCI = 16;

__device__ __forceinline__ float ld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld(const float* p) { return *p; }

template <typename TIN, bool OUT_BF16, bool RELU>
__global__ void __launch_bounds__(128) k_conv3(const TIN* __restrict__ in, long in_bs, int Cin,
                                               const bf16* __restrict__ mask, long mask_bs,
                                               const bf16* __restrict__ w, const float* __restrict__ bias,
                                               void* __restrict__ out, long out_bs, int Cout, int H, int W) {
    __shared__ float si[kCI][kCT + 2][kCT + 3];
    __shared__ float sw[kCI][9][kCO];
    const int tid = threadIdx.x;
    const int nco = (Cout + kCO - 1) / kCO;
    const int b = blockIdx.z / nco, o0 = (blockIdx.z % nco) * kCO;
    const int X0 = blockIdx.x * kCT, Y0 = blockIdx.y * kCT;
    const int tx = tid & 15, ty = (tid >> 4) * 2;
    float acc[2][kCO];
#pragma unroll
    for (int o = 0; o < kCO; ++o) {
        const float bb = (bias && o0 + o < Cout) ? bias[o0 + o] : 0.f;
        acc[0][o] = bb;
        acc[1][o] = bb;
    }
    const TIN* inb = in + (long)b * in_bs;
    const bf16* mb = mask ? mask + (long)b * mask_bs : nullptr;
    const long plane = (long)H * W;
    for (int c0 = 0; c0 < Cin; c0 += kCI) {
        __syncthreads();
        for (int e = tid; e < kCI * (kCT + 2) * (kCT + 2); e += 128) {
            const int c = e / ((kCT + 2) * (kCT + 2)), r = e % ((kCT + 2) * (kCT + 2));
            const int yy = Y0 - 1 + r / (kCT + 2), xx = X0 - 1 + r % (kCT + 2);
            float v = 0.f;
            if (c0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const long off = (long)(c0 + c) * plane + (long)yy * W + xx;
                v = ld(inb + off);
                if (mb && !(ld(mb + off) > 0.f)) v = 0.f;
                if (sizeof(TIN) == 4) v = __bfloat162float(__float2bfloat16_rn(v));   // gradients enter as BF16
            }
            si[c][r / (kCT + 2)][r % (kCT + 2)] = v;
        }
        for (int e = tid; e < kCI * 9 * kCO; e += 128) {
            const int o = e % kCO, k = (e / kCO) % 9, c = e / (kCO * 9);
            sw[c][k][o] = (c0 + c < Cin && o0 + o < Cout)
                              ? __bfloat162float(w[((long)(o0 + o) * Cin + c0 + c) * 9 + k]) : 0.f;
        }
        __syncthreads();
        const int cmax = min(kCI, Cin - c0);
        for (int c = 0; c < cmax; ++c) {
            float v[4][3];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) v[r][q] = si[c][ty + r][tx + q];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float a0 = v[k / 3][k % 3], a1 = v[k / 3 + 1][k % 3];
#pragma unroll
                for (int o = 0; o < kCO; ++o) {
                    const float ww = sw[c][k][o];
                    acc[0][o] = fmaf(a0, ww, acc[0][o]);
                    acc[1][o] = fmaf(a1, ww, acc[1][o]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int y = Y0 + ty + r, x = X0 + tx;
        if (y >= H || x >= W) continue;
#pragma unroll
        for (int o = 0; o < kCO; ++o) {
            if (o0 + o >= Cout) break;
            float v = acc[r][o];
            if (RELU) v = fmaxf(v, 0.f);
            const long off = (long)b * out_bs + (long)(o0 + o) * plane + (long)y * W + x;
            if (OUT_BF16) ((bf16*)out)[off] = __float2bfloat16_rn(v);
            else ((float*)out)[off] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// conv3x3 forward on the tensor cores (tcgen05): an implicit GEMM with
// M = a 16 x 8 pixel tile (128 rows), N = COUT output channels, K = 9 taps x
// Cin in steps of 16 channels; BF16 operands, FP32 accumulator in tensor
// memory.  Per 16-channel chunk the 18 x 10 input halo is staged in shared
// memory as [channel group of 8][row][col][8 channels], so the A operand of
// a tap is one 16-byte copy per (pixel, channel group) into the canonical
// K-major layout; B comes pre-packed in that layout (k_pack_tc).  The
// operands are double-buffered: step s + 1 is built while the MMA of step s
// runs; its completion (tcgen05.commit -> mbarrier) frees the buffer.  The
// epilogue adds the bias, applies ReLU and stores BF16 (NCHW).
// ---------------------------------------------------------------------------
constexpr int kTcvTW = 16, kTcvTH = 8;
constexpr int kTcvHW = kTcvTW + 2, kTcvHH = kTcvTH + 2;      // halo 18 x 10

__device__ __forceinline__ int tc_off(int row, int k) {      // bytes; rows of 16 K-elements
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// MODE 0: forward (BF16 input, + bias, ReLU, BF16 output).  MODE 1: input
// gradient (FP32 gradient input times the ReLU mask of the layer, rounded to
// BF16 on load; FP32 output, no bias).
// A CTA computes output channels blockIdx.z * COUT .. + COUT - 1 of
// cout_total (the N dimension is split over CTAs for the small deep levels).
template <int COUT, int MODE>
__global__ void __launch_bounds__(256) k_conv3_tc(const void* __restrict__ in_, long in_bs, int Cin,
                                                  const bf16* __restrict__ mask, long mask_bs,
                                                  const uint4* __restrict__ wpk, const float* __restrict__ bias,
                                                  void* __restrict__ out_, long out_bs, int H, int W,
                                                  int tiles_x, int cout_total, int* err) {
    constexpr int TCOLS = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : (COUT <= 128 ? 128 : 256));
    const int oc0 = blockIdx.z * COUT;
    __shared__ __align__(128) uint4 halo[2 * kTcvHH * kTcvHW];          // [cg][y][x] x 8 BF16
    __shared__ __align__(1024) uint4 sA[2][3][128 * 2];                 // 2 buffers x 3 taps x 128 rows x 32 B
    __shared__ __align__(1024) uint4 sB[2][3][COUT * 2];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = blockIdx.x, b = blockIdx.y;
    const int X0 = (t % tiles_x) * kTcvTW, Y0 = (t / tiles_x) * kTcvTH;
    const long plane = (long)H * W;
    if (warp == 0) {
        tmem_alloc(&s_taddr, TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    const int nchunk = (Cin + 15) / 16;
    constexpr uint32_t idesc = idesc_f16(128, COUT, true);
    int s = 0;
    bool ok = true;
    for (int ch = 0; ch < nchunk && ok; ++ch) {
        const int c0 = ch * 16;
        __syncthreads();      // the previous chunk's A builds have read the halo
        bf16* hb = (bf16*)halo;
        for (int e = tid; e < 16 * kTcvHH * kTcvHW; e += 256) {
            const int c = e / (kTcvHH * kTcvHW), pix = e % (kTcvHH * kTcvHW);
            const int yy = Y0 - 1 + pix / kTcvHW, xx = X0 - 1 + pix % kTcvHW;
            bf16 v = __float2bfloat16_rn(0.f);
            if (c0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const long off = (long)(c0 + c) * plane + (long)yy * W + xx;
                if (MODE == 0) {
                    v = ((const bf16*)in_)[(long)b * in_bs + off];
                } else {
                    float g = ((const float*)in_)[(long)b * in_bs + off];
                    if (mask && !(__bfloat162float(mask[(long)b * mask_bs + off]) > 0.f)) g = 0.f;
                    v = __float2bfloat16_rn(g);
                }
            }
            hb[((c >> 3) * kTcvHH * kTcvHW + pix) * 8 + (c & 7)] = v;
        }
        __syncthreads();
        // one step = one kernel row (3 taps): three MMAs per barrier
        for (int dy = 0; dy < 3; ++dy, ++s) {
            const int buf = s & 1;
            if (s >= 2 && !mbar_wait_bounded(&bar[buf], (unsigned)(((s - 2) >> 1) & 1))) {
                s_abort = 1;
                atomicOr(err, 16);
            }
            {   // A: pixel m = tid & 127, channel group tid >> 7, the three taps of row dy
                const int m = tid & 127, cg = tid >> 7;
                const int y = (m >> 4) + dy, x = m & 15;
                const uint4* hrow = halo + (cg * kTcvHH + y) * kTcvHW + x;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) sA[buf][dx][tc_off(m, 8 * cg) >> 4] = hrow[dx];
            }
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const uint4* wsrc = wpk + (long)((3 * dy + dx) * nchunk + ch) * cout_total * 2 + oc0 * 2;
                for (int q = tid; q < COUT * 2; q += 256) sB[buf][dx][q] = wsrc[q];
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (s_abort) { ok = false; break; }
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
                    umma_f16(taddr, smem_desc(smem_u32(&sA[buf][dx][0]), 128, 256),
                             smem_desc(smem_u32(&sB[buf][dx][0]), 128, 256), idesc, (s > 0 || dx > 0) ? 1u : 0u);
                umma_commit(&bar[buf]);
            }
        }
    }
    // s MMAs were issued; the last one's commit covers all earlier ones (also
    // after an abort, before the tensor memory is released)
    if (s > 0 && !mbar_wait_bounded(&bar[(s - 1) & 1], (unsigned)(((s - 1) >> 1) & 1))) {
        atomicOr(err, 16);
        ok = false;
    }
    tc_fence_after();
    if (ok) {
        // epilogue: warp w reads lanes 32 (w % 4) .. and half (w / 4) of the columns
        const int q = warp & 3, half = warp >> 2;
        const int m = 32 * q + lane;
        const int y = Y0 + (m >> 4), x = X0 + (m & 15);
        const bool pin = y < H && x < W;
        constexpr int CH = COUT / 2;
        for (int o0 = half * CH; o0 < (half + 1) * CH; o0 += 16) {
            uint32_t v[16];
            __syncwarp();
            tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)o0, v);
            if (pin) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const long off = (long)b * out_bs + (long)(oc0 + o0 + j) * plane + (long)y * W + x;
                    if (MODE == 0)
                        ((bf16*)out_)[off] = __float2bfloat16_rn(fmaxf(__uint_as_float(v[j]) + bias[oc0 + o0 + j], 0.f));
                    else
                        ((float*)out_)[off] = __uint_as_float(v[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, TCOLS);
}

// Packs the transposed, flipped weights of a 3x3 layer for the input
// gradient on k_conv3_tc: output channel n = the layer's input channel,
// chunk channel j = the layer's output channel ch*16 + j, tap k -> 8 - k.
__global__ void k_pack_tc_t(const float* __restrict__ w, int O, int C, bf16* __restrict__ dst) {
    const int nchunk = (O + 15) / 16;
    const long n = (long)9 * nchunk * C * 16;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = (int)(i % 16), c = (int)((i / 16) % C);
    const int ch = (int)((i / ((long)16 * C)) % nchunk), k = (int)(i / ((long)16 * C * nchunk));
    const int o = ch * 16 + j;
    const float v = o < O ? w[((long)o * C + c) * 9 + (8 - k)] : 0.f;
    dst[(long)(k * nchunk + ch) * C * 16 + tc_off(c, j) / 2] = __float2bfloat16_rn(v);
}

// Packs the BF16 weights of a 3x3 layer for k_conv3_tc: for tap k and
// channel chunk ch, the COUT x 16 block (output o, channel c0 + j) in the
// canonical K-major layout; channels past Cin are zero.
__global__ void k_pack_tc(const float* __restrict__ w, int O, int C, bf16* __restrict__ dst) {
    const int nchunk = (C + 15) / 16;
    const long n = (long)9 * nchunk * O * 16;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = (int)(i % 16), o = (int)((i / 16) % O);
    const int ch = (int)((i / ((long)16 * O)) % nchunk), k = (int)(i / ((long)16 * O * nchunk));
    const int c = ch * 16 + j;
    const float v = c < C ? w[((long)o * C + c) * 9 + k] : 0.f;
    dst[(long)(k * nchunk + ch) * O * 16 + tc_off(o, j) / 2] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// conv3x3 weight gradient on the tensor cores, first stage (split over
// image rows):  D[o][c*9 + t] = sum_p gz[o][p] * in[c][p + off_t]  with
// M = 128 output channels (zero rows past Cout), N = 16 input channels x 9
// taps = 144, K = 16 consecutive pixels of one image row per MMA.  gz is the
// FP32 gradient times the ReLU mask, rounded to BF16 (as everywhere a
// gradient enters a convolution); in is the BF16 layer input.  Per step the
// three input rows around the pixel row (16 channels x 18 pixels) are staged
// in shared memory and the operands are built into double buffers in the
// canonical K-major layout.  Needs W % 16 == 0.  The accumulator (144 of 256
// TMEM columns) is written as this slice's partial sums [o][c][t].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_conv3_wgrad_tc(const float* __restrict__ gout, long g_bs,
                                                        const bf16* __restrict__ act, long a_bs,
                                                        const bf16* __restrict__ in, long in_bs, int Cin,
                                                        int Cout, int H, int W, int B, int rows_per,
                                                        float* __restrict__ part, int* err) {
    __shared__ __align__(16) bf16 srow[16][3][20];                      // [c][row][x0-1 .. x0+16]
    __shared__ __align__(1024) uint4 sA[2][128 * 2];
    __shared__ __align__(1024) uint4 sB[2][144 * 2];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.x * 16, o0 = blockIdx.y * 128;
    const long plane = (long)H * W;
    const long r_begin = (long)blockIdx.z * rows_per, r_end = min((long)B * H, r_begin + rows_per);
    if (warp == 0) {
        tmem_alloc(&s_taddr, 256);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    constexpr uint32_t idesc = idesc_f16(128, 144, true);
    int s = 0;
    bool ok = true;
    for (long br = r_begin; br < r_end && ok; ++br) {
        const int b = (int)(br / H), y = (int)(br % H);
        for (int x0 = 0; x0 < W && ok; x0 += 16, ++s) {
            const int buf = s & 1;
            if (s >= 2 && !mbar_wait_bounded(&bar[buf], (unsigned)(((s - 2) >> 1) & 1))) {
                s_abort = 1;
                atomicOr(err, 16);
            }
            // the three input rows of 16 channels, pixels x0-1 .. x0+16 (zero outside)
            for (int e = tid; e < 16 * 3 * 18; e += 256) {
                const int c = e / 54, r = (e / 18) % 3, xi = e % 18;
                const int yy = y - 1 + r, xx = x0 - 1 + xi;
                bf16 v = __float2bfloat16_rn(0.f);
                if (c0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
                    v = in[(long)b * in_bs + (long)(c0 + c) * plane + (long)yy * W + xx];
                srow[c][r][xi] = v;
            }
            {   // A: row o = tid & 127, pixels 8h .. 8h + 7 with h = tid >> 7
                const int o = tid & 127, h = tid >> 7;
                uint32_t pk[4] = {0u, 0u, 0u, 0u};
                if (o0 + o < Cout) {
                    const long off = (long)(o0 + o) * plane + (long)y * W + x0 + 8 * h;
                    const float4 g0 = *(const float4*)(gout + (long)b * g_bs + off);
                    const float4 g1 = *(const float4*)(gout + (long)b * g_bs + off + 4);
                    float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                    if (act) {
                        const uint4 mr = *(const uint4*)(act + (long)b * a_bs + off);
                        const bf16* mv = (const bf16*)&mr;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (!(__bfloat162float(mv[j]) > 0.f)) gv[j] = 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        pk[j] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(gv[2 * j])) |
                                ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(gv[2 * j + 1])) << 16);
                }
                sA[buf][tc_off(o, 8 * h) >> 4] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            __syncthreads();      // srow complete
            for (int q = tid; q < 144 * 2; q += 256) {   // B: row n = c*9 + t, pixels 8h .. 8h + 7
                const int n = q >> 1, h = q & 1, c = n / 9, t = n % 9;
                const bf16* src = &srow[c][t / 3][8 * h + t % 3];
                uint32_t pk[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    pk[j] = (uint32_t)__bfloat16_as_ushort(src[2 * j]) | ((uint32_t)__bfloat16_as_ushort(src[2 * j + 1]) << 16);
                sB[buf][tc_off(n, 8 * h) >> 4] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (s_abort) { ok = false; break; }
            if (tid == 0) {
                tc_fence_after();
                umma_f16(taddr, smem_desc(smem_u32(&sA[buf][0]), 128, 256), smem_desc(smem_u32(&sB[buf][0]), 128, 256),
                         idesc, s > 0 ? 1u : 0u);
                umma_commit(&bar[buf]);
            }
        }
    }
    if (s > 0 && !mbar_wait_bounded(&bar[(s - 1) & 1], (unsigned)(((s - 1) >> 1) & 1))) {
        atomicOr(err, 16);
        ok = false;
    }
    tc_fence_after();
    if (ok && warp < 4) {
        const int o = 32 * warp + lane;
        for (int n0 = 0; n0 < 144; n0 += 16) {
            uint32_t v[16];
            __syncwarp();
            if (s > 0) {
                tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)n0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0u;
            }
            if (o0 + o < Cout) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + j, c = n / 9, t = n % 9;
                    if (c0 + c < Cin)
                        part[((long)blockIdx.z * Cout * Cin + (long)(o0 + o) * Cin + c0 + c) * 9 + t] =
                            __uint_as_float(v[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, 256);
}

// ---------------------------------------------------------------------------
// conv3x3 weight gradient, first stage: partial sums over a slice of the
// (batch, row) range for a 16 x 16 block of (output, input) channels.
//   gW[o][c][k] = sum_{b,y,x} gz[b][o][y][x] * in[b][c][y+ky-1][x+kx-1]
// with gz = gout * (a > 0) (a = the layer's post-ReLU output).  One thread
// per (o, c) pair keeps 9 sums; rows are streamed through shared memory.
// ---------------------------------------------------------------------------
template <typename TIN>
__global__ void __launch_bounds__(256) k_conv3_wgrad(const float* __restrict__ gout, long g_bs,
                                                     const bf16* __restrict__ act, long a_bs,
                                                     const TIN* __restrict__ in, long in_bs, int Cin,
                                                     int Cout, int H, int W, int B, int rows_per,
                                                     float* __restrict__ part) {
    constexpr int XT = 32;
    __shared__ float sg[16][XT];
    __shared__ float sx[16][3][XT + 2];
    const int tid = threadIdx.x, oc = tid >> 4, cc = tid & 15;
    const int nci = (Cin + 15) / 16;
    const int o0 = (blockIdx.x / nci) * 16, c0 = (blockIdx.x % nci) * 16;
    const long plane = (long)H * W;
    const long r_begin = (long)blockIdx.y * rows_per, r_end = min((long)B * H, r_begin + rows_per);
    float s[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) s[k] = 0.f;
    for (long br = r_begin; br < r_end; ++br) {
        const int b = (int)(br / H), y = (int)(br % H);
        for (int x0 = 0; x0 < W; x0 += XT) {
            __syncthreads();
            for (int e = tid; e < 16 * XT; e += 256) {
                const int o = e / XT, x = x0 + e % XT;
                float v = 0.f;
                if (o0 + o < Cout && x < W) {
                    const long off = (long)(o0 + o) * plane + (long)y * W + x;
                    v = gout[(long)b * g_bs + off];
                    if (act && !(__bfloat162float(act[(long)b * a_bs + off]) > 0.f)) v = 0.f;
                    v = __bfloat162float(__float2bfloat16_rn(v));   // gradients enter as BF16
                }
                sg[o][e % XT] = v;
            }
            for (int e = tid; e < 16 * 3 * (XT + 2); e += 256) {
                const int c = e / (3 * (XT + 2)), r = (e / (XT + 2)) % 3, xi = e % (XT + 2);
                const int yy = y - 1 + r, xx = x0 - 1 + xi;
                float v = 0.f;
                if (c0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < W)
                    v = ld(in + (long)b * in_bs + (long)(c0 + c) * plane + (long)yy * W + xx);
                sx[c][r][xi] = v;
            }
            __syncthreads();
            const int xn = min(XT, W - x0);
            for (int x = 0; x < xn; ++x) {
                const float gv = sg[oc][x];
#pragma unroll
                for (int k = 0; k < 9; ++k) s[k] = fmaf(gv, sx[cc][k / 3][x + k % 3], s[k]);
            }
        }
    }
    if (o0 + oc < Cout && c0 + cc < Cin) {
        float* p = part + ((long)blockIdx.y * Cout * Cin + (long)(o0 + oc) * Cin + c0 + cc) * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) p[k] = s[k];
    }
}

// Sum of the S partials in a fixed order (+= into g when accumulate).
__global__ void k_reduce_parts(const float* __restrict__ part, int S, long n, float* __restrict__ g) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = 0.f;
    for (int s = 0; s < S; ++s) v += part[(long)s * n + i];
    g[i] = v;
}

// Bias gradient (and the 1x1 layer's weight gradient when inp != nullptr):
// per output channel o (block), sums over (b, pixel) in a fixed order.
//   gb[o] = sum gz[b][o][p];   gW[o][c] = sum gz[b][o][p] * inp[b][c][p]
__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ gout, long g_bs,
                                                   const bf16* __restrict__ act, long a_bs, int B,
                                                   long plane, float* __restrict__ gb) {
    __shared__ float sh[256];
    const int o = blockIdx.x;
    float s = 0.f;
    for (int b = 0; b < B; ++b)
        for (long p = threadIdx.x; p < plane; p += 256) {
            const long off = (long)o * plane + p;
            float v = gout[(long)b * g_bs + off];
            if (act && !(__bfloat162float(act[(long)b * a_bs + off]) > 0.f)) v = 0.f;
            s += v;
        }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[o] = sh[0];
}

__global__ void __launch_bounds__(256) k_conv1_wgrad(const float* __restrict__ gout, int Cout,
                                                     const bf16* __restrict__ in, int Cin, int B,
                                                     long plane, float* __restrict__ gw) {
    __shared__ float sh[256];
    const int o = blockIdx.x / Cin, c = blockIdx.x % Cin;
    float s = 0.f;
    for (int b = 0; b < B; ++b)
        for (long p = threadIdx.x; p < plane; p += 256)
            s = fmaf(gout[((long)b * Cout + o) * plane + p],
                     __bfloat162float(in[((long)b * Cin + c) * plane + p]), s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gw[o * Cin + c] = sh[0];
}

// Final layer: out = xq + bias + W d0 (FP32), W [Cout][Cin] (BF16 copy).
__global__ void k_conv1_fwd(const bf16* __restrict__ d0, int Cin, const bf16* __restrict__ w,
                            const float* __restrict__ bias, const bf16* __restrict__ xq, int Cout,
                            long plane, int B, float* __restrict__ out) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)B * plane) return;
    const int b = (int)(i / plane);
    const long p = i % plane;
    for (int o = 0; o < Cout; ++o) {
        float v = bias[o];
        for (int c = 0; c < Cin; ++c)
            v = fmaf(__bfloat162float(w[o * Cin + c]), __bfloat162float(d0[((long)b * Cin + c) * plane + p]), v);
        const long off = ((long)b * Cout + o) * plane + p;
        out[off] = __bfloat162float(xq[off]) + v;
    }
}

// gd0[b][c][p] = sum_o W[o][c] gout[b][o][p]
__global__ void k_conv1_dgrad(const float* __restrict__ gout, int Cout, const bf16* __restrict__ w,
                              int Cin, long plane, int B, float* __restrict__ gd) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)B * plane) return;
    const int b = (int)(i / plane);
    const long p = i % plane;
    for (int c = 0; c < Cin; ++c) {
        float v = 0.f;
        for (int o = 0; o < Cout; ++o)
            v = fmaf(__bfloat162float(w[o * Cin + c]), gout[((long)b * Cout + o) * plane + p], v);
        gd[((long)b * Cin + c) * plane + p] = v;
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// maxpool 2x2: in view (bs_in), out contiguous [B][C][H/2][W/2]
__global__ void k_pool(const bf16* __restrict__ in, long in_bs, int C, int H, int W, int B,
                       bf16* __restrict__ out) {
    const int Ho = H / 2, Wo = W / 2;
    const long n = (long)B * C * Ho * Wo;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int xo = (int)(i % Wo), yo = (int)((i / Wo) % Ho), c = (int)((i / ((long)Wo * Ho)) % C);
    const int b = (int)(i / ((long)Wo * Ho * C));
    const bf16* p = in + (long)b * in_bs + (long)c * H * W + (long)(2 * yo) * W + 2 * xo;
    float m = __bfloat162float(p[0]);
    m = fmaxf(m, __bfloat162float(p[1]));
    m = fmaxf(m, __bfloat162float(p[W]));
    m = fmaxf(m, __bfloat162float(p[W + 1]));
    out[i] = __float2bfloat16_rn(m);
}

// gradient of the pooling (to the first maximum), plus an optional skip
// gradient: g_e = pool^T(gin) + skip, written as [B][C][H][W]
__global__ void k_pool_bwd(const bf16* __restrict__ e, long e_bs, const float* __restrict__ gin,
                           const float* __restrict__ skip, long skip_bs, int C, int H, int W, int B,
                           float* __restrict__ ge) {
    const int Ho = H / 2, Wo = W / 2;
    const long n = (long)B * C * Ho * Wo;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int xo = (int)(i % Wo), yo = (int)((i / Wo) % Ho), c = (int)((i / ((long)Wo * Ho)) % C);
    const int b = (int)(i / ((long)Wo * Ho * C));
    const bf16* p = e + (long)b * e_bs + (long)c * H * W + (long)(2 * yo) * W + 2 * xo;
    const float v[4] = {__bfloat162float(p[0]), __bfloat162float(p[1]), __bfloat162float(p[W]),
                        __bfloat162float(p[W + 1])};
    const float m = fmaxf(fmaxf(v[0], v[1]), fmaxf(v[2], v[3]));
    int first = 3;
    for (int k = 2; k >= 0; --k)
        if (v[k] == m) first = k;
    const float g = gin[i];
    for (int k = 0; k < 4; ++k) {
        const long off = (long)c * H * W + (long)(2 * yo + k / 2) * W + 2 * xo + k % 2;
        float s = k == first ? g : 0.f;
        if (skip) s += skip[(long)b * skip_bs + off];
        ge[(long)b * C * H * W + off] = s;
    }
}

// nearest upsampling of d [B][C][H/2][W/2] into channels 0..C-1 of a view
__global__ void k_up(const bf16* __restrict__ d, int C, int H, int W, int B, bf16* __restrict__ out,
                     long out_bs) {
    const long n = (long)B * C * H * W;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % W), y = (int)((i / W) % H), c = (int)((i / ((long)W * H)) % C);
    const int b = (int)(i / ((long)W * H * C));
    out[(long)b * out_bs + (long)c * H * W + (long)y * W + x] =
        d[(((long)b * C + c) * (H / 2) + y / 2) * (W / 2) + x / 2];
}

// gradient of the upsampling: sum of the 4 children (channels 0..C-1 of g)
__global__ void k_up_bwd(const float* __restrict__ g, long g_bs, int C, int H, int W, int B,
                         float* __restrict__ gd) {
    const int Ho = H / 2, Wo = W / 2;
    const long n = (long)B * C * Ho * Wo;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int xo = (int)(i % Wo), yo = (int)((i / Wo) % Ho), c = (int)((i / ((long)Wo * Ho)) % C);
    const int b = (int)(i / ((long)Wo * Ho * C));
    const float* p = g + (long)b * g_bs + (long)c * H * W + (long)(2 * yo) * W + 2 * xo;
    gd[i] = (p[0] + p[1]) + (p[W] + p[W + 1]);
}

// loss partials (FP64 per block) and dL/dout = 2 (out - t) / n
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ out, const float* __restrict__ t,
                                             long n, float* __restrict__ g, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (long i = (long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long)gridDim.x * 256) {
        const float d = out[i] - t[i];
        if (g) g[i] = 2.f * d / (float)n;
        s += (double)d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Adam on the FP32 master weights, then the BF16 copy used by the forward
// pass and the transposed, flipped BF16 copy used by the input gradient.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// wb = bf16(w) for a conv3 weight [O][C][9]; wt[c][o][8-k] = wb[o][c][k]
__global__ void k_pack_w(const float* __restrict__ w, int O, int C, int K, bf16* __restrict__ wb,
                         bf16* __restrict__ wt) {
    const long n = (long)O * C * K;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bf16 q = __float2bfloat16_rn(w[i]);
    wb[i] = q;
    if (wt) {
        const int k = (int)(i % K), c = (int)((i / K) % C), o = (int)(i / ((long)K * C));
        wt[((long)c * O + o) * K + (K - 1 - k)] = q;
    }
}

}  // namespace unet
}  // namespace tnlm

// ===========================================================================
// The network object and its C entry points.
// ===========================================================================
using namespace tnlm::unet;

namespace {

struct Layer {
    int cout, cin, k;
    long woff, boff;       // offsets in the flat parameter vector (floats)
};

long grid1(long n) { return (n + 255) / 256; }

}  // namespace

struct tnlm_unet {
    int device, in_ch, out_ch, base, levels;
    std::vector<Layer> layers;
    long nparam = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32 [nparam]
    tnlm::unet::bf16 *wb = nullptr, *wt = nullptr;                  // BF16 copies
    tnlm::unet::bf16* wtc = nullptr;                                // tensor-core packing of 3x3 layers
    std::vector<long> tcoff;                                        // per layer offset in wtc (-1: none)
    tnlm::unet::bf16* wtct = nullptr;                               // same for the input gradients
    std::vector<long> tcofft;
    int* derr = nullptr;                                            // device error flags
    int num_sms = 148;
    long adam_t = 0;
    // activations (BF16) and gradient scratch (FP32), sized for cap_pixels * batch
    long cap = 0;
    void* act = nullptr;
    float* scratch = nullptr;
    float* parts = nullptr;
    double* loss_part = nullptr;
    long part_cap = 0;
};

namespace {

thread_local char u_err[256];

tnlm_status ufail(tnlm_status s, const char* msg, cudaError_t e = cudaSuccess) {
    snprintf(u_err, sizeof(u_err), "%s%s%s", msg, e != cudaSuccess ? ": " : "",
             e != cudaSuccess ? cudaGetErrorString(e) : "");
    return s;
}

#define UCK(call, what)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return ufail(e_ == cudaErrorMemoryAllocation ? TNLM_ERR_OOM : TNLM_ERR_CUDA, what, e_); \
    } while (0)

// Buffers of one forward/backward pass for batch B at H x W.
struct Plan {
    int L, B, H, W;
    std::vector<int> c;                  // channels per level
    std::vector<long> hw;                // pixels per level
    // BF16 activations
    bf16* xq;                            // input [B][in][H][W]
    std::vector<bf16*> ain;              // pooled input of encoder level l>0 [B][c_{l-1}][hw_l]
    std::vector<bf16*> e1;               // encoder first conv output [B][c_l][hw_l]
    std::vector<bf16*> cat;              // decoder concat buffer of level l: [B][c_{l+1} + c_l][hw_l]; e_l lives at channel c_{l+1}
    std::vector<bf16*> eL;               // e_{L-1} [B][c_{L-1}][hw_{L-1}]
    std::vector<bf16*> d1, d2;           // decoder conv outputs [B][c_l][hw_l]
    float* out;                          // [B][out][H][W]
    long act_bytes;
};

long plan_sizes(const tnlm_unet* n, int B, int H, int W, Plan* P, char* base) {
    // lays out the BF16 activations (base may be nullptr to only measure)
    P->L = n->levels; P->B = B; P->H = H; P->W = W;
    P->c.assign(P->L, 0); P->hw.assign(P->L, 0);
    P->ain.assign(P->L, nullptr); P->e1.assign(P->L, nullptr); P->cat.assign(P->L, nullptr);
    P->d1.assign(P->L, nullptr); P->d2.assign(P->L, nullptr); P->eL.assign(1, nullptr);
    long off = 0;
    auto take = [&](long elems) -> bf16* {
        bf16* p = base ? (bf16*)(base + off) : nullptr;
        off += (elems * 2 + 255) / 256 * 256;
        return p;
    };
    for (int l = 0; l < P->L; ++l) {
        P->c[l] = n->base << l;
        P->hw[l] = (long)(H >> l) * (W >> l);
    }
    P->xq = take((long)B * n->in_ch * H * W);
    for (int l = 0; l < P->L; ++l) {
        if (l > 0) P->ain[l] = take((long)B * P->c[l - 1] * P->hw[l]);
        P->e1[l] = take((long)B * P->c[l] * P->hw[l]);
        if (l < P->L - 1) P->cat[l] = take((long)B * (P->c[l + 1] + P->c[l]) * P->hw[l]);
        else P->eL[0] = take((long)B * P->c[l] * P->hw[l]);
        if (l < P->L - 1) {
            P->d1[l] = take((long)B * P->c[l] * P->hw[l]);
            P->d2[l] = take((long)B * P->c[l] * P->hw[l]);
        }
    }
    P->act_bytes = off;
    return off;
}

// e_l as a view (pointer, batch stride)
bf16* e_ptr(const Plan& P, int l, long* bs) {
    if (l == P.L - 1) {
        *bs = (long)P.c[l] * P.hw[l];
        return P.eL[0];
    }
    *bs = (long)(P.c[l + 1] + P.c[l]) * P.hw[l];
    return P.cat[l] + (long)P.c[l + 1] * P.hw[l];
}

tnlm_status ensure_capacity(tnlm_unet* n, int B, int H, int W, Plan* P) {
    const long need = plan_sizes(n, B, H, W, P, nullptr);
    const long pix = (long)B * H * W;
    // FP32 gradient scratch: 4 buffers of the widest level-0 tensor
    const long widest = (long)(n->base * 3 > n->in_ch ? n->base * 3 : n->in_ch);
    const long sc = 4 * widest * pix + (long)B * n->out_ch * H * W;
    if (need > n->cap) {
        cudaFree(n->act);
        cudaFree(n->scratch);
        n->act = nullptr;
        n->scratch = nullptr;
        UCK(cudaMalloc(&n->act, need), "activation buffers");
        UCK(cudaMalloc(&n->scratch, sizeof(float) * sc), "gradient buffers");
        n->cap = need;
    }
    plan_sizes(n, B, H, W, P, (char*)n->act);
    P->out = n->scratch + 4 * widest * pix;
    return TNLM_OK;
}

template <typename TIN, bool OB, bool RELU>
void conv3(const TIN* in, long in_bs, int Cin, const bf16* mask, long mask_bs, const bf16* w,
           const float* bias, void* out, long out_bs, int Cout, int H, int W, int B, cudaStream_t st) {
    dim3 grid((W + kCT - 1) / kCT, (H + kCT - 1) / kCT, B * ((Cout + kCO - 1) / kCO));
    k_conv3<TIN, OB, RELU><<<grid, 128, 0, st>>>(in, in_bs, Cin, mask, mask_bs, w, bias, out, out_bs,
                                                 Cout, H, W);
}

// Output channels per CTA of the tensor-core convolution: 64 (32 when the
// count is not a multiple of 64, or when 64 would not fill twice the SMs);
// with three taps per step double-buffered this keeps the static shared
// memory under 48 KB.
int tc_n_tile(int cout, int ctas, int sms) {
    int nt = cout % 64 == 0 ? 64 : 32;
    if (nt == 64 && (long)ctas * (cout / 64) < 2L * sms) nt = 32;
    return nt;
}

template <int MODE>
bool tc_launch(int nt, dim3 grid, cudaStream_t st, const void* in, long in_bs, int cin, const bf16* mask, long m_bs,
               const uint4* wp, const float* bias, void* out, long out_bs, int H, int W, int tx, int cout, int* err) {
    switch (nt) {
        case 32: k_conv3_tc<32, MODE><<<grid, 256, 0, st>>>(in, in_bs, cin, mask, m_bs, wp, bias, out, out_bs, H, W, tx, cout, err); return true;
        case 64: k_conv3_tc<64, MODE><<<grid, 256, 0, st>>>(in, in_bs, cin, mask, m_bs, wp, bias, out, out_bs, H, W, tx, cout, err); return true;
        default: return false;
    }
}

// Forward 3x3 layer: the tensor-core kernel for 32/64/128/256 output
// channels, the CUDA-core one otherwise.
void conv3_fwd(tnlm_unet* n, int li, const bf16* in, long in_bs, int Cin, bf16* out, long out_bs, int Cout,
               int H, int W, int B, cudaStream_t st) {
    const Layer& Ly = n->layers[li];
    const long to = n->tcoff[li];
    if (to >= 0) {
        const int tx = (W + kTcvTW - 1) / kTcvTW, ty = (H + kTcvTH - 1) / kTcvTH;
        const int nt = tc_n_tile(Cout, tx * ty * B, n->num_sms);
        dim3 grid(tx * ty, B, Cout / nt);
        const uint4* wp = (const uint4*)(n->wtc + to);
        if (tc_launch<0>(nt, grid, st, in, in_bs, Cin, nullptr, 0, wp, n->w + Ly.boff, out, out_bs, H, W, tx, Cout,
                         n->derr))
            return;
    }
    conv3<bf16, true, true>(in, in_bs, Cin, nullptr, 0, n->wb + Ly.woff, n->w + Ly.boff, out, out_bs, Cout, H, W, B, st);
}

// Input gradient of 3x3 layer li: g (FP32, the layer's Cout channels, times
// the mask) -> out (FP32, the layer's Cin channels).  Tensor cores when the
// layer's Cin is 32/64/96/128/192/256, else the CUDA-core kernel.
void conv3_dgrad(tnlm_unet* n, int li, const float* g, long g_bs, const bf16* mask, long m_bs, float* out,
                 long out_bs, int H, int W, int B, cudaStream_t st) {
    const Layer& Ly = n->layers[li];
    const long to = n->tcofft[li];
    if (to >= 0) {
        const int tx = (W + kTcvTW - 1) / kTcvTW, ty = (H + kTcvTH - 1) / kTcvTH;
        const int nt = tc_n_tile(Ly.cin, tx * ty * B, n->num_sms);
        dim3 grid(tx * ty, B, Ly.cin / nt);
        const uint4* wp = (const uint4*)(n->wtct + to);
        if (tc_launch<1>(nt, grid, st, g, g_bs, Ly.cout, mask, m_bs, wp, nullptr, out, out_bs, H, W, tx, Ly.cin,
                         n->derr))
            return;
    }
    conv3<float, false, false>(g, g_bs, Ly.cout, mask, m_bs, n->wt + Ly.woff, nullptr, out, out_bs, Ly.cin, H, W, B, st);
}

tnlm_status forward(tnlm_unet* n, const float* x, const Plan& P, cudaStream_t st) {
    const int L = P.L, B = P.B;
    const long n0 = (long)B * n->in_ch * P.H * P.W;
    k_to_bf16<<<grid1(n0), 256, 0, st>>>(x, P.xq, n0);
    int li = 0;
    for (int l = 0; l < L; ++l) {
        const int H = P.H >> l, W = P.W >> l;
        const bf16* in;
        long in_bs;
        int cin;
        if (l == 0) {
            in = P.xq; in_bs = (long)n->in_ch * P.hw[0]; cin = n->in_ch;
        } else {
            long ebs;
            const bf16* ep = e_ptr(P, l - 1, &ebs);
            const long np = (long)B * P.c[l - 1] * P.hw[l];
            k_pool<<<grid1(np), 256, 0, st>>>(ep, ebs, P.c[l - 1], H * 2, W * 2, B, P.ain[l]);
            in = P.ain[l]; in_bs = (long)P.c[l - 1] * P.hw[l]; cin = P.c[l - 1];
        }
        conv3_fwd(n, li++, in, in_bs, cin, P.e1[l], (long)P.c[l] * P.hw[l], P.c[l], H, W, B, st);
        long ebs;
        bf16* ep = e_ptr(P, l, &ebs);
        conv3_fwd(n, li++, P.e1[l], (long)P.c[l] * P.hw[l], P.c[l], ep, ebs, P.c[l], H, W, B, st);
    }
    const bf16* d = P.eL[0];
    for (int l = L - 2; l >= 0; --l) {
        const int H = P.H >> l, W = P.W >> l;
        const long cbs = (long)(P.c[l + 1] + P.c[l]) * P.hw[l];
        const long nu = (long)B * P.c[l + 1] * P.hw[l];
        k_up<<<grid1(nu), 256, 0, st>>>(d, P.c[l + 1], H, W, B, P.cat[l], cbs);
        conv3_fwd(n, li++, P.cat[l], cbs, P.c[l + 1] + P.c[l], P.d1[l], (long)P.c[l] * P.hw[l], P.c[l], H, W, B, st);
        conv3_fwd(n, li++, P.d1[l], (long)P.c[l] * P.hw[l], P.c[l], P.d2[l], (long)P.c[l] * P.hw[l], P.c[l], H, W,
                  B, st);
        d = P.d2[l];
    }
    const Layer& f = n->layers[li];
    const long pix = (long)B * P.hw[0];
    k_conv1_fwd<<<grid1(pix), 256, 0, st>>>(d, P.c[0], n->wb + f.woff, n->w + f.boff, P.xq, n->out_ch,
                                            P.hw[0], B, P.out);
    UCK(cudaGetLastError(), "forward launch");
    return TNLM_OK;
}

// weight + bias gradients of one conv3 layer (gz = gout * (act > 0))
template <typename TIN>
tnlm_status conv3_param_grads(tnlm_unet* n, const Layer& Ly, const float* gout, long g_bs,
                              const bf16* act, long a_bs, const TIN* in, long in_bs, int H, int W, int B,
                              cudaStream_t st) {
    const long rows = (long)B * H;
    const bool tc = sizeof(TIN) == 2 && W % 16 == 0;
    // row slices: the tensor-core kernel gets enough CTAs for ~4 per SM
    long S = rows < 64 ? rows : 64;
    if (tc) {
        const long per = (long)((Ly.cin + 15) / 16) * ((Ly.cout + 127) / 128);
        S = (4L * n->num_sms + per - 1) / per;
        S = S < 1 ? 1 : (S > rows ? rows : S);
    }
    const int rows_per = (int)((rows + S - 1) / S);
    S = (rows + rows_per - 1) / rows_per;
    const long nw = (long)Ly.cout * Ly.cin * 9;
    if ((long)S * nw > n->part_cap) {
        cudaFree(n->parts);
        n->parts = nullptr;
        UCK(cudaMalloc(&n->parts, sizeof(float) * S * nw), "gradient partials");
        n->part_cap = (long)S * nw;
    }
    if (tc) {
        dim3 grid((Ly.cin + 15) / 16, (Ly.cout + 127) / 128, (unsigned)S);
        k_conv3_wgrad_tc<<<grid, 256, 0, st>>>(gout, g_bs, act, a_bs, (const bf16*)in, in_bs, Ly.cin, Ly.cout, H,
                                               W, B, rows_per, n->parts, n->derr);
    } else {
        const int blocks = ((Ly.cout + 15) / 16) * ((Ly.cin + 15) / 16);
        k_conv3_wgrad<TIN><<<dim3(blocks, (unsigned)S), 256, 0, st>>>(gout, g_bs, act, a_bs, in, in_bs, Ly.cin, Ly.cout,
                                                            H, W, B, rows_per, n->parts);
    }
    k_reduce_parts<<<grid1(nw), 256, 0, st>>>(n->parts, (int)S, nw, n->g + Ly.woff);
    k_bias_grad<<<Ly.cout, 256, 0, st>>>(gout, g_bs, act, a_bs, B, (long)H * W, n->g + Ly.boff);
    UCK(cudaGetLastError(), "gradient launch");
    return TNLM_OK;
}

tnlm_status backward(tnlm_unet* n, const Plan& P, const float* gout_final, cudaStream_t st) {
    const int L = P.L, B = P.B;
    const long pix0 = (long)B * P.hw[0];
    const long widest = (long)(n->base * 3 > n->in_ch ? n->base * 3 : n->in_ch);
    // four FP32 buffers of widest x pix0: S0 and the first half of S2 rotate
    // the running gradient, S1 holds level 0's concatenation gradient, the
    // second half of S2 and S3 hold those of the deeper levels
    float* S0 = n->scratch;
    float* S1 = S0 + widest * pix0;
    float* S2 = S1 + widest * pix0;
    int li = (int)n->layers.size() - 1;
    // final 1x1: dW, db, gd0 -> S0 [B][c0][hw0]
    const Layer& f = n->layers[li--];
    const bf16* d0 = L > 1 ? P.d2[0] : P.eL[0];
    k_conv1_wgrad<<<f.cout * f.cin, 256, 0, st>>>(gout_final, n->out_ch, d0, P.c[0], B, P.hw[0],
                                                  n->g + f.woff);
    k_bias_grad<<<f.cout, 256, 0, st>>>(gout_final, (long)n->out_ch * P.hw[0], nullptr, 0, B, P.hw[0],
                                        n->g + f.boff);
    k_conv1_dgrad<<<grid1(pix0), 256, 0, st>>>(gout_final, n->out_ch, n->wb + f.woff, P.c[0], P.hw[0], B, S0);
    float* g = S0;          // gradient w.r.t. the current decoder output (post-ReLU value)
    // skip gradients of e_l: kept in S3 region? They are needed later, so give
    // them their own storage: the concat gradient of level l stays in a
    // buffer until the encoder pass (we keep one per level below)
    std::vector<float*> skipg(L, nullptr);
    std::vector<long> skipbs(L, 0);
    // the concat gradients are produced level 0 first (largest); keep them in
    // S1 (level 0) and in freshly carved space of S2/S3 for deeper levels
    float* carve = S2 + widest * pix0 / 2;
    for (int l = 0; l <= L - 2; ++l) {
        const int H = P.H >> l, W = P.W >> l;
        const long hw = P.hw[l];
        const int cl = P.c[l], cu = P.c[l + 1];
        const int ib = li--, ia = li--;
        const Layer& b = n->layers[ib];
        const Layer& a = n->layers[ia];
        // conv b: input d1, output d2 (mask d2)
        tnlm_status s = conv3_param_grads<bf16>(n, b, g, (long)cl * hw, P.d2[l], (long)cl * hw, P.d1[l],
                                                (long)cl * hw, H, W, B, st);
        if (s != TNLM_OK) return s;
        float* gd1 = (g == S0) ? S2 : S0;
        conv3_dgrad(n, ib, g, (long)cl * hw, P.d2[l], (long)cl * hw, gd1, (long)cl * hw, H, W, B, st);
        // conv a: input concat, output d1 (mask d1)
        s = conv3_param_grads<bf16>(n, a, gd1, (long)cl * hw, P.d1[l], (long)cl * hw, P.cat[l],
                                    (long)(cu + cl) * hw, H, W, B, st);
        if (s != TNLM_OK) return s;
        float* gc = (l == 0) ? S1 : carve;
        const long gcbs = (long)(cu + cl) * hw;
        conv3_dgrad(n, ia, gd1, (long)cl * hw, P.d1[l], (long)cl * hw, gc, gcbs, H, W, B, st);
        skipg[l] = gc + (long)cu * hw;
        skipbs[l] = gcbs;
        if (l > 0) carve += (long)B * (cu + cl) * hw;
        // gradient of d_{l+1}: up^T of the first cu channels
        float* gn = (gd1 == S0) ? S2 : S0;
        if (l == 0) gn = S0 == g ? S2 : S0;
        const long nd = (long)B * cu * P.hw[l + 1];
        k_up_bwd<<<grid1(nd), 256, 0, st>>>(gc, gcbs, cu, H, W, B, gn);
        g = gn;
    }
    // encoder, deepest first; g = gradient w.r.t. e_l (post-ReLU)
    for (int l = L - 1; l >= 0; --l) {
        const int H = P.H >> l, W = P.W >> l;
        const long hw = P.hw[l];
        const int cl = P.c[l];
        const int ib = li--, ia = li--;
        const Layer& b = n->layers[ib];
        const Layer& a = n->layers[ia];
        long ebs;
        const bf16* ep = e_ptr(P, l, &ebs);
        // conv b: input e1, output e (mask e)
        tnlm_status s = conv3_param_grads<bf16>(n, b, g, (long)cl * hw, ep, ebs, P.e1[l], (long)cl * hw, H, W,
                                                B, st);
        if (s != TNLM_OK) return s;
        float* ge1 = (g == S0) ? S2 : S0;
        conv3_dgrad(n, ib, g, (long)cl * hw, ep, ebs, ge1, (long)cl * hw, H, W, B, st);
        // conv a: input x (level 0) or pooled e_{l-1}, output e1 (mask e1)
        const bf16* in = l == 0 ? P.xq : P.ain[l];
        const int cin = l == 0 ? n->in_ch : P.c[l - 1];
        s = conv3_param_grads<bf16>(n, a, ge1, (long)cl * hw, P.e1[l], (long)cl * hw, in, (long)cin * hw, H,
                                    W, B, st);
        if (s != TNLM_OK) return s;
        if (l == 0) break;
        float* gin = (ge1 == S0) ? S2 : S0;
        conv3_dgrad(n, ia, ge1, (long)cl * hw, P.e1[l], (long)cl * hw, gin, (long)cin * hw, H, W, B, st);
        // gradient of e_{l-1}: pool^T(gin) + its skip gradient
        long pbs;
        const bf16* pe = e_ptr(P, l - 1, &pbs);
        float* gprev = (gin == S0) ? S2 : S0;
        const long np = (long)B * cin * hw;
        k_pool_bwd<<<grid1(np), 256, 0, st>>>(pe, pbs, gin, skipg[l - 1], skipbs[l - 1], cin, H * 2, W * 2, B,
                                              gprev);
        g = gprev;
    }
    UCK(cudaGetLastError(), "backward launch");
    return TNLM_OK;
}

tnlm_status repack(tnlm_unet* n, cudaStream_t st) {
    for (size_t i = 0; i < n->layers.size(); ++i) {
        const Layer& Ly = n->layers[i];
        const long nw = (long)Ly.cout * Ly.cin * Ly.k * Ly.k;
        k_pack_w<<<grid1(nw), 256, 0, st>>>(n->w + Ly.woff, Ly.cout, Ly.cin, Ly.k * Ly.k, n->wb + Ly.woff,
                                            Ly.k == 3 ? n->wt + Ly.woff : nullptr);
        if (n->tcoff[i] >= 0) {
            const long np = 9L * ((Ly.cin + 15) / 16) * Ly.cout * 16;
            k_pack_tc<<<grid1(np), 256, 0, st>>>(n->w + Ly.woff, Ly.cout, Ly.cin, n->wtc + n->tcoff[i]);
        }
        if (n->tcofft[i] >= 0) {
            const long np = 9L * ((Ly.cout + 15) / 16) * Ly.cin * 16;
            k_pack_tc_t<<<grid1(np), 256, 0, st>>>(n->w + Ly.woff, Ly.cout, Ly.cin, n->wtct + n->tcofft[i]);
        }
    }
    UCK(cudaGetLastError(), "weight packing");
    return TNLM_OK;
}

bool shape_ok(const tnlm_unet* n, int B, int H, int W) {
    const int q = 1 << (n->levels - 1);
    return B >= 1 && H >= q && W >= q && H % q == 0 && W % q == 0 && (long)B * H * W <= (1L << 28);
}

}  // namespace

extern "C" {

const char* tnlm_unet_last_error(void) { return u_err; }

tnlm_status tnlm_unet_create(int in_ch, int out_ch, int base, int levels, int device, tnlm_unet** out) {
    u_err[0] = 0;
    if (!out) return ufail(TNLM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (in_ch < 1 || out_ch < 1 || base < 1 || levels < 1 || levels > 8 || (base << (levels - 1)) > 4096)
        return ufail(TNLM_ERR_INVALID_ARG, "bad network shape");
    if (in_ch != out_ch) return ufail(TNLM_ERR_INVALID_ARG, "the residual output needs in_ch == out_ch");
    if (cudaSetDevice(device) != cudaSuccess) return ufail(TNLM_ERR_INVALID_ARG, "device not available");
    tnlm_unet* n = new tnlm_unet();
    n->device = device; n->in_ch = in_ch; n->out_ch = out_ch; n->base = base; n->levels = levels;
    cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, device);
    long off = 0;
    auto add = [&](int co, int ci, int k) {
        Layer Ly{co, ci, k, off, off + (long)co * ci * k * k};
        off = Ly.boff + co;
        n->layers.push_back(Ly);
    };
    int cin = in_ch;
    for (int l = 0; l < levels; ++l) {
        add(base << l, cin, 3);
        add(base << l, base << l, 3);
        cin = base << l;
    }
    for (int l = levels - 2; l >= 0; --l) {
        add(base << l, (base << (l + 1)) + (base << l), 3);
        add(base << l, base << l, 3);
    }
    add(out_ch, base, 1);
    n->nparam = off;
    cudaError_t e = cudaMalloc(&n->w, sizeof(float) * off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->wb, sizeof(bf16) * off * 2);
    if (e != cudaSuccess) {
        cudaFree(n->w);
        delete n;
        return ufail(TNLM_ERR_OOM, "parameter buffers", e);
    }
    n->g = n->w + off; n->m = n->g + off; n->v = n->m + off;
    n->wt = n->wb + off;
    long tco = 0, tcot = 0;
    for (const Layer& Ly : n->layers) {
        const bool tc = Ly.k == 3 && (Ly.cout == 32 || Ly.cout == 64 || Ly.cout == 128 || Ly.cout == 256);
        n->tcoff.push_back(tc ? tco : -1);
        if (tc) tco += 9L * ((Ly.cin + 15) / 16) * Ly.cout * 16;
        const bool tt = Ly.k == 3 && (Ly.cin == 32 || Ly.cin == 64 || Ly.cin == 96 || Ly.cin == 128 ||
                                      Ly.cin == 192 || Ly.cin == 256);
        n->tcofft.push_back(tt ? tcot : -1);
        if (tt) tcot += 9L * ((Ly.cout + 15) / 16) * Ly.cin * 16;
    }
    e = cudaMalloc(&n->wtc, sizeof(bf16) * (tco > 0 ? tco : 1));
    if (e == cudaSuccess) e = cudaMalloc(&n->wtct, sizeof(bf16) * (tcot > 0 ? tcot : 1));
    if (e == cudaSuccess) e = cudaMalloc(&n->derr, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(n->w); cudaFree(n->wb); cudaFree(n->wtc); cudaFree(n->wtct);
        delete n;
        return ufail(TNLM_ERR_OOM, "parameter buffers", e);
    }
    cudaMemset(n->wtc, 0, sizeof(bf16) * (tco > 0 ? tco : 1));
    cudaMemset(n->wtct, 0, sizeof(bf16) * (tcot > 0 ? tcot : 1));
    cudaMemset(n->derr, 0, sizeof(int));
    cudaMemset(n->w, 0, sizeof(float) * off * 4);
    cudaMemset(n->wb, 0, sizeof(bf16) * off * 2);
    *out = n;
    return TNLM_OK;
}

void tnlm_unet_destroy(tnlm_unet* n) {
    if (!n) return;
    cudaSetDevice(n->device);
    cudaDeviceSynchronize();
    cudaFree(n->w); cudaFree(n->wb); cudaFree(n->wtc); cudaFree(n->wtct); cudaFree(n->derr); cudaFree(n->act);
    cudaFree(n->scratch); cudaFree(n->parts);
    cudaFree(n->loss_part);
    delete n;
}

long long tnlm_unet_param_count(const tnlm_unet* n) { return n ? n->nparam : 0; }

tnlm_status tnlm_unet_set_params(tnlm_unet* n, const float* h_params) {
    u_err[0] = 0;
    if (!n || !h_params) return ufail(TNLM_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(n->device);
    UCK(cudaMemcpy(n->w, h_params, sizeof(float) * n->nparam, cudaMemcpyHostToDevice), "upload");
    UCK(cudaMemset(n->m, 0, sizeof(float) * n->nparam * 2), "reset moments");
    n->adam_t = 0;
    tnlm_status s = repack(n, 0);
    if (s != TNLM_OK) return s;
    UCK(cudaDeviceSynchronize(), "sync");
    return TNLM_OK;
}

tnlm_status tnlm_unet_get_params(const tnlm_unet* n, float* h_params, float* h_grads) {
    u_err[0] = 0;
    if (!n) return ufail(TNLM_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(n->device);
    UCK(cudaDeviceSynchronize(), "sync");
    if (h_params) UCK(cudaMemcpy(h_params, n->w, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost), "download");
    if (h_grads) UCK(cudaMemcpy(h_grads, n->g, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost), "download");
    return TNLM_OK;
}

tnlm_status tnlm_unet_forward(tnlm_unet* n, const float* d_x, float* d_out, int batch, int h, int w,
                              void* stream) {
    u_err[0] = 0;
    if (!n || !d_x || !d_out) return ufail(TNLM_ERR_INVALID_ARG, "NULL argument");
    if (!shape_ok(n, batch, h, w)) return ufail(TNLM_ERR_INVALID_ARG, "sizes must be multiples of 2^(levels-1)");
    cudaSetDevice(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    tnlm_status s = ensure_capacity(n, batch, h, w, &P);
    if (s != TNLM_OK) return s;
    s = forward(n, d_x, P, st);
    if (s != TNLM_OK) return s;
    UCK(cudaMemcpyAsync(d_out, P.out, sizeof(float) * batch * n->out_ch * h * w, cudaMemcpyDeviceToDevice, st),
        "output copy");
    return TNLM_OK;
}

tnlm_status tnlm_unet_grads(tnlm_unet* n, const float* d_x, const float* d_target, int batch, int h, int w,
                            double* loss, void* stream) {
    u_err[0] = 0;
    if (!n || !d_x || !d_target) return ufail(TNLM_ERR_INVALID_ARG, "NULL argument");
    if (!shape_ok(n, batch, h, w)) return ufail(TNLM_ERR_INVALID_ARG, "sizes must be multiples of 2^(levels-1)");
    cudaSetDevice(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    tnlm_status s = ensure_capacity(n, batch, h, w, &P);
    if (s != TNLM_OK) return s;
    s = forward(n, d_x, P, st);
    if (s != TNLM_OK) return s;
    const long no = (long)batch * n->out_ch * h * w;
    const int nb = 256;
    if (!n->loss_part) UCK(cudaMalloc(&n->loss_part, sizeof(double) * nb), "loss partials");
    // dL/dout overwrites the output buffer in place (out is not needed afterwards)
    float* gout = P.out;
    k_mse<<<nb, 256, 0, st>>>(P.out, d_target, no, gout, n->loss_part);
    s = backward(n, P, gout, st);
    if (s != TNLM_OK) return s;
    if (loss) {
        std::vector<double> hp(nb);
        UCK(cudaMemcpyAsync(hp.data(), n->loss_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, st), "loss");
        UCK(cudaStreamSynchronize(st), "sync");
        double t = 0.0;
        for (double v : hp) t += v;
        *loss = t / (double)no;
        int err = 0;
        UCK(cudaMemcpy(&err, n->derr, sizeof(int), cudaMemcpyDeviceToHost), "error flags");
        if (err) {
            cudaMemset(n->derr, 0, sizeof(int));
            return ufail(TNLM_ERR_TIMEOUT, "a tensor-core wait timed out");
        }
    }
    return TNLM_OK;
}

tnlm_status tnlm_unet_adam_step(tnlm_unet* n, float lr, float beta1, float beta2, float eps, void* stream) {
    u_err[0] = 0;
    if (!n) return ufail(TNLM_ERR_INVALID_ARG, "NULL argument");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return ufail(TNLM_ERR_INVALID_ARG, "bad Adam constants");
    cudaSetDevice(n->device);
    cudaStream_t st = (cudaStream_t)stream;
    n->adam_t++;
    const float c1 = 1.f - powf(beta1, (float)n->adam_t), c2 = 1.f - powf(beta2, (float)n->adam_t);
    k_adam<<<grid1(n->nparam), 256, 0, st>>>(n->w, n->g, n->m, n->v, n->nparam, lr, beta1, beta2, eps, c1, c2);
    return repack(n, st);
}

}  // extern "C"
