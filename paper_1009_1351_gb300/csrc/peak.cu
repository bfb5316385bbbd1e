// Microbenchmarks of the two arithmetic pipes the projector pair and the
// sweep use: FP32 fused multiply-add issue (the roofline denominator of the
// ALU-bound projector and backprojector, an FMA counted as one operation)
// and the ex2.approx special-function unit.  Each thread runs 8 independent
// dependency chains so that the pipes, not the latencies, set the rate; the
// grid holds 8 blocks of 256 threads per SM.
#include "internal.cuh"

namespace tnlm {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(float* out, int iters, float a, float b) {
    float x[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) x[j] = fmaf(x[j], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += x[j];
    out[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(float* out, int iters, float a) {
    float x[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) x[j] = ex2_approx(x[j] * a);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += x[j];
    out[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

}  // namespace tnlm

using namespace tnlm;

extern "C" tnlm_status tnlm_measure_peaks(int device, double* fp32_ops, double* ex2_ops) {
    if (!fp32_ops && !ex2_ops) return TNLM_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = 8 * (sms > 0 ? sms : 1);
    float* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * blocks * kPeakThreads);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int iters = 4096;
    const double per_launch = (double)blocks * kPeakThreads * iters * kPeakUnroll * kPeakChains;
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        double* dst = which == 0 ? fp32_ops : ex2_ops;
        if (!dst) continue;
        float best = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first is a warm-up
            e = cudaEventRecord(e0, st);
            if (which == 0) k_peak_fma<<<blocks, kPeakThreads, 0, st>>>(out, iters, 0.999f, 1e-3f);
            else k_peak_ex2<<<blocks, kPeakThreads, 0, st>>>(out, iters, 0.125f);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
        }
        if (e == cudaSuccess) *dst = per_launch / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (prev >= 0) cudaSetDevice(prev);
    return e == cudaSuccess ? TNLM_OK : (e == cudaErrorMemoryAllocation ? TNLM_ERR_OOM : TNLM_ERR_CUDA);
}
