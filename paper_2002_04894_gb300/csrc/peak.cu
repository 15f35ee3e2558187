// Arithmetic-pipe microbenchmarks: the peaks that the rooflines of the
// evaluation kernels divide by (the near field is bound by the FP32 pipe in
// the mixed form and by the FP64 pipe in the plain form; its reciprocal
// square roots run on the XU pipe). Each kernel keeps independent chains of
// one instruction per thread, enough of them to cover the pipe's latency,
// on a grid of whole multiples of the SM count, and is timed with CUDA events
// on the caller's stream after one untimed launch.

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

__device__ float g_peak_sink_f;
__device__ double g_peak_sink_d;

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 4;

// 16 chains of FFMA per thread: 32 flop per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(int64_t iters, float a, float b) {
    float c[16];
#pragma unroll
    for (int k = 0; k < 16; k++) c[k] = (float)(threadIdx.x + k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 16; k++) c[k] = fmaf(c[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 16; k++) s += c[k];
    if (s == -1.2345f) g_peak_sink_f = s;  // never true for these inputs; keeps the chains live
}

// 8 chains of packed FFMA2 per thread: 32 flop per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(int64_t iters, float a, float b) {
    float2 c[8];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < 8; k++) c[k] = make_float2((float)(threadIdx.x + k), (float)k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) c[k] = __ffma2_rn(c[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += c[k].x + c[k].y;
    if (s == -1.2345f) g_peak_sink_f = s;
}

// 8 chains of DFMA per thread: 16 flop per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(int64_t iters, double a, double b) {
    double c[8];
#pragma unroll
    for (int k = 0; k < 8; k++) c[k] = (double)(threadIdx.x + k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) c[k] = fma(c[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += c[k];
    if (s == -1.2345) g_peak_sink_d = s;
}

// 8 chains of rsqrt.approx.ftz (XU pipe) per thread, each fed by an FADD:
// 8 reciprocal square roots per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_rsqrt(int64_t iters, float b) {
    float c[8];
#pragma unroll
    for (int k = 0; k < 8; k++) c[k] = 1.0f + (float)(threadIdx.x + k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            float r;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(c[k] + b));
            c[k] = r;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += c[k];
    if (s == -1.2345f) g_peak_sink_f = s;
}

}  // namespace

}  // namespace fmm

extern "C" int fmm_measure_peak(int kind, int64_t iters, void *stream, double *ops_per_s, double *ms) {
    using namespace fmm;
    if (!ops_per_s || iters < 1 || kind < 0 || kind > 3) return FMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = sm_count() * kPeakBlocksPerSM;
    const double per_iter[4] = {32.0, 32.0, 16.0, 8.0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto launch = [&](int64_t it) {
        switch (kind) {
            case 0: FMM_LAUNCH(k_peak_ffma, grid, kPeakThreads, 0, st, it, 0.999f, 1e-3f); break;
            case 1: FMM_LAUNCH(k_peak_ffma2, grid, kPeakThreads, 0, st, it, 0.999f, 1e-3f); break;
            case 2: FMM_LAUNCH(k_peak_dfma, grid, kPeakThreads, 0, st, it, 0.999, 1e-3); break;
            default: FMM_LAUNCH(k_peak_rsqrt, grid, kPeakThreads, 0, st, it, 0.5f); break;
        }
    };
    float t = 0.f;
    if (e == cudaSuccess) {
        launch(std::max<int64_t>(iters / 8, 1));  // untimed: clocks up, code loaded
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) launch(iters);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e);
    const double ops = (double)grid * kPeakThreads * (double)iters * per_iter[kind];
    *ops_per_s = ops / (t * 1e-3);
    if (ms) *ms = t;
    return FMM_OK;
}
