// Microbenchmarks of the device's own peaks: the denominators of the
// roofline fractions reported for the kernels bound by FP32 / FP64
// arithmetic and by HBM.
//
// k_fma_f32    independent FP32 FMA chains per thread (scalar FFMA)
// k_fma_f32x2  the same with paired FP32 instructions (FFMA2 on float2)
// k_fma_f64    independent FP64 FMA chains
// k_copy       float4 grid-stride copy of a buffer far larger than L2
//
// Each arithmetic kernel keeps CH chains of x = x * a + b in registers
// (|a| < 1, so the values stay bounded), runs enough warps per SM to cover
// the FMA latency, and stores its chains only under a condition that never
// holds for the values used, so no chain is removed.
#include <cuda_runtime.h>

#include "internal.h"

namespace sfoc {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kUnroll = 16;

template <int CH>
__global__ void __launch_bounds__(kPeakThreads) k_fma_f32(float* __restrict__ sink, int iters, float a, float b) {
    float x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
#pragma unroll
            for (int i = 0; i < CH; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void __launch_bounds__(kPeakThreads) k_fma_f32x2(float* __restrict__ sink, int iters, float a, float b) {
    float2 x[CH];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i * 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
#pragma unroll
            for (int i = 0; i < CH; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i].x + x[i].y;
    if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void __launch_bounds__(kPeakThreads) k_fma_f64(double* __restrict__ sink, int iters, double a, double b) {
    double x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
#pragma unroll
            for (int i = 0; i < CH; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    if (s == -1.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_copy(const float4* __restrict__ src, float4* __restrict__ dst,
                                                       size_t n4) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// best (shortest) of `reps` timed launches after one warm-up, in ms
template <typename F>
cudaError_t best_ms(F launch, cudaStream_t st, int reps, float* out) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    if (e == cudaSuccess) {
        launch();
        e = cudaGetLastError();
    }
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *out = best;
    return e;
}

}  // namespace

cudaError_t measure_peaks(cudaStream_t st, int sms, double* fp32, double* fp32x2, double* fp64, double* hbm) {
    constexpr int CH = 8;
    const int blocks = sms * 8;                          // 64 warps per SM
    const double threads = (double)blocks * kPeakThreads;
    float* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(double) * (size_t)blocks * kPeakThreads);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    const int it32 = 4096, it64 = 64;
    e = best_ms([&] { k_fma_f32<CH><<<blocks, kPeakThreads, 0, st>>>(sink, it32, 0.999f, 1e-4f); }, st, 5, &ms);
    if (e == cudaSuccess) *fp32 = 2.0 * threads * CH * kUnroll * it32 / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess)
        e = best_ms([&] { k_fma_f32x2<CH><<<blocks, kPeakThreads, 0, st>>>(sink, it32 / 2, 0.999f, 1e-4f); }, st, 5,
                    &ms);
    if (e == cudaSuccess) *fp32x2 = 4.0 * threads * CH * kUnroll * (it32 / 2) / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess)
        e = best_ms([&] { k_fma_f64<CH><<<blocks, kPeakThreads, 0, st>>>((double*)sink, it64, 0.999, 1e-4); }, st,
                    5, &ms);
    if (e == cudaSuccess) *fp64 = 2.0 * threads * CH * kUnroll * it64 / (ms * 1e-3) / 1e12;
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    // HBM: 2 x 1 GiB, read once and written once per launch
    const size_t bytes = (size_t)1 << 30;
    float4 *a = nullptr, *b = nullptr;
    e = cudaMalloc(&a, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, bytes, st);
    if (e == cudaSuccess)
        e = best_ms([&] { k_copy<<<sms * 8, kPeakThreads, 0, st>>>(a, b, bytes / 16); }, st, 5, &ms);
    if (e == cudaSuccess) *hbm = 2.0 * bytes / (ms * 1e-3) / 1e9;
    cudaFree(a);
    cudaFree(b);
    return e;
}

}  // namespace sfoc
