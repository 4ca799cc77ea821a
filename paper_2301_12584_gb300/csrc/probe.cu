// Throughput probes for the rooflines the driver does not measure: FP32 FMA
// (scalar and paired f32x2), FP64 FMA, and L2 read bandwidth.  Each runs a
// fixed, bounded amount of work on every SM and is timed with CUDA events on
// the caller's stream; results are whole-GPU rates.
#include "common.cuh"
#include "internal.h"

#include <cuda_runtime.h>

#include <algorithm>

namespace krp {
namespace {

constexpr int PROBE_THREADS = 256;

// 8 independent FMA chains per thread; the result is kept live by a store
// that depends on every chain.
__global__ void __launch_bounds__(PROBE_THREADS) probe_fp32(float* __restrict__ sink, int iters) {
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = 1e-3f * (threadIdx.x + q);
    const float m = 0.9999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = fmaf(a[q], m, c);
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += a[q];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_fp32x2(float* __restrict__ sink, int iters) {
    float2 a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = make_float2(1e-3f * (threadIdx.x + q), 2e-3f * (threadIdx.x + q));
    const float2 m = make_float2(0.9999f, 0.9998f), c = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = ffma2(a[q], m, c);
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += a[q].x + a[q].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_fp64(double* __restrict__ sink, int iters) {
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = 1e-3 * (threadIdx.x + q);
    const double m = 0.9999, c = 1e-7;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += a[q];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// `passes` reads of an n4-float4 buffer (small enough to stay in L2).
__global__ void __launch_bounds__(PROBE_THREADS) probe_l2(const float4* __restrict__ buf, int64_t n4, int passes,
                                                          float* __restrict__ sink) {
    float t = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            t += v.x + v.y + v.z + v.w;
        }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace
}  // namespace krp

using namespace krp;

extern "C" krp_status krp_probe_peaks(double* out_host, void* stream) {
    if (!out_host) return KRP_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return KRP_ECUDA;
    const int blocks = sms * 8;
    const int64_t nthreads = (int64_t)blocks * PROBE_THREADS;
    const int64_t l2_bytes = 64ll << 20;   // 64 MB, inside GB300's 129 MB L2
    const int64_t n4 = l2_bytes / 16;
    float* sink = nullptr;
    float4* buf = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&sink, nthreads * sizeof(double)) != cudaSuccess) return KRP_ENOMEM;
    if (cudaMalloc(&buf, l2_bytes) != cudaSuccess) {
        cudaFree(sink);
        return KRP_ENOMEM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemsetAsync(buf, 0, l2_bytes, st);
    auto timed = [&](auto launch) -> double {
        launch();   // warm-up
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return (double)ms * 1e-3;
    };
    const int it32 = 1 << 16, it64 = 1 << 11, passes = 20;
    const double t32 = timed([&] { probe_fp32<<<blocks, PROBE_THREADS, 0, st>>>(sink, it32); });
    const double t32x2 = timed([&] { probe_fp32x2<<<blocks, PROBE_THREADS, 0, st>>>(sink, it32); });
    const double t64 = timed([&] { probe_fp64<<<blocks, PROBE_THREADS, 0, st>>>(reinterpret_cast<double*>(sink), it64); });
    const double tl2 = timed([&] { probe_l2<<<blocks, PROBE_THREADS, 0, st>>>(buf, n4, passes, sink); });
    for (int q = 0; q < 8; ++q) count_launch();
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(buf);
    if (err != cudaSuccess) return KRP_ECUDA;
    const double fma32 = (double)nthreads * it32 * 8, fma64 = (double)nthreads * it64 * 8;
    out_host[0] = 2.0 * fma32 / t32 * 1e-12;          // FP32 TFLOP/s, scalar FMA
    out_host[1] = 2.0 * 2.0 * fma32 / t32x2 * 1e-12;  // FP32 TFLOP/s, paired f32x2 FMA
    out_host[2] = 2.0 * fma64 / t64 * 1e-12;          // FP64 TFLOP/s
    out_host[3] = (double)l2_bytes * passes / tl2 * 1e-9;   // L2 read GB/s
    return KRP_OK;
}
