// Throughput probes (a measurement tool, not part of libkrpls): FP32 FMA
// (scalar and paired f32x2), FP64 FMA, and L2 read bandwidth, the
// denominators of the SIMT-, FP64- and L2-bound rooflines.  Each runs a fixed,
// bounded amount of work on every SM and is timed with CUDA events on the
// caller's stream; results are whole-GPU rates.  Built on its own into
// libkrpprobe.so and called by `python -m paper_2301_12584_gb300.profile_cases
// peaks`.
//
// int krp_probe_peaks(double* out_host, void* stream): out_host[0] FP32
// TFLOP/s with scalar FMA, [1] FP32 TFLOP/s with paired (f32x2) FMA, [2] FP64
// TFLOP/s, [3] L2 read GB/s (64 MB buffer).  Allocates and frees 64 MB of
// device memory; synchronous.  Returns 0, or -1 (NULL output), -2 (allocation
// failed), -3 (a CUDA call failed).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace krpprobe {
namespace {

// Two FP32 fused multiply-adds in one instruction.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    uint64_t d;
    const uint64_t ua = *reinterpret_cast<uint64_t*>(&a), ub = *reinterpret_cast<uint64_t*>(&b),
                   uc = *reinterpret_cast<uint64_t*>(&c);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(ua), "l"(ub), "l"(uc));
    return *reinterpret_cast<float2*>(&d);
}

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
}  // namespace krpprobe

using namespace krpprobe;

extern "C" int krp_probe_peaks(double* out_host, void* stream) {
    if (!out_host) return -1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return -3;
    const int blocks = sms * 8;
    const int64_t nthreads = (int64_t)blocks * PROBE_THREADS;
    const int64_t l2_bytes = 64ll << 20;   // 64 MB, inside GB300's 129 MB L2
    const int64_t n4 = l2_bytes / 16;
    float* sink = nullptr;
    float4* buf = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&sink, nthreads * sizeof(double)) != cudaSuccess) return -2;
    if (cudaMalloc(&buf, l2_bytes) != cudaSuccess) {
        cudaFree(sink);
        return -2;
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
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(buf);
    if (err != cudaSuccess) return -3;
    const double fma32 = (double)nthreads * it32 * 8, fma64 = (double)nthreads * it64 * 8;
    out_host[0] = 2.0 * fma32 / t32 * 1e-12;          // FP32 TFLOP/s, scalar FMA
    out_host[1] = 2.0 * 2.0 * fma32 / t32x2 * 1e-12;  // FP32 TFLOP/s, paired f32x2 FMA
    out_host[2] = 2.0 * fma64 / t64 * 1e-12;          // FP64 TFLOP/s
    out_host[3] = (double)l2_bytes * passes / tl2 * 1e-9;   // L2 read GB/s
    return 0;
}
