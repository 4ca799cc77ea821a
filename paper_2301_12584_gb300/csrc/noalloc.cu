// Dense sketched solve without any device allocation (krp_solve_dense_noalloc).
//
// For callers that cannot call cudaMalloc: for example a host framework that
// owns all device memory through its own pool and forbids other allocations,
// or a latency-critical loop where an allocation could fail under a tight
// memory budget or stall the device.  The caller passes the sketched rows,
// weights, right-hand sides, the output and a device status word; the solve's
// scratch (per-CTA partial sums of SAᵀSA and SAᵀSB) lives in the file-scope
// array below, which every GPU that runs this library keeps until the process
// exits.
//
// The kernels are the ones krp_solve_dense runs (solve.cu); only where their
// scratch lives differs.
#include "common.cuh"
#include "internal.h"

namespace krp {

// kernels defined in solve.cu
__global__ void normal_partial(const float* __restrict__ SA, const float* __restrict__ w,
                               const float* __restrict__ B, int64_t J, int R, int nrhs, int64_t rows_per_cta,
                               float* __restrict__ part, float* __restrict__ part_exp);
__global__ void normal_solve(const float* __restrict__ part, int nparts, int R, int nrhs, int mode, int flags,
                            float* __restrict__ X, double* __restrict__ Xd, int* __restrict__ status,
                            double* __restrict__ gbuf, const float* __restrict__ part_exp);

}  // namespace krp

namespace {

// Limits of the allocation-free solve.
constexpr int NA_MAX_R = 32;
constexpr int NA_MAX_NRHS = 16;
constexpr int NA_MAX_PARTS = 512;
constexpr int NA_MAX_OUT = NA_MAX_R * (NA_MAX_R + 1) / 2 + NA_MAX_R * NA_MAX_NRHS;  // 1040 floats per partial

// Scratch shared by every call on a device: NA_MAX_PARTS partials of
// NA_MAX_OUT floats, then one exponent per partial (2.13 MB).  Each call
// overwrites the partials it uses before reading them, so the array needs no
// initial value.
static __device__ __align__(256) float g_krp_noalloc_scratch[NA_MAX_PARTS * NA_MAX_OUT + NA_MAX_PARTS];

// Device address of the scratch in the current device's context (the
// symbol's name is only a host-side stand-in and must not be passed to a
// kernel).  Looked up on every call: the address is fixed within a context,
// but a context made after cudaDeviceReset, or another context on the same
// device, may hold the library's device code elsewhere, so no address is
// kept between calls.  After the first lookup in a context (which may load
// the device code) a lookup is a host-side table read.
float* scratch_for(cudaError_t* err) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_krp_noalloc_scratch);
    return *err == cudaSuccess ? static_cast<float*>(p) : nullptr;
}

}  // namespace

extern "C" krp_status krp_solve_dense_noalloc(int64_t J, int R, const float* SA, const float* weight,
                                              const float* B_rows, int nrhs, float* X, int flags, int* status,
                                              void* stream) {
    using namespace krp;
    if (!SA || !weight || !B_rows || !X || !status) return fail(nullptr, KRP_EINVAL, "krp_solve_dense_noalloc: NULL buffer");
    if (J < 1 || J >= ((int64_t)1 << 31))
        return fail(nullptr, KRP_EINVAL, "krp_solve_dense_noalloc: need 1 <= J < 2^31");
    if (R < 1 || R > NA_MAX_R || nrhs < 1 || nrhs > NA_MAX_NRHS)
        return fail(nullptr, KRP_EINVAL,
                    "krp_solve_dense_noalloc: R must be in [1, 32] and nrhs in [1, 16] (fixed scratch size)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(nullptr, KRP_ECUDA, std::string("krp_solve_dense_noalloc: ") + cudaGetErrorString(e));
    float* base = scratch_for(&e);
    if (!base) return fail(nullptr, KRP_ECUDA, std::string("krp_solve_dense_noalloc: scratch address: ") +
                                                   cudaGetErrorString(e));
    float* part = base;
    const int T = tri_size(R);
    const int nout = T + R * nrhs;
    int64_t np = (J + 255) / 256;
    if (np > 2 * (int64_t)sms) np = 2 * (int64_t)sms;
    if (np > NA_MAX_PARTS) np = NA_MAX_PARTS;
    const int nparts = (int)np;
    const int64_t rows_per_cta = (J + nparts - 1) / nparts;
    // the kernels only ever raise the status word, so it is cleared first, on the same stream
    e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e != cudaSuccess) return fail(nullptr, KRP_ECUDA, std::string("krp_solve_dense_noalloc: ") + cudaGetErrorString(e));
    const dim3 grid1(nparts, (nout + 256 * 8 - 1) / (256 * 8));
    float* part_exp = part + (size_t)nparts * nout;
    normal_partial<<<grid1, 256, (size_t)32 * (R + nrhs) * 4, st>>>(SA, weight, B_rows, J, R, nrhs, rows_per_cta,
                                                                   part, part_exp); count_launch();
    const size_t small = 64 * 8 + 2 * (R / 2 + 1) * 8 + 2 * (R / 2 + 1) * 4 + 16;
    const size_t mats = (size_t)(2 * R * R + R * nrhs) * 8;
    normal_solve<<<1, 256, small + mats, st>>>(part, nparts, R, nrhs, 0, flags, X, nullptr, status, nullptr,
                                               part_exp); count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, KRP_ECUDA, std::string("krp_solve_dense_noalloc: ") + cudaGetErrorString(e));
    return KRP_OK;
}
