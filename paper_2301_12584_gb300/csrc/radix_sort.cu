// Stable LSD radix sort of (key, value) pairs of 32-bit words, 8 key bits per
// pass, for the deterministic sampled-fiber solve (sparse.cu): equal keys keep
// their input order, so sums taken over a sorted run are always added in the
// same order.
//
// A pass over n pairs: rs_hist counts each 2048-pair tile's digits into
// hist[digit][tile]; three scan launches (sc_*) turn hist into exclusive
// offsets (digit-major, so that offset(d, tile) = pairs of smaller digits +
// pairs of digit d in earlier tiles); rs_scatter sorts each tile by the digit in shared memory
// with eight stable one-bit splits (each a block-wide scan of the threads'
// zero counts), then writes every pair to offset(d, tile) + its rank among the
// tile's pairs of digit d.  Positions past n within the last tile hold pads
// (key 0xFFFFFFFF, digit 0xFF, initially last), which stay behind every real
// pair of the tile and are not written.  n may be a device value (a count
// another kernel produced): the kernels then loop over the tiles it implies
// on a grid sized for an upper bound, and no host read-back is needed.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace krp {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_IPT = 8;                         // pairs per thread, contiguous
constexpr int RS_TILE = RS_THREADS * RS_IPT;      // 2048

__device__ __forceinline__ int64_t rs_count(int64_t n, const int64_t* n_dev) { return n_dev ? *n_dev : n; }

__global__ void __launch_bounds__(RS_THREADS) rs_hist(const uint32_t* __restrict__ keys, int64_t n_host,
                                                      const int64_t* __restrict__ n_dev, int shift,
                                                      uint32_t* __restrict__ hist) {
    __shared__ uint32_t cnt[256];
    const int64_t n = rs_count(n_host, n_dev);
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        cnt[threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = tile * RS_TILE;
        for (int q = threadIdx.x; q < RS_TILE; q += RS_THREADS)
            if (base + q < n) atomicAdd(&cnt[(keys[base + q] >> shift) & 255u], 1u);
        __syncthreads();
        hist[(int64_t)threadIdx.x * ntiles + tile] = cnt[threadIdx.x];
        __syncthreads();
    }
}

// Exclusive scan in place of m words, by one CTA of 1024 threads.
__device__ __forceinline__ void rs_scan_body(uint32_t* __restrict__ a, int64_t m) {
    __shared__ uint32_t part[1024];
    const int64_t per = (m + 1023) / 1024;
    const int64_t lo = threadIdx.x * per, hi = min(m, lo + per);
    uint32_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += a[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum;
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// Exclusive scan in place of the m = 256 * ntiles words of hist (ntiles from
// n), in three launches over segments of SC_SEG words: the segments' sums,
// their exclusive scan (one CTA), then each segment's scan plus its offset.
constexpr int SC_THREADS = 1024;
constexpr int SC_SEG = SC_THREADS * 8;

__device__ __forceinline__ int64_t rs_words(int64_t n_host, const int64_t* n_dev) {
    return 256 * ((rs_count(n_host, n_dev) + RS_TILE - 1) / RS_TILE);
}

__global__ void __launch_bounds__(SC_THREADS) sc_sums(const uint32_t* __restrict__ a, int64_t n_host,
                                                      const int64_t* __restrict__ n_dev, uint32_t* __restrict__ bsum) {
    __shared__ uint32_t warp_tot[SC_THREADS / 32];
    const int64_t m = rs_words(n_host, n_dev);
    const int64_t base = (int64_t)blockIdx.x * SC_SEG + threadIdx.x * 8;
    uint32_t v = 0;
    if (base < m) {   // m is a multiple of 256: a thread's 8 words are all in range or none is
        const uint4 x = *reinterpret_cast<const uint4*>(a + base);
        const uint4 y = *reinterpret_cast<const uint4*>(a + base + 4);
        v = x.x + x.y + x.z + x.w + y.x + y.y + y.z + y.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SC_THREADS / 32; ++w) t += warp_tot[w];
        bsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) sc_bscan(uint32_t* __restrict__ bsum, int64_t n_host,
                                                 const int64_t* __restrict__ n_dev) {
    rs_scan_body(bsum, (rs_words(n_host, n_dev) + SC_SEG - 1) / SC_SEG);
}

__global__ void __launch_bounds__(SC_THREADS) sc_apply(uint32_t* __restrict__ a, int64_t n_host,
                                                       const int64_t* __restrict__ n_dev,
                                                       const uint32_t* __restrict__ bsum) {
    __shared__ uint32_t warp_tot[SC_THREADS / 32];
    const int64_t m = rs_words(n_host, n_dev);
    if ((int64_t)blockIdx.x * SC_SEG >= m) return;   // uniform across the CTA
    const int64_t base = (int64_t)blockIdx.x * SC_SEG + threadIdx.x * 8;
    uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (base < m) {
        const uint4 x = *reinterpret_cast<const uint4*>(a + base);
        const uint4 y = *reinterpret_cast<const uint4*>(a + base + 4);
        w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w; w[4] = y.x; w[5] = y.y; w[6] = y.z; w[7] = y.w;
    }
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += w[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t before = bsum[blockIdx.x];
    for (int q = 0; q < warp; ++q) before += warp_tot[q];
    uint32_t run = before + inc - t;
    if (base < m) {
        uint4 x, y;
        x.x = run; run += w[0];
        x.y = run; run += w[1];
        x.z = run; run += w[2];
        x.w = run; run += w[3];
        y.x = run; run += w[4];
        y.y = run; run += w[5];
        y.z = run; run += w[6];
        y.w = run;
        *reinterpret_cast<uint4*>(a + base) = x;
        *reinterpret_cast<uint4*>(a + base + 4) = y;
    }
}

// Block-wide exclusive scan of one value per thread; *total gets the sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) {
        const uint32_t t = warp_tot[w];
        if (w < warp) before += t;
        all += t;
    }
    __syncthreads();   // warp_tot is reused by the next scan
    *total = all;
    return before + inc - v;
}

__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         int64_t n_host, const int64_t* __restrict__ n_dev,
                                                         int shift, const uint32_t* __restrict__ off) {
    __shared__ uint32_t sk[RS_TILE], sv[RS_TILE];
    __shared__ uint32_t warp_tot[RS_THREADS / 32];
    __shared__ uint32_t dstart[256];
    const int64_t n = rs_count(n_host, n_dev);
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * RS_TILE;
        const int nvalid = (int)min((int64_t)RS_TILE, n - base);
        uint32_t k[RS_IPT], v[RS_IPT];
#pragma unroll
        for (int i = 0; i < RS_IPT; ++i) {
            const int q = threadIdx.x * RS_IPT + i;
            k[i] = q < nvalid ? kin[base + q] : 0xFFFFFFFFu;
            v[i] = q < nvalid ? vin[base + q] : 0u;
        }
        for (int b = 0; b < 8; ++b) {   // stable one-bit splits, lowest digit bit first
            uint32_t zeros = 0;
#pragma unroll
            for (int i = 0; i < RS_IPT; ++i) zeros += ((k[i] >> (shift + b)) & 1u) ^ 1u;
            uint32_t Z;
            const uint32_t zb = block_exclusive_scan(zeros, warp_tot, &Z);
            uint32_t z = zb, o = Z + threadIdx.x * RS_IPT - zb;
#pragma unroll
            for (int i = 0; i < RS_IPT; ++i) {
                const uint32_t pos = ((k[i] >> (shift + b)) & 1u) ? o++ : z++;
                sk[pos] = k[i];
                sv[pos] = v[i];
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < RS_IPT; ++i) {
                k[i] = sk[threadIdx.x * RS_IPT + i];
                v[i] = sv[threadIdx.x * RS_IPT + i];
            }
            __syncthreads();
        }
        // the tile is now ordered by digit; first position of each digit in it
        dstart[threadIdx.x] = 0xFFFFFFFFu;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RS_IPT; ++i) {
            const int q = threadIdx.x * RS_IPT + i;
            const uint32_t d = (k[i] >> shift) & 255u;
            const uint32_t prev = q > 0 ? (sk[q - 1] >> shift) & 255u : 256u;
            if (q < nvalid && d != prev) dstart[d] = q;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RS_IPT; ++i) {
            const int q = threadIdx.x * RS_IPT + i;
            if (q < nvalid) {
                const uint32_t d = (k[i] >> shift) & 255u;
                const int64_t dst = (int64_t)off[(int64_t)d * ntiles + tile] + (q - dstart[d]);
                kout[dst] = k[i];
                vout[dst] = v[i];
            }
        }
        __syncthreads();   // dstart and the tile buffers are reused by the next tile
    }
}

}  // namespace

// Exclusive scans in place, one CTA of 1024 threads: n words (uint32, host
// count) or the first *n_dev int64 words, whose total is written to *total.
__global__ void __launch_bounds__(1024) scan_u32_kernel(uint32_t* __restrict__ a, int64_t n) {
    rs_scan_body(a, n);
}
__global__ void __launch_bounds__(1024) scan_i64_kernel(int64_t* __restrict__ a, const int64_t* __restrict__ n_dev,
                                                        int64_t* __restrict__ total) {
    __shared__ int64_t part[1024];
    const int64_t n = *n_dev;
    const int64_t per = (n + 1023) / 1024;
    const int64_t lo = threadIdx.x * per, hi = min(n, lo + per);
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += a[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - sum;
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t v = a[i];
        a[i] = run;
        run += v;
    }
    if (threadIdx.x == 1023) *total = part[1023];
}

cudaError_t exclusive_scan_u32(uint32_t* a, int64_t n, cudaStream_t st) {
    scan_u32_kernel<<<1, 1024, 0, st>>>(a, n);
    count_launch();
    return cudaGetLastError();
}
cudaError_t exclusive_scan_i64(int64_t* a, const int64_t* n_dev, int64_t* total, cudaStream_t st) {
    scan_i64_kernel<<<1, 1024, 0, st>>>(a, n_dev, total);
    count_launch();
    return cudaGetLastError();
}

// The digit counts (256 per tile) and, after them, the scan's segment sums.
size_t radix_sort_hist_words(int64_t n) {
    const size_t m = (size_t)256 * (size_t)((n + RS_TILE - 1) / RS_TILE);
    return m + (m + SC_SEG - 1) / SC_SEG + 4;
}

// Stable sort of n pairs by the low `bits` bits of the keys.  (k0, v0) hold the
// input; (k1, v1) are work arrays of n words; hist has radix_sort_hist_words(n)
// words.  n_dev (may be null): the count in device memory, n then being an
// upper bound on it.  On return *in_work says whether the sorted pairs are in
// (k1, v1).  grid: CTAs per kernel (persistent over the tiles).
cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist, int64_t n,
                             const int64_t* n_dev, int bits, int grid, bool* in_work, cudaStream_t st) {
    *in_work = false;
    if (n <= 0) return cudaSuccess;
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, grid));
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    const int64_t m = 256 * ntiles;   // hist words for the bound n
    const unsigned nseg = (unsigned)((m + SC_SEG - 1) / SC_SEG);
    uint32_t* bsum = hist + ((m + 3) & ~(int64_t)3);
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist<<<g, RS_THREADS, 0, st>>>(ki, n, n_dev, shift, hist);
        sc_sums<<<nseg, SC_THREADS, 0, st>>>(hist, n, n_dev, bsum);
        sc_bscan<<<1, 1024, 0, st>>>(bsum, n, n_dev);
        sc_apply<<<nseg, SC_THREADS, 0, st>>>(hist, n, n_dev, bsum);
        rs_scatter<<<g, RS_THREADS, 0, st>>>(ki, vi, ko, vo, n, n_dev, shift, hist);
        for (int q = 0; q < 5; ++q) count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        std::swap(ki, ko);
        std::swap(vi, vo);
        *in_work = !*in_work;
    }
    return cudaSuccess;
}

}  // namespace krp

using namespace krp;

extern "C" krp_status krp_debug_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, void* stream) {
    if (!keys || !vals || n < 1 || n >= ((int64_t)1 << 31) || bits < 1 || bits > 32)
        return fail(nullptr, KRP_EINVAL, "krp_debug_sort_pairs: bad arguments");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *k1 = nullptr, *v1 = nullptr, *hist = nullptr;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMalloc(&k1, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&v1, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&hist, radix_sort_hist_words(n) * 4);
    bool in1 = false;
    if (e == cudaSuccess) e = radix_sort_pairs(keys, vals, k1, v1, hist, n, nullptr, bits, sms * 4, &in1, st);
    if (e == cudaSuccess && in1) e = cudaMemcpyAsync(keys, k1, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && in1) e = cudaMemcpyAsync(vals, v1, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(k1);
    cudaFree(v1);
    cudaFree(hist);
    return e == cudaSuccess ? KRP_OK : fail(nullptr, KRP_ECUDA, std::string("krp_debug_sort_pairs: ") + cudaGetErrorString(e));
}
