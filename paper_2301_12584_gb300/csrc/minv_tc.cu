// a8 (sparse): U_j = Y M⁻¹ on the tcgen05 tensor cores in split TF32
// (TF32x3), for the sketched solve of Alg. 6 (Y = SBᵀSA, M = SAᵀSA).
//
// Every operand x is split as x = hi + lo (hi = tf32(x), lo = tf32(x - hi),
// about 22 significant bits together); a product is hi hi' + hi lo' + lo hi'
// with FP32 accumulation in tensor memory (the dropped lo lo' and the
// rounding of lo are below 2^-21 |x||y|).
//
// A CTA keeps M⁻¹ (FP64, symmetric: its rows are the columns B needs) as the
// B operand, K-major hi and lo copies in shared memory, and walks tiles of
// 128 rows of Y: its threads split the tile into K-major hi and lo copies
// (8-row x 16-byte core matrices, no swizzle, as the BF16 leaf kernel lays
// them out; the rows are read into registers a tile ahead), thread 0 issues KP/8 x 3 MMAs (M = 128, N = NP, K = 8 each) into
// a 128 x NP FP32 accumulator in tensor memory, commits them to an mbarrier
// that every thread waits on (bounded), and the warps read the accumulator
// back (warp w: lanes 32 (w mod 4) .., column half w / 4), store U's rows and,
// for the ALS sweep, add the squares of every column over the tile's rows
// (reduce-scatter across the warp, double-float per lane across tiles) into
// the CTA's partial column sums, summed over CTAs in CTA order afterwards.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace krp {

cudaError_t launch_sumsq_reduce(const double* part, int nparts, int R, double* sumsq, cudaStream_t st);

namespace {

constexpr int MT_THREADS = 256;
constexpr int MT_WAIT_TRIES = 1 << 16;

__device__ __forceinline__ uint32_t mt_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle (start, leading byte offset
// between core matrices along K, stride byte offset between 8-row groups,
// version bits 46-48 = 0b001).
__device__ __forceinline__ uint64_t mt_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32 (format 2), both
// K-major, N = np, M = 128.
__device__ __forceinline__ uint32_t mt_idesc(int np) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mt_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool mt_wait(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < MT_WAIT_TRIES; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mt_saddr(bar)), "r"(parity), "r"(100000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mt_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (round to nearest).
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// Byte offset of element (row p, k) in a K-major operand with kp columns of K.
__device__ __forceinline__ uint32_t mt_off(int p, int k, int kp) {
    return (uint32_t)(p >> 3) * (uint32_t)(kp >> 2) * 128u + (uint32_t)(k >> 2) * 128u + (uint32_t)(p & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

// MT_LD: float4 loads per thread per tile, 128 rows x KP/4 quads over 256
// threads (4, 7 or 13 for KP <= 32, 56, 104)
template <int MT_LD>
__global__ void __launch_bounds__(MT_THREADS) minv_tc(const float* __restrict__ Y, int RSY,
                                                      const double* __restrict__ Minv, int64_t I, int R, int KP,
                                                      int NP, uint32_t tcols, float* __restrict__ U,
                                                      double* __restrict__ part, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ double colsum[8][128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t abytes = 128u * (uint32_t)KP * 4u, bbytes = (uint32_t)NP * (uint32_t)KP * 4u;
    unsigned char* Ah = smem;
    unsigned char* Al = Ah + abytes;
    unsigned char* Bh = Al + abytes;
    unsigned char* Bl = Bh + bbytes;
    const uint32_t sboA = (uint32_t)(KP >> 2) * 128u;   // also B's: both have KP columns of K

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(mt_saddr(&tmem_base)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mt_saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B = M⁻¹ (row n of B's K-major copy = row n of the symmetric M⁻¹), zero padded
    for (int e = tid; e < NP * KP; e += MT_THREADS) {
        const int n = e / KP, k = e % KP;
        uint32_t hi = 0, lo = 0;
        if (n < R && k < R) {
            const double x = Minv[(size_t)n * R + k];
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"((float)x));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"((float)(x - (double)__uint_as_float(hi))));
        }
        *reinterpret_cast<uint32_t*>(Bh + mt_off(n, k, KP)) = hi;
        *reinterpret_cast<uint32_t*>(Bl + mt_off(n, k, KP)) = lo;
    }
    for (int e = tid; e < 8 * 128; e += MT_THREADS) colsum[e >> 7][e & 127] = 0.0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = mt_idesc(NP);
    uint32_t phase = 0;
    bool alive = true;
    df ss[2] = {df{0.f, 0.f}, df{0.f, 0.f}};   // this lane's column (32 per chunk) sums, chunks of its half
    const int nq = KP >> 2;                      // 16-byte quads of K per row
    const int64_t ntiles = (I + 127) / 128;
    // A tile's rows are read into registers one tile ahead (all of a thread's
    // loads issued together), so that they arrive while the previous tile's
    // products and epilogue run; rows >= I and columns >= R read as zero.
    float4 cur[MT_LD];
    auto load_tile = [&](int64_t tile) {
        const int64_t r0 = tile * 128;
        const int nr = tile < ntiles ? (int)min((int64_t)128, I - r0) : 0;
#pragma unroll
        for (int i = 0; i < MT_LD; ++i) {
            const int e = tid + i * MT_THREADS;
            const int p = e / nq, q = e - p * nq;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < 128 * nq && p < nr && 4 * q < R) {
                v = __ldg(reinterpret_cast<const float4*>(Y + (r0 + p) * (int64_t)RSY + 4 * q));
                if (4 * q + 1 >= R) v.y = 0.f;   // columns >= R of Y's row are padding
                if (4 * q + 2 >= R) v.z = 0.f;
                if (4 * q + 3 >= R) v.w = 0.f;
            }
            cur[i] = v;
        }
    };
    load_tile(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x) {
        const int64_t r0 = tile * 128;
        const int nr = (int)min((int64_t)128, I - r0);
        // A = the tile's rows (K-major), split
#pragma unroll
        for (int i = 0; i < MT_LD; ++i) {
            const int e = tid + i * MT_THREADS;
            if (e < 128 * nq) {
                const int p = e / nq, q = e - p * nq;
                uint4 h, l;
                tf32_split(cur[i].x, h.x, l.x);
                tf32_split(cur[i].y, h.y, l.y);
                tf32_split(cur[i].z, h.z, l.z);
                tf32_split(cur[i].w, h.w, l.w);
                const uint32_t off = mt_off(p, 4 * q, KP);
                *reinterpret_cast<uint4*>(Ah + off) = h;
                *reinterpret_cast<uint4*>(Al + off) = l;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = mt_saddr(Ah), al = mt_saddr(Al), bh = mt_saddr(Bh), bl = mt_saddr(Bl);
            for (int ks = 0; ks < KP / 8; ++ks) {
                const uint32_t ko = (uint32_t)ks * 256u;   // two core-matrix columns per K = 8
                mt_mma(tmem, mt_desc(ah + ko, 128u, sboA), mt_desc(bh + ko, 128u, sboA), idesc, ks > 0);
                mt_mma(tmem, mt_desc(ah + ko, 128u, sboA), mt_desc(bl + ko, 128u, sboA), idesc, 1u);
                mt_mma(tmem, mt_desc(al + ko, 128u, sboA), mt_desc(bh + ko, 128u, sboA), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             mt_saddr(&bar))
                         : "memory");
        }
        load_tile(tile + gridDim.x);   // the next tile's rows, while the products run
        const bool ok = mt_wait(&bar, phase);
        alive = __syncthreads_and(ok) != 0;
        if (!alive) break;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w reads lanes 32 (w % 4) .. (rows of the tile) and the
        // column chunks c = w / 4, w / 4 + 2, ... of 32
        const int row = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        for (int ch = warp >> 2, slot = 0; 32 * ch < NP; ch += 2, ++slot) {
            float v[32];
            mt_ld32(tmem + lane_base + (uint32_t)(32 * ch), v);
            if (row < nr) {
                float* dst = U + (r0 + row) * (int64_t)R + 32 * ch;
                const int ncol = min(32, R - 32 * ch);
                if ((R & 3) == 0) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (4 * q < ncol) *reinterpret_cast<float4*>(dst + 4 * q) =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (q < ncol) dst[q] = v[q];
                }
            }
            if (part) {
                // squares of this chunk's 32 columns over the warp's 32 rows,
                // reduce-scattered so that lane q holds column 32 ch + q
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = row < nr ? v[q] * v[q] : 0.f;
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    const bool upper = (lane & off) != 0;
#pragma unroll
                    for (int i = 0; i < off; ++i) {
                        const float send = upper ? v[i] : v[i + off];
                        const float keep = upper ? v[i + off] : v[i];
                        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                    }
                }
                if (slot < 2) ss[slot] = df_add(ss[slot], df{v[0], 0.f});
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // the accumulator and the A tiles are reused by the next tile
    }
    if (part && alive) {
        for (int ch = warp >> 2, slot = 0; 32 * ch < NP && slot < 2; ch += 2, ++slot)
            colsum[warp][32 * ch + lane] = (double)ss[slot].hi + (double)ss[slot].lo;
        __syncthreads();
        for (int c = tid; c < R; c += MT_THREADS) {
            double a = 0.0;
            for (int w = 0; w < 8; ++w) a += colsum[w][c];   // warps whose chunks miss c hold 0
            part[(size_t)blockIdx.x * 128 + c] = a;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!alive) {
        if (tid == 0) mt_wait(&bar, phase);   // an MMA may still be in flight: one more bounded wait
        __syncthreads();
        if (tid == 0) set_status(status, KRP_ETIMEOUT);
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

}  // namespace

// The tensor-core form serves R <= 104: the hi and lo copies of M⁻¹ (NP x KP)
// and of a 128-row tile of Y (128 x KP) then fit one CTA's shared memory.
// sumsq (may be null): Σ_i U[i, c]² via part (CTA partials).
bool minv_tc_supported(int R) { return R >= 1 && R <= 104; }

cudaError_t launch_minv_tc(const float* Y, int RSY, const double* Minv, int64_t I, int R, float* U, double* sumsq,
                           double* part, int* status, int num_sms, cudaStream_t st) {
    const int KP = (R + 7) & ~7, NP = (R + 31) & ~31;
    const uint32_t tcols = NP <= 32 ? 32u : NP <= 64 ? 64u : 128u;
    const size_t sm = (size_t)2 * 128 * KP * 4 + (size_t)2 * NP * KP * 4;
    auto k = KP <= 32 ? minv_tc<4> : KP <= 56 ? minv_tc<7> : minv_tc<13>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, MT_THREADS, sm);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, (int)(512 / tcols)));
    const int64_t ntiles = (I + 127) / 128;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms * std::min(per_sm, 2));
    k<<<(unsigned)grid, MT_THREADS, sm, st>>>(Y, RSY, Minv, I, R, KP, NP, tcols, U, sumsq ? part : nullptr, status);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess || !sumsq) return e;
    return launch_sumsq_reduce(part, (int)grid, R, sumsq, st);
}

}  // namespace krp
