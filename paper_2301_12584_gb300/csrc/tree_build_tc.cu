// a1 (split precision): leaf Grams G^v = U[S(v)]ᵀU[S(v)] of the segment tree
// (Alg. 3, Eq. partial_gram) on the tcgen05 tensor cores.
//
// Each FP32 entry x is split into BF16 parts x = hi + lo + O(2^-17 |x|)
// (hi = bf16(x), lo = bf16(x - hi)); a Gram is formed as
// hiᵀhi + hiᵀlo + loᵀhi with FP32 accumulation in tensor memory, so each
// product carries about 16 significant bits against FP32's 24 (the dropped
// loᵀlo term and the rounding of lo are each below 2^-17 |x||y|).
//
// One 128 x 128 x Fp product places 128/RP leaves side by side (RP = R padded
// to 16, 32, 64 or 128): row block b of both operands holds leaf b transposed
// (its R columns along M or N, its F rows along K, zero padding), so block
// (b, b) of the product is leaf b's Gram and the off-diagonal blocks are
// discarded.  The operand tile is written once, K-major in 8 x 16-byte core
// matrices without swizzle, and serves as both A and B.  Warp w reads TMEM
// lanes 32w..32w+31, i.e. rows of the Gram of the leaf those lanes hold, and
// writes their upper triangles into the group's leaf array; the pairwise sums
// up the tree are the FP32 kernel's, in plain FP32 (the leaves' own ~1e-5
// error dominates the sums' rounding).
//
// Per CTA: 128 threads, 128 TMEM columns; thread 0 issues the MMAs and commits
// them to an mbarrier that every thread waits on with a bounded number of
// tries (KRP_ETIMEOUT instead of a hang).  Shared memory is padded to at least
// 48 KB so that at most four CTAs (4 x 128 = 512 TMEM columns) share an SM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tree_reduce.cuh"

#include <algorithm>

namespace krp {
namespace {

constexpr uint32_t TC_COLS = 128;
// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, N = 128, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr int TC_WAIT_TRIES = 1 << 16;

__device__ __forceinline__ uint32_t tc_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// byte offset (between core matrices along K), stride-dimension byte offset
// (between 8-row groups along M/N), and the fixed version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < TC_WAIT_TRIES; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(tc_saddr(bar)), "r"(parity), "r"(100000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 lanes x 32 columns of FP32 from TMEM (lane base in bits 31..16 of taddr).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
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

// kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major, N = 128, M = 128.
constexpr uint32_t TC_IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(TC_IDESC_TF32), "r"(accumulate)
        : "memory");
}

// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (round to nearest):
// about 22 significant bits together.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// TF: TF32x3 operands (hi and lo TF32, 4 elements per 16-byte core-matrix
// row, K = 8 per MMA, F padded to 8) instead of BF16x3 (8 elements per row,
// K = 16 per MMA, F padded to 16); everything else is shared.
template <int RP, int LB, bool TF = false>
__global__ void __launch_bounds__(128) tree_leaves_tc(const float* __restrict__ U, int64_t I, int R, int F, int Fp,
                                                      int64_t L, int G, int Tp, float* __restrict__ tree,
                                                      float* __restrict__ top, float* __restrict__ copy_to,
                                                      int* __restrict__ status) {
    constexpr int NL = 128 / RP;              // leaves side by side in one product
    constexpr int NCH = (LB + NL - 1) / NL;   // products per group of LB leaves
    constexpr int EPC = TF ? 4 : 8;           // K elements per 16-byte core-matrix row
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T = tri_size(R);
    const int nk8 = Fp / EPC;                       // core-matrix columns along K
    const uint32_t sbo = (uint32_t)nk8 * 128u;      // bytes per 8-row group along M/N
    unsigned char* Xh = smem;
    unsigned char* Xl = smem + 128u * sbo / 8u;     // 128 rows x Fp operands
    float* sG = reinterpret_cast<float*>(Xl + 128u * sbo / 8u);
    float* stk = sG + (size_t)LB * Tp;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&tmem_base)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < LB * Tp; e += blockDim.x)
        if (e % Tp >= T) sG[e] = 0.f;  // packed tail stays zero
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    bool alive = true;
    const int64_t leaf0 = (int64_t)blockIdx.x * G * LB;

    for (int g = 0; g < G && alive; ++g) {
        const int64_t gleaf0 = leaf0 + (int64_t)g * LB;
        for (int ch = 0; ch < NCH && alive; ++ch) {
            // operand tile: row p = RP * b + c holds column c of leaf b, K = its rows
            for (int task = tid; task < 128 * nk8; task += 128) {
                const int p = task & 127, k8 = task >> 7;
                const int b = p / RP, c = p % RP;
                const int ll = ch * NL + b;
                const int64_t row0 = (gleaf0 + ll) * (int64_t)F + EPC * k8;
                const bool col_ok = ll < LB && c < R;
                float v[EPC];
#pragma unroll
                for (int i = 0; i < EPC; ++i) {
                    const int64_t row = row0 + i;
                    const bool ok = col_ok && EPC * k8 + i < F && row < I;
                    v[i] = ok ? __ldg(U + row * R + c) : 0.f;
                    if (ok && copy_to) copy_to[row * R + c] = v[i];
                }
                uint4 h, l;
                if constexpr (TF) {
                    split_tf32(v[0], h.x, l.x);
                    split_tf32(v[1], h.y, l.y);
                    split_tf32(v[2], h.z, l.z);
                    split_tf32(v[3], h.w, l.w);
                } else {
                    split2(v[0], v[1], h.x, l.x);
                    split2(v[2], v[3], h.y, l.y);
                    split2(v[EPC - 4], v[EPC - 3], h.z, l.z);
                    split2(v[EPC - 2], v[EPC - 1], h.w, l.w);
                }
                const uint32_t off = (uint32_t)(p >> 3) * sbo + (uint32_t)k8 * 128u + (uint32_t)(p & 7) * 16u;
                *reinterpret_cast<uint4*>(Xh + off) = h;
                *reinterpret_cast<uint4*>(Xl + off) = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t xh = tc_saddr(Xh), xl = tc_saddr(Xl);
                // two 16-byte core-matrix columns per MMA (K = 16 BF16 or 8 TF32)
                for (int ks = 0; ks < Fp / (2 * EPC); ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256u;
                    if constexpr (TF) {
                        tc_mma_tf32(tmem, tc_desc(xh + ko, 128u, sbo), tc_desc(xh + ko, 128u, sbo), ks > 0);
                        tc_mma_tf32(tmem, tc_desc(xh + ko, 128u, sbo), tc_desc(xl + ko, 128u, sbo), 1u);
                        tc_mma_tf32(tmem, tc_desc(xl + ko, 128u, sbo), tc_desc(xh + ko, 128u, sbo), 1u);
                    } else {
                        tc_mma(tmem, tc_desc(xh + ko, 128u, sbo), tc_desc(xh + ko, 128u, sbo), ks > 0);
                        tc_mma(tmem, tc_desc(xh + ko, 128u, sbo), tc_desc(xl + ko, 128u, sbo), 1u);
                        tc_mma(tmem, tc_desc(xl + ko, 128u, sbo), tc_desc(xh + ko, 128u, sbo), 1u);
                    }
                }
                tc_commit(&bar);
            }
            const bool ok = tc_wait(&bar, phase);
            alive = __syncthreads_and(ok) != 0;
            if (!alive) break;
            phase ^= 1u;
            tc_fence_after();
            const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
            if (RP >= 32) {
                const int b = (32 * warp) / RP;
                const int r = (32 * warp + lane) % RP;
                const int ll = ch * NL + b;
                float* gr = sG + (size_t)ll * Tp + tri_index(r, r, R) - r;  // &G[r][0] of packed row r
#pragma unroll 1
                for (int blk = 0; blk < RP / 32; ++blk) {
                    float v[32];
                    tc_ld32(tmem + lane_base + (uint32_t)(b * RP + 32 * blk), v);
                    if (ll < LB && r < R) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const int c = 32 * blk + q;
                            if (c >= r && c < R) gr[c] = v[q];
                        }
                    }
                }
            } else {  // RP == 16: lanes 0-15 and 16-31 hold two different leaves
                float v[32];
                tc_ld32(tmem + lane_base + (uint32_t)(32 * warp), v);
                const int half = lane >> 4;
                const int r = lane & 15;
                const int ll = ch * NL + 2 * warp + half;
                if (ll < LB && r < R) {
                    float* gr = sG + (size_t)ll * Tp + tri_index(r, r, R) - r;
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int c = q & 15;
                        if ((q >> 4) == half && c >= r && c < R) gr[c] = v[q];
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
        }
        if (!alive) break;
        reduce_group<LB, false>(sG, stk, tree, top, L, gleaf0, g, G, Tp, blockIdx.x);
        __syncthreads();
    }

    tc_fence_before();
    __syncthreads();
    if (!alive) {
        // an MMA may still be in flight: give it one more bounded wait before freeing TMEM
        if (tid == 0) tc_wait(&bar, phase);
        __syncthreads();
        if (tid == 0) set_status(status, KRP_ETIMEOUT);
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
    }
}

// Persistent, pipelined form (F R % 4 == 0, shared memory permitting).  A CTA
// walks blocks of G groups of LB leaves (block v covers leaves
// [v G LB, (v+1) G LB) and leaves its subtree root in top slot v), in chunks
// of 128/RP leaves: one chunk's rows are one contiguous run of U (NL F R
// floats, a stage), brought in by a bulk copy S chunks ahead (S = 3 for
// RP <= 32, 2 for RP = 64, 1 for RP = 128, where one chunk is a whole leaf
// of up to 64 KB); the sub-16-byte tail of a ragged last chunk comes by plain
// loads.
// Iteration i: wait for chunk i's rows, split them into the operand buffer
// (i mod 2) and write the factor copy; thread 0 then refills the stage with
// chunk i+S and issues chunk i's MMAs into TMEM buffer (i mod 2); meanwhile
// the warps wait for chunk i-1's products, read its leaf Grams, and sum a
// completed group up the tree.
template <int RP>
struct PipeCfg {
    static constexpr int S = RP <= 32 ? 3 : RP == 64 ? 2 : 1;   // stages
    static constexpr int MINB = RP <= 32 ? 2 : 1;                // CTAs per SM
};

__device__ __forceinline__ void tc_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tc_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_saddr(bar)) : "memory");
}
__device__ __forceinline__ void tc_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc_saddr(dst)),
                 "l"(src), "r"(bytes), "r"(tc_saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Position of a chunk in a CTA's walk: block vb, group g, chunk ch of the group.
struct ChunkPos {
    int64_t vb;
    int g, ch;
};
template <int NCH>
__device__ __forceinline__ void chunk_next(ChunkPos& c, int G) {
    if (++c.ch == NCH) {
        c.ch = 0;
        if (++c.g == G) {
            c.g = 0;
            c.vb += gridDim.x;
        }
    }
}

constexpr int PIPE_THREADS = 256;

template <int RP, int LB>
__global__ void __launch_bounds__(PIPE_THREADS, PipeCfg<RP>::MINB)
    tree_leaves_tc_pipe(const float* __restrict__ U, int64_t I, int R, int F, int Fp, int64_t L, int G, int Tp,
                        int64_t nvb, int stage_floats, float* __restrict__ tree, float* __restrict__ top,
                        float* __restrict__ copy_to, int* __restrict__ status) {
    constexpr int NL = 128 / RP;
    constexpr int NCH = (LB + NL - 1) / NL;
    constexpr int S = PipeCfg<RP>::S;
    constexpr int NT = PIPE_THREADS;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t mdone[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T = tri_size(R);
    const int nk8 = Fp >> 3;
    const uint32_t sbo = (uint32_t)nk8 * 128u;
    const uint32_t xbytes = 16u * sbo;  // 128 rows x Fp bf16
    float* stages = reinterpret_cast<float*>(smem);                  // stage_floats: a multiple of 32
    unsigned char* X = smem + (size_t)S * stage_floats * 4;         // [buffer][hi, lo]
    float* sG = reinterpret_cast<float*>(X + 4 * xbytes);
    float* stk = sG + (size_t)LB * Tp;
    const bool dense_shape = (F == Fp) && (R == RP);  // no padding inside a full chunk

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&tmem_base)),
                     "r"(2 * TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < S; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(&full[b])) : "memory");
        for (int b = 0; b < 2; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(&mdone[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < LB * Tp; e += NT)
        if (e % Tp >= T) sG[e] = 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    const int64_t my_vb = (int64_t)blockIdx.x < nvb ? (nvb - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nchunks = my_vb * G * NCH;
    auto rows_of = [&](const ChunkPos& c, int64_t& row0, int& nl, int& nvalid) {
        nl = min(NL, LB - c.ch * NL);
        row0 = ((c.vb * G + c.g) * LB + (int64_t)c.ch * NL) * F;
        nvalid = (int)max((int64_t)0, min((int64_t)nl * F, I - row0));
    };
    ChunkPos ahead{(int64_t)blockIdx.x, 0, 0};  // thread 0: next chunk to fetch
    int64_t issued = 0;
    auto issue = [&](int64_t i) {
        int64_t row0;
        int nl, nvalid;
        rows_of(ahead, row0, nl, nvalid);
        uint64_t* b = &full[i % S];
        // row0 R is a multiple of 4 (F R % 4 == 0): the source is 16-byte aligned
        const uint32_t bytes = ((uint32_t)nvalid * (uint32_t)R * 4u) & ~15u;
        if (bytes) {
            tc_expect_tx(b, bytes);
            tc_bulk_load(stages + (size_t)(i % S) * stage_floats, U + row0 * R, bytes, b);
        } else {
            tc_arrive(b);
        }
        chunk_next<NCH>(ahead, G);
        issued = i + 1;
    };
    if (tid == 0)
        for (int64_t i = 0; i < nchunks && i < S; ++i) issue(i);

    bool alive = true;
    int64_t consumed = 0, mma_issued = 0, mma_waited = 0;
    ChunkPos cur{(int64_t)blockIdx.x, 0, 0}, prev = cur;
    for (int64_t i = 0; i <= nchunks; ++i) {
        if (i < nchunks) {
            const int st = (int)(i % S);
            const bool ok = tc_wait(&full[st], (uint32_t)((i / S) & 1));
            alive = __syncthreads_and(ok) != 0;
            if (!alive) break;
            consumed = i + 1;
            int64_t row0;
            int nl, nvalid;
            rows_of(cur, row0, nl, nvalid);
            float* sU = stages + (size_t)st * stage_floats;
            const int nval = nvalid * R, ntail = nval & 3;   // floats past the bulk copy
            if (ntail) {                                     // CTA-uniform
                if (tid < ntail) sU[nval - ntail + tid] = U[row0 * R + nval - ntail + tid];
                __syncthreads();
            }
            unsigned char* Xh = X + (size_t)(i & 1) * 2 * xbytes;
            unsigned char* Xl = Xh + xbytes;
            const bool full_chunk = dense_shape && nl == NL && nvalid == NL * F;
            for (int task = tid; task < 128 * nk8; task += NT) {
                const int p = task & 127, k8 = task >> 7;
                const int b = p / RP, c = p % RP;
                const int rr0 = b * F + 8 * k8;
                float v[8];
                if (full_chunk) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = sU[(rr0 + q) * R + c];
                } else {
                    const bool col_ok = b < nl && c < R;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int rr = rr0 + q;
                        v[q] = (col_ok && 8 * k8 + q < F && rr < nvalid) ? sU[rr * R + c] : 0.f;
                    }
                }
                uint4 h, l;
                split2(v[0], v[1], h.x, l.x);
                split2(v[2], v[3], h.y, l.y);
                split2(v[4], v[5], h.z, l.z);
                split2(v[6], v[7], h.w, l.w);
                const uint32_t off = (uint32_t)(p >> 3) * sbo + (uint32_t)k8 * 128u + (uint32_t)(p & 7) * 16u;
                *reinterpret_cast<uint4*>(Xh + off) = h;
                *reinterpret_cast<uint4*>(Xl + off) = l;
            }
            if (copy_to) {
                float4* dst = reinterpret_cast<float4*>(copy_to + row0 * R);
                const float4* srcv = reinterpret_cast<const float4*>(sU);
                for (int q = tid; q < nval / 4; q += NT) dst[q] = srcv[q];
                if (tid < ntail) copy_to[row0 * R + nval - ntail + tid] = sU[nval - ntail + tid];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                if (i + S < nchunks) issue(i + S);
                const uint32_t xh = tc_saddr(Xh), xl = tc_saddr(Xl);
                const uint32_t d = tmem + (uint32_t)(i & 1) * TC_COLS;
                for (int ks = 0; ks < Fp / 16; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256u;
                    tc_mma(d, tc_desc(xh + ko, 128u, sbo), tc_desc(xh + ko, 128u, sbo), ks > 0);
                    tc_mma(d, tc_desc(xh + ko, 128u, sbo), tc_desc(xl + ko, 128u, sbo), 1u);
                    tc_mma(d, tc_desc(xl + ko, 128u, sbo), tc_desc(xh + ko, 128u, sbo), 1u);
                }
                tc_commit(&mdone[i & 1]);
            }
            mma_issued = i + 1;
        }
        if (i >= 1) {
            const int64_t j = i - 1;
            const bool ok = tc_wait(&mdone[j & 1], (uint32_t)((j >> 1) & 1));
            alive = __syncthreads_and(ok) != 0;
            if (!alive) break;
            mma_waited = j + 1;
            tc_fence_after();
            int64_t row0;
            int nl, nvalid;
            rows_of(prev, row0, nl, nvalid);
            // warp w reads TMEM lanes 32 (w mod 4) .. +31 and half (w / 4) of the
            // RP columns of the leaf those lanes hold
            const int qd = warp & 3, hf = warp >> 2;
            const uint32_t tbase = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(j & 1) * TC_COLS;
            if (RP >= 32) {
                const int b = (32 * qd) / RP, r = (32 * qd + lane) % RP;
                float* gr = (b < nl && r < R) ? sG + (size_t)(prev.ch * NL + b) * Tp + tri_index(r, r, R) - r
                                              : nullptr;
#pragma unroll
                for (int t = 0; t < RP / 32; ++t) {
                    const int c0 = hf * (RP / 2) + 16 * t;
                    float v[16];
                    tc_ld16(tbase + (uint32_t)(b * RP + c0), v);
                    if (gr) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int c = c0 + q;
                            if (c >= r && c < R) gr[c] = v[q];
                        }
                    }
                }
            } else {  // RP == 16: lanes 0-15 hold leaf 2qd, lanes 16-31 leaf 2qd+1; half hf holds leaf 2qd+hf
                float v[16];
                tc_ld16(tbase + (uint32_t)(32 * qd + 16 * hf), v);   // leaf 2qd+hf's 16 columns
                const int b = 2 * qd + hf, r = lane & 15;
                if ((lane >> 4) == hf && b < nl && r < R) {
                    float* gr = sG + (size_t)(prev.ch * NL + b) * Tp + tri_index(r, r, R) - r;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (q >= r && q < R) gr[q] = v[q];
                }
            }
            tc_fence_before();
            if (prev.ch == NCH - 1) {
                __syncthreads();
                reduce_group<LB, false>(sG, stk, tree, top, L, (prev.vb * G + prev.g) * LB, prev.g, G, Tp, prev.vb);
            }
            chunk_next<NCH>(prev, G);
        }
        if (i < nchunks) chunk_next<NCH>(cur, G);
        __syncthreads();
    }

    tc_fence_before();
    __syncthreads();
    if (!alive) {
        // let copies and products already in flight land before the CTA exits
        if (tid == 0) {
            for (int64_t c = consumed; c < issued; ++c) tc_wait(&full[c % S], (uint32_t)((c / S) & 1));
            for (int64_t c = mma_waited; c < mma_issued; ++c) tc_wait(&mdone[c & 1], (uint32_t)((c >> 1) & 1));
            set_status(status, KRP_ETIMEOUT);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_COLS) : "memory");
    }
}

int padded_rank(int R) { return R <= 16 ? 16 : R <= 32 ? 32 : R <= 64 ? 64 : 128; }

int tc_fp(int F, bool tf) { return tf ? (F + 7) / 8 * 8 : (F + 15) / 16 * 16; }

size_t tc_smem(int F, int LB, int G, int Tp, bool tf = false) {
    const int Fp = tc_fp(F, tf);
    int lv = 0;
    while ((1 << lv) < G) ++lv;
    // the cross-group stack only when there are groups to merge
    const size_t need = (size_t)2 * 128 * Fp * (tf ? 4 : 2) + (size_t)LB * Tp * 4 +
                        (G > 1 ? (size_t)2 * (lv + 1) * Tp * 4 : 0);
    return std::max<size_t>(need, 48 * 1024);  // at most 4 CTAs (512 TMEM columns) per SM
}

template <int RP, int LB, bool TF>
cudaError_t launch_tc(const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp, float* tree, float* top,
                      float* copy_to, int* status, int64_t ctas, size_t smem, cudaStream_t st) {
    auto k = tree_leaves_tc<RP, LB, TF>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int Fp = tc_fp(F, TF);
    k<<<(unsigned)ctas, 128, smem, st>>>(U, I, R, F, Fp, L, G, Tp, tree, top, copy_to, status); count_launch();
    return cudaGetLastError();
}

template <int RP, bool TF>
cudaError_t launch_tc_lb(int LB, const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp, float* tree,
                         float* top, float* copy_to, int* status, int64_t ctas, size_t smem, cudaStream_t st) {
    switch (LB) {
        case 1: return launch_tc<RP, 1, TF>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        case 2: return launch_tc<RP, 2, TF>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        case 4: return launch_tc<RP, 4, TF>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        case 8: return launch_tc<RP, 8, TF>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        default: return launch_tc<RP, 16, TF>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
    }
}

int pipe_stages(int RP) { return RP <= 32 ? PipeCfg<32>::S : RP == 64 ? PipeCfg<64>::S : PipeCfg<128>::S; }
// one chunk: 128/RP leaves x F rows x R columns, padded to 128 bytes
int pipe_stage_floats(int R, int F) { return ((128 / padded_rank(R)) * F * R + 31) / 32 * 32; }
size_t pipe_smem(int R, int F, int LB, int G, int Tp) {
    const int Fp = (F + 15) / 16 * 16;
    int lv = 0;
    while ((1 << lv) < G) ++lv;
    return (size_t)pipe_stages(padded_rank(R)) * pipe_stage_floats(R, F) * 4 + (size_t)1024 * Fp +
           (size_t)LB * Tp * 4 + (G > 1 ? (size_t)2 * (lv + 1) * Tp * 4 : 0);
}
constexpr size_t PIPE_SMEM_MAX = 220 * 1024;

template <int RP, int LB>
cudaError_t launch_pipe(const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp, float* tree, float* top,
                        float* copy_to, int* status, int64_t nvb, size_t smem, int num_sms, cudaStream_t st) {
    auto k = tree_leaves_tc_pipe<RP, LB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // MINB CTAs per SM by design (the occupancy query reports one 105 KB CTA
    // per SM at RP <= 32 although two are resident: 0.28 vs 0.17 ms at 2^21 rows)
    const int Fp = (F + 15) / 16 * 16;
    const int64_t grid = std::min<int64_t>(nvb, (int64_t)PipeCfg<RP>::MINB * num_sms);
    k<<<(unsigned)grid, PIPE_THREADS, smem, st>>>(U, I, R, F, Fp, L, G, Tp, nvb, pipe_stage_floats(R, F), tree, top,
                                                  copy_to, status);
    count_launch();
    return cudaGetLastError();
}

template <int RP>
cudaError_t launch_pipe_lb(int LB, const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp, float* tree,
                           float* top, float* copy_to, int* status, int64_t nvb, size_t smem, int num_sms,
                           cudaStream_t st) {
    switch (LB) {
        case 1: return launch_pipe<RP, 1>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, nvb, smem, num_sms, st);
        case 2: return launch_pipe<RP, 2>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, nvb, smem, num_sms, st);
        case 4: return launch_pipe<RP, 4>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, nvb, smem, num_sms, st);
        default: return launch_pipe<RP, 8>(U, I, R, F, L, G, Tp, tree, top, copy_to, status, nvb, smem, num_sms, st);
    }
}

}  // namespace

bool tree_tc_supported(int R, int F) { return R >= 1 && R <= 128 && F >= 1 && F <= 128; }

// The pipelined form needs F R % 4 == 0 and a 16-byte aligned source (every
// chunk starts on a 16-byte boundary) and its stages, operand buffers and one
// leaf Gram within the shared memory of an SM.
bool tree_tc_pipelined(int R, int F, const float* U) {
    if (R < 1 || R > 128 || F < 1 || F > 128 || (F * R) % 4 != 0 || ((uintptr_t)U & 15u) != 0) return false;
    const int Tp = (tri_size(R) + 7) & ~7;
    return pipe_smem(R, F, 1, 1, Tp) <= PIPE_SMEM_MAX;
}

// Geometry of the tensor-core leaf kernels.  Pipelined: the largest LB <=
// min(8, L) leaves per group, then G = 2 groups per block when L allows, that
// fit the shared memory; padded to 80 KB so that at most two CTAs
// (2 x 256 TMEM columns) share an SM.  Else:
// LB leaves per group (power of two, <= 16, <= L, one group's leaf Grams
// <= 64 KB), G groups per CTA (power of two, <= 8, shared memory <= 200 KB).
void tree_tc_geometry(int R, int F, int64_t L, int Tp, bool pipelined, int* LB_out, int* G_out, size_t* smem_out,
                      bool tf32) {
    (void)R;
    int LB = 1, G = 1;
    size_t smem;
    if (pipelined) {
        int lb = 1;
        while (lb < 8 && (int64_t)lb * 2 <= L) lb *= 2;
        size_t need = 0;
        for (bool done = false; lb >= 1 && !done; lb /= 2)
            for (int g = L / lb >= 2 ? 2 : 1; g >= 1 && !done; --g) {
                need = pipe_smem(R, F, lb, g, Tp);
                if (need <= PIPE_SMEM_MAX || (lb == 1 && g == 1)) {
                    LB = lb;
                    G = g;
                    done = true;
                }
            }
        smem = std::max<size_t>(need, 80 * 1024);
    } else {
        while (LB < 16 && (int64_t)LB * 2 <= L && (size_t)LB * 2 * Tp * 4 <= 64 * 1024) LB *= 2;
        const int64_t groups = L / LB;
        while (G < 8 && (int64_t)G * 2 <= groups && tc_smem(F, LB, G * 2, Tp, tf32) <= 200 * 1024) G *= 2;
        smem = tc_smem(F, LB, G, Tp, tf32);
    }
    *LB_out = LB;
    *G_out = G;
    *smem_out = smem;
}

cudaError_t launch_tree_leaves_tc(const float* U, int64_t I, int R, int F, int64_t L, int LB, int G, int Tp,
                                  float* tree, float* top, float* copy_to, int* status, int64_t ctas, size_t smem,
                                  bool pipelined, int num_sms, cudaStream_t st, bool tf32) {
    if (tf32) switch (padded_rank(R)) {
            case 16: return launch_tc_lb<16, true>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
            case 32: return launch_tc_lb<32, true>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
            case 64: return launch_tc_lb<64, true>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
            default: return launch_tc_lb<128, true>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        }
    if (pipelined) switch (padded_rank(R)) {
            case 16: return launch_pipe_lb<16>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, num_sms, st);
            case 32: return launch_pipe_lb<32>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, num_sms, st);
            case 64: return launch_pipe_lb<64>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, num_sms, st);
            default: return launch_pipe_lb<128>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, num_sms, st);
        }
    switch (padded_rank(R)) {
        case 16: return launch_tc_lb<16, false>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        case 32: return launch_tc_lb<32, false>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        case 64: return launch_tc_lb<64, false>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
        default: return launch_tc_lb<128, false>(LB, U, I, R, F, L, G, Tp, tree, top, copy_to, status, ctas, smem, st);
    }
}

}  // namespace krp
