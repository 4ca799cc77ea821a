// a7 + a8 (sparse) + a9: sampled-fiber lookup, SBᵀSA, Y M⁻¹, column
// normalisation, and the STS-CP sweep (Sec. 3.3; Alg. 6; App. A.9; fit of
// Sec. 4.3).
//
// Mode-j index (built once, host sort as in the paper's preprocessing): every
// nonzero gets the key packing its coordinates in the modes k != j (ascending
// k, ceil(log2 I_k) bits each); nonzeros are sorted by key, equal keys form a
// mode-j fiber (one row of mat(T, j)ᵀ restricted to its nonzeros).
//
// Solve, with every sum taken in a fixed order (the result does not depend on
// scheduling, so a sweep and its CUDA-graph replay are bit-identical):
//   1. a thread per sampled tuple binary-searches its key among the fiber keys;
//   2. the samples are sorted by fiber id (stable radix sort, radix_sort.cu):
//      samples of one fiber share its nonzeros, so each distinct sampled
//      fiber u gets acc_u = Σ_s w_s SA[s, :] over its run of samples (seg_sums:
//      fixed chunks of sorted positions, runs that cross a chunk summed from
//      per-chunk partials in chunk order);
//   3. its (fiber, nonzero) pairs are numbered by a scan of the fibers'
//      lengths and sorted by the nonzero's mode-j row;
//   4. the run of pairs of each row i_j forms Y[i_j, :] = Σ v acc_u in an
//      order fixed by the sorted positions (the same chunked sums) and stores
//      it (Y = SBᵀ SA, I_j x R; untouched rows stay zero);
//   5. U_j = Y M⁻¹ with M = SAᵀ SA (FP64 Cholesky inverse, applied in FP32),
//      the column sums of squares as per-CTA partials summed in CTA order.
#include "common.cuh"
#include "internal.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <vector>

namespace krp {

// radix_sort.cu
size_t radix_sort_hist_words(int64_t n);
cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist, int64_t n,
                             const int64_t* n_dev, int bits, int grid, bool* in_work, cudaStream_t st);
cudaError_t exclusive_scan_u32(uint32_t* a, int64_t n, cudaStream_t st);
cudaError_t exclusive_scan_i64(int64_t* a, const int64_t* n_dev, int64_t* total, cudaStream_t st);

struct LookupParams {
    const uint64_t* fkeys;
    const int64_t* fptr;
    const int32_t* fidx;
    const float* fval;
    int64_t nfib;
    int other[16];
    int kbits[16];
    int n_other;
    const int32_t* idx;  // N x J
    const float* weight;
    const float* SA;     // J x R
    int64_t J;
    int R;
    float* Y;            // I_j x RS, RS = R rounded up to 4 (columns >= R stay zero)
    int RS;
};

// Step 1: per sample, its fiber id (nfib when the tuple has no nonzero) as a
// sort key, and its index as the value.
__global__ void __launch_bounds__(256) fiber_find(LookupParams P, uint32_t* __restrict__ key,
                                                  uint32_t* __restrict__ val) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < P.J; s += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
        for (int q = 0; q < P.n_other; ++q)
            k = (k << P.kbits[q]) | (uint64_t)(uint32_t)P.idx[(int64_t)P.other[q] * P.J + s];
        int64_t lo = 0, hi = P.nfib;  // lower_bound over the sorted fiber keys
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(P.fkeys + mid) < k)
                lo = mid + 1;
            else
                hi = mid;
        }
        key[s] = (uint32_t)((lo < P.nfib && __ldg(P.fkeys + lo) == k) ? lo : P.nfib);
        val[s] = (uint32_t)s;
    }
}

// Step 2a: run heads of the sorted fiber ids (flag 1 at the first sample of
// each distinct sampled fiber), to be scanned into distinct-fiber numbers.
__global__ void __launch_bounds__(256) run_heads(const uint32_t* __restrict__ key, int64_t J, uint32_t nfib,
                                                 uint32_t* __restrict__ flag) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= J; p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = p < J && key[p] != nfib && (p == 0 || key[p] != key[p - 1]) ? 1u : 0u;
}

// Step 2b: with scan = the exclusive scan of the head flags, distinct fiber
// u = (heads before p) owns positions useg[2u] .. useg[2u + 1] - 1; its fiber
// id and length (poff[u], scanned next); cnt[0] = the number of distinct fibers.
__global__ void __launch_bounds__(256) run_segments(const uint32_t* __restrict__ key, int64_t J, uint32_t nfib,
                                                    const uint32_t* __restrict__ scan,
                                                    const int64_t* __restrict__ fptr, int64_t* __restrict__ useg,
                                                    int64_t* __restrict__ ufib, int64_t* __restrict__ poff,
                                                    int64_t* __restrict__ cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < J; p += (int64_t)gridDim.x * blockDim.x) {
        if (p == 0) cnt[0] = scan[J];
        const uint32_t f = key[p];
        if (f == nfib) continue;
        const bool head = p == 0 || key[p - 1] != f;
        const bool tail = p == J - 1 || key[p + 1] != f;
        const int64_t u = head ? scan[p] : (int64_t)scan[p] - 1;
        if (head) {
            useg[2 * u] = p;
            ufib[u] = f;
            poff[u] = __ldg(fptr + f + 1) - __ldg(fptr + f);
        }
        if (tail) useg[2 * u + 1] = p + 1;
    }
}

// Step 3: pair w (of cnt[1]) belongs to distinct fiber u (poff[u] <= w <
// poff[u + 1]) and is its nonzero w - poff[u]: key = that nonzero's mode-j
// row, value = w, and its fiber and nonzero on the side.
__global__ void __launch_bounds__(256) pair_fill(LookupParams P, const int64_t* __restrict__ ufib,
                                                 const int64_t* __restrict__ poff, const int64_t* __restrict__ cnt,
                                                 uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                                                 uint32_t* __restrict__ pu, uint32_t* __restrict__ pn) {
    const int64_t U = cnt[0], npairs = cnt[1];
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < npairs; w += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = U - 1;   // last u with poff[u] <= w
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (poff[mid] <= w)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t n = __ldg(P.fptr + ufib[lo]) + (w - poff[lo]);
        key[w] = (uint32_t)__ldg(P.fidx + n);
        val[w] = (uint32_t)w;
        pu[w] = (uint32_t)lo;
        pn[w] = (uint32_t)n;
    }
}

// Step 4a: the sorted pairs' distinct-fiber index and value, in sorted order.
__global__ void __launch_bounds__(256) pair_gather(LookupParams P, const uint32_t* __restrict__ val,
                                                   const uint32_t* __restrict__ pu, const uint32_t* __restrict__ pn,
                                                   const int64_t* __restrict__ cnt, uint32_t* __restrict__ su,
                                                   float* __restrict__ sv) {
    const int64_t npairs = cnt[1];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npairs; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = val[q];
        su[q] = pu[w];
        sv[q] = __ldg(P.fval + pn[w]);
    }
}

__device__ __forceinline__ void warp_reduce_scatter32(float (&a)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? a[i] : a[i + off];
            const float keep = upper ? a[i + off] : a[i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
}

// Steps 2c and 4b: sums over runs of equal keys in a sorted list, out[o] =
// Σ_p v_p X[u_p, :] over the run's positions p in order.  Step 2c (FIBER):
// the samples sorted by fiber, u_p = the sample, v_p = its weight, X = SA,
// o = the distinct fiber's number (the scanned head flag at the run's head):
// acc_u = Σ w_s SA[s, :].  Step 4b: the (row, pair) list sorted by mode-j row,
// u_p = the pair's distinct fiber, v_p = its value, X = acc, o = the row:
// Y[i, :] = Σ v acc_u.
//
// A run can be very long (a fiber that leverage sampling hits thousands of
// times; a row of a Zipf mode with a large share of the nonzeros), so warps
// take fixed chunks of sorted positions rather than runs (SEG_CH for the
// pairs, SEG_CH_S for the J samples, which then still make many chunks): a
// run inside a chunk is summed there and written out; the piece of a run that continues
// from the previous chunk (slot 0) and the piece of one that goes on into
// the next (slot 1) are written to per-chunk partials, which seg_fix then adds
// in chunk order.  Inside a chunk, runs of one position (four at a time) and
// of up to 32 are summed in order with the lanes over columns; a longer piece
// with position q on lane (q - start) mod 32, each lane in order, then a fixed
// butterfly.  Every sum's order depends only on the sorted positions, so the
// result does not depend on scheduling.
constexpr int SEG_CH = 1024;
constexpr int SEG_CH_S = 64;

struct SegSrc {
    const uint32_t* key;     // sorted run keys
    const uint32_t* su;      // 4b: per position, the row of X
    const float* sv;         // 4b: per position, the scale
    const uint32_t* sval;    // 2c: per position, the sample (row of X; its weight scales it)
    const float* weight;     // 2c: the samples' weights
    const uint32_t* scan;    // 2c: exclusive scan of the run-head flags (the output numbers)
    const float* X;          // source rows, stride R
    float* out;              // output rows, stride RO
    int R, RO;
};

template <bool FIBER>
__device__ __forceinline__ void seg_uv(const SegSrc& S, int64_t p, uint32_t& u, float& v) {
    if (FIBER) {
        u = S.sval[p];
        v = __ldg(S.weight + u);
    } else {
        u = S.su[p];
        v = S.sv[p];
    }
}
template <bool FIBER>
__device__ __forceinline__ int64_t seg_count(const int64_t* cnt, const int64_t* useg) {
    if (FIBER) return cnt[0] > 0 ? useg[2 * cnt[0] - 1] : 0;   // the found samples (the rest sort last)
    return cnt[1];
}

// info[c] = (slot 0 used, the run of slot 0 ends in chunk c, slot 1 used, slot 1's output number)
template <bool FIBER>
__global__ void __launch_bounds__(256) seg_sums(SegSrc S, const int64_t* __restrict__ cnt,
                                                const int64_t* __restrict__ useg, float* __restrict__ part,
                                                uint4* __restrict__ info) {
    const int lane = threadIdx.x & 31;
    constexpr int CH = FIBER ? SEG_CH_S : SEG_CH;
    const int64_t n = seg_count<FIBER>(cnt, useg);
    const int64_t nch = (n + CH - 1) / CH;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int R = S.R;
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nch; c += warps) {
        const int64_t cb = c * CH, ce = min(cb + CH, n);
        const bool cont_run = cb > 0 && S.key[cb - 1] == S.key[cb];
        uint32_t has0 = 0, end0 = 0, has1 = 0, out1 = 0;
        for (int64_t sb = cb; sb < ce; sb += 32) {
            const int64_t p = sb + lane;
            const bool valid = p < ce;
            const uint32_t kr = p < n ? S.key[p] : 0xffffffffu;
            uint32_t ku = 0;
            float kv = 0.f;
            if (valid) seg_uv<FIBER>(S, p, ku, kv);
            const uint32_t kprev = __shfl_up_sync(0xffffffffu, kr, 1);
            const uint32_t knext = __shfl_down_sync(0xffffffffu, kr, 1);
            const uint32_t prev = lane == 0 ? (p > 0 && p - 1 < n ? S.key[p - 1] : 0xffffffffu) : kprev;
            const uint32_t next = lane == 31 ? (p + 1 < n ? S.key[p + 1] : 0xffffffffu) : knext;
            const bool start = valid && (p == cb || prev != kr);
            const bool is_cont = p == cb && cont_run;
            const bool single = start && !is_cont && next != kr;
            // runs of one position, four at a time (their loads in flight together)
            unsigned singles = __ballot_sync(0xffffffffu, single);
            while (singles) {
                int hs[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    hs[t] = singles ? __ffs(singles) - 1 : -1;
                    singles &= singles ? singles - 1 : 0u;
                }
                uint32_t us[4];
                int64_t os[4];
                float vs[4], xs[4][4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int src = hs[t] < 0 ? 0 : hs[t];
                    us[t] = __shfl_sync(0xffffffffu, ku, src);
                    vs[t] = __shfl_sync(0xffffffffu, kv, src);
                    const uint32_t kt = __shfl_sync(0xffffffffu, kr, src);
                    os[t] = hs[t] < 0 ? 0 : (FIBER ? (int64_t)S.scan[sb + src] : (int64_t)kt);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        xs[t][q] = (hs[t] >= 0 && lane + 32 * q < R) ? __ldg(S.X + (int64_t)us[t] * R + lane + 32 * q)
                                                                      : 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (hs[t] >= 0 && lane + 32 * q < R) S.out[os[t] * S.RO + lane + 32 * q] = vs[t] * xs[t][q];
            }
            unsigned heads = __ballot_sync(0xffffffffu, start && !single);
            while (heads) {
                const int h = __ffs(heads) - 1;
                heads &= heads - 1;
                const int64_t p0 = sb + h;
                const uint32_t row = __shfl_sync(0xffffffffu, kr, h);
                // the piece's end within the chunk: from the lanes' keys, then
                // 32 positions at a time
                const unsigned same = __ballot_sync(0xffffffffu, valid && kr == row) >> h;
                const bool to_end = same == (0xffffffffu >> h);
                int64_t e = to_end ? sb + 32 : p0 + __ffs(~same) - 1;
                if (to_end)
                    for (;;) {
                        const int64_t q = e + lane;
                        const unsigned more = __ballot_sync(0xffffffffu, q < ce && S.key[q] == row);
                        if (more != 0xffffffffu) {
                            e += __ffs(~more) - 1;
                            break;
                        }
                        e += 32;
                    }
                const bool cont = p0 == cb && cont_run;
                const bool cross = e == ce && ce < n && S.key[ce] == row;
                float* dst;
                if (cont) {
                    dst = part + (c * 2 + 0) * R;
                    has0 = 1;
                    end0 = cross ? 0u : 1u;
                } else if (cross) {
                    dst = part + (c * 2 + 1) * R;
                    has1 = 1;
                    out1 = FIBER ? S.scan[p0] : row;
                } else {
                    dst = S.out + (FIBER ? (int64_t)S.scan[p0] : (int64_t)row) * S.RO;
                }
                if (e - p0 <= 32) {
                    float a[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int64_t q = p0; q < e; ++q) {
                        const int i = (int)(q - sb);
                        uint32_t u;
                        float v;
                        if (i < 32) {   // warp-uniform
                            u = __shfl_sync(0xffffffffu, ku, i);
                            v = __shfl_sync(0xffffffffu, kv, i);
                        } else {
                            seg_uv<FIBER>(S, q, u, v);
                        }
                        const float* xu = S.X + (int64_t)u * R;
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            if (lane + 32 * w < R) a[w] = fmaf(v, __ldg(xu + lane + 32 * w), a[w]);
                    }
#pragma unroll
                    for (int w = 0; w < 4; ++w)
                        if (lane + 32 * w < R) dst[lane + 32 * w] = a[w];
                } else {
                    for (int c0 = 0; c0 < R; c0 += 32) {
                        float a[32];
#pragma unroll
                        for (int w = 0; w < 32; ++w) a[w] = 0.f;
                        for (int64_t q = p0 + lane; q < e; q += 32) {
                            uint32_t u;
                            float v;
                            seg_uv<FIBER>(S, q, u, v);
                            const float* xu = S.X + (int64_t)u * R + c0;
#pragma unroll
                            for (int w = 0; w < 32; ++w)
                                if (c0 + w < R) a[w] = fmaf(v, __ldg(xu + w), a[w]);
                        }
                        warp_reduce_scatter32(a);
                        if (c0 + lane < R) dst[c0 + lane] = a[0];
                    }
                }
            }
        }
        if (lane == 0) info[c] = make_uint4(has0, end0, has1, out1);
    }
}

// The runs that cross chunks: slot 1 of the chunk where the run starts, then
// slot 0 of each following chunk up to the one where it ends, in that order.
template <bool FIBER>
__global__ void __launch_bounds__(256) seg_fix(SegSrc S, const int64_t* __restrict__ cnt,
                                               const int64_t* __restrict__ useg, const float* __restrict__ part,
                                               const uint4* __restrict__ info) {
    const int lane = threadIdx.x & 31;
    constexpr int CH = FIBER ? SEG_CH_S : SEG_CH;
    const int64_t n = seg_count<FIBER>(cnt, useg);
    const int64_t nch = (n + CH - 1) / CH;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int R = S.R;
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nch; c += warps) {
        const uint4 in = info[c];
        if (!in.z) continue;
        float a[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) a[w] = lane + 32 * w < R ? part[(c * 2 + 1) * R + lane + 32 * w] : 0.f;
        for (int64_t d = c + 1; d < nch; ++d) {
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if (lane + 32 * w < R) a[w] += part[(d * 2 + 0) * R + lane + 32 * w];
            if (info[d].y) break;
        }
        float* dst = S.out + (int64_t)in.w * S.RO;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (lane + 32 * w < R) dst[lane + 32 * w] = a[w];
    }
}

// U[i, :] = Y[i, :] M⁻¹ (M⁻¹ FP64 -> FP32 in shared memory) and, when part
// is non-null, the CTA's Σ_i U[i, c]² over its rows into part[cta][c]
// (double-float partials per thread, summed in thread order; the CTAs'
// partials are then summed in CTA order by sumsq_reduce).  Persistent CTAs walk tiles of TM rows of
// Y (read into registers a tile ahead, coalesced), staged in shared memory
// with row stride R | 1 (the rows a warp reads
// fall in distinct banks); thread (ty, tx) accumulates RT rows x 8 columns,
// {4tx .. 4tx+3} and {RP/2 + 4tx ..}, against float4 rows of M⁻¹ (columns
// >= R zero).  RP = R padded to 32, 64 or 128.
constexpr int MINV_THREADS = 256;
template <int RP>
struct MinvCfg {
    static constexpr int TX = RP / 8, TY = MINV_THREADS / TX, RT = 4, TM = TY * RT;
    // M⁻¹, then the Y tile, which the final column reduction reuses for
    // 8 x MINV_THREADS doubles
    static size_t smem(int R) {
        return (size_t)RP * RP * 4 + std::max<size_t>((size_t)TM * (R | 1) * 4, (size_t)8 * MINV_THREADS * 8);
    }
};

template <int RP>
__global__ void __launch_bounds__(MINV_THREADS, 2) apply_minv(const float* __restrict__ Y, int RSY,
                                                              const double* __restrict__ Minv, int64_t I, int R,
                                                              float* __restrict__ U, double* __restrict__ part) {
    using C = MinvCfg<RP>;
    constexpr int TX = C::TX, RT = C::RT, TM = C::TM;
    extern __shared__ __align__(16) float sm[];
    float* sM = sm;              // [R][RP]
    float* sY = sM + RP * RP;    // [TM][RS]
    const int RS = R | 1;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k < R; k += MINV_THREADS / 32)
        for (int c = lane; c < RP; c += 32) sM[k * RP + c] = c < R ? (float)Minv[k * R + c] : 0.f;
    df ss[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ss[q] = df{0.f, 0.f};
    const int64_t ntiles = (I + TM - 1) / TM;
    // A tile of Y is TM contiguous rows of RSY floats (RSY a multiple of 4):
    // at most 8 float4 per thread, read into registers one tile ahead so that
    // they arrive during the previous tile's products.
    constexpr int LDN = 8;
    static_assert(TM * RP / 4 <= LDN * MINV_THREADS, "tile larger than the prefetch registers");
    float4 pre[LDN];
    auto load_tile = [&](int64_t tile) {
        const int64_t r0 = tile * TM;
        const int64_t nq = tile < ntiles ? (int64_t)min((int64_t)TM, I - r0) * RSY / 4 : 0;
        const float4* src = reinterpret_cast<const float4*>(Y + r0 * RSY);
#pragma unroll
        for (int i = 0; i < LDN; ++i) {
            const int e = threadIdx.x + i * MINV_THREADS;
            pre[i] = e < nq ? __ldg(src + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    load_tile(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * TM;
        const int nr = (int)min((int64_t)TM, I - r0);
        __syncthreads();   // the previous tile's reads of sY (and the writes of sM) are done
#pragma unroll
        for (int i = 0; i < LDN; ++i) {
            const int e = threadIdx.x + i * MINV_THREADS;
            const int row = (4 * e) / RSY, col = 4 * e - row * RSY;
            if (row < nr) {
                const float v[4] = {pre[i].x, pre[i].y, pre[i].z, pre[i].w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (col + j < R) sY[row * RS + col + j] = v[j];
            }
        }
        __syncthreads();
        load_tile(tile + gridDim.x);
        float2 acc[RT][4];
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = make_float2(0.f, 0.f);
        const float* yrow = sY + ty * RT * RS;
        for (int k = 0; k < R; ++k) {
            const float4 m0 = *reinterpret_cast<const float4*>(sM + k * RP + 4 * tx);
            const float4 m1 = *reinterpret_cast<const float4*>(sM + k * RP + RP / 2 + 4 * tx);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float y = yrow[r * RS + k];
                const float2 yy = make_float2(y, y);
                acc[r][0] = ffma2(yy, make_float2(m0.x, m0.y), acc[r][0]);
                acc[r][1] = ffma2(yy, make_float2(m0.z, m0.w), acc[r][1]);
                acc[r][2] = ffma2(yy, make_float2(m1.x, m1.y), acc[r][2]);
                acc[r][3] = ffma2(yy, make_float2(m1.z, m1.w), acc[r][3]);
            }
        }
        // rows >= nr hold stale shared memory: neither written nor summed
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int row = ty * RT + r;
            if (row >= nr) continue;
            float* dst = U + (r0 + row) * R;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c0 = h * (RP / 2) + 4 * tx;
                const float v[4] = {acc[r][2 * h].x, acc[r][2 * h].y, acc[r][2 * h + 1].x, acc[r][2 * h + 1].y};
                if ((R & 3) == 0 && c0 + 3 < R) {
                    *reinterpret_cast<float4*>(dst + c0) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c0 + q < R) dst[c0 + q] = v[q];
                }
                if (part) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) ss[4 * h + q] = df_add(ss[4 * h + q], df{v[q] * v[q], 0.f});
                }
            }
        }
    }
    if (!part) return;
    // column totals: the TY threads of a column group in fixed order
    __syncthreads();
    double* red = reinterpret_cast<double*>(sY);   // [TY][8 x TX] doubles <= TM * RS floats
#pragma unroll
    for (int q = 0; q < 8; ++q) red[ty * 8 * TX + q * TX + tx] = (double)ss[q].hi + (double)ss[q].lo;
    __syncthreads();
    for (int col = threadIdx.x; col < R; col += MINV_THREADS) {
        const int h = col / (RP / 2), rem = col % (RP / 2), t = rem / 4, q = 4 * h + rem % 4;
        double a = 0.0;
        for (int y = 0; y < C::TY; ++y) a += red[y * 8 * TX + q * TX + t];
        part[(size_t)blockIdx.x * 128 + col] = a;
    }
}

// σ²[c] = the CTAs' partials of column c, summed in CTA order.
__global__ void sumsq_reduce(const double* __restrict__ part, int nparts, int R, double* __restrict__ sumsq) {
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        double a = 0.0;
        for (int b = 0; b < nparts; ++b) a += part[(size_t)b * 128 + c];
        sumsq[c] = a;
    }
}

cudaError_t launch_sumsq_reduce(const double* part, int nparts, int R, double* sumsq, cudaStream_t st) {
    sumsq_reduce<<<1, 128, 0, st>>>(part, nparts, R, sumsq);
    count_launch();
    return cudaGetLastError();
}

// minv_tc.cu: U = Y M⁻¹ on tensor cores in split TF32 (R <= 104)
bool minv_tc_supported(int R);
cudaError_t launch_minv_tc(const float* Y, int RSY, const double* Minv, int64_t I, int R, float* U, double* sumsq,
                           double* part, int* status, int num_sms, cudaStream_t st);

template <int RP>
cudaError_t launch_minv_t(const float* Y, int RSY, const double* Minv, int64_t I, int R, float* U, double* sumsq,
                          double* part, int num_sms, cudaStream_t st) {
    using C = MinvCfg<RP>;
    const size_t sm = C::smem(R);
    cudaError_t e = cudaFuncSetAttribute(apply_minv<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (I + C::TM - 1) / C::TM;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms * 2);
    apply_minv<RP><<<(unsigned)grid, MINV_THREADS, sm, st>>>(Y, RSY, Minv, I, R, U, sumsq ? part : nullptr);
    count_launch();
    if (sumsq) {
        sumsq_reduce<<<1, 128, 0, st>>>(part, (int)grid, R, sumsq);
        count_launch();
    }
    return cudaGetLastError();
}

// Y: I x RSY (row stride RSY >= R); sumsq (may be null): the column sums of
// squares of U, via part (2 x SMs x 128 doubles)
cudaError_t launch_apply_minv(const float* Y, int RSY, const double* Minv, int64_t I, int R, float* U,
                              double* sumsq, double* part, int num_sms, cudaStream_t st) {
    if (R <= 32) return launch_minv_t<32>(Y, RSY, Minv, I, R, U, sumsq, part, num_sms, st);
    if (R <= 64) return launch_minv_t<64>(Y, RSY, Minv, I, R, U, sumsq, part, num_sms, st);
    return launch_minv_t<128>(Y, RSY, Minv, I, R, U, sumsq, part, num_sms, st);
}

// U[:, c] /= σ_c (a zero column stays zero), σ_c = sqrt(σ²_c) to sigma;
// a warp per row, lanes over columns.
__global__ void __launch_bounds__(256) col_scale(float* __restrict__ U, int64_t I, int R,
                                                 const double* __restrict__ sumsq, float* __restrict__ sigma) {
    __shared__ float inv[128];
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        const double sg = sqrt(sumsq[c]);
        inv[c] = sg > 0.0 ? (float)(1.0 / sg) : 1.f;
        if (blockIdx.x == 0) sigma[c] = (float)sg;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < I;
         i += (int64_t)gridDim.x * (blockDim.x >> 5))
        for (int c = lane; c < R; c += 32) U[i * R + c] *= inv[c];
}

// ⟨T, T̃⟩ = Σ_nnz v Σ_r σ_r Π_k U_k[i_k, r]  (FP64 accumulation).
struct FitParams {
    const float* U[16];
    const int32_t* coords;  // N x nnz
    const float* vals;
    const float* sigma;
    int64_t nnz;
    int N, R;
    double* out;   // one partial per CTA
};

__global__ void __launch_bounds__(256) fit_inner(FitParams P) {
    __shared__ double red[8];
    double a = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P.nnz; e += (int64_t)gridDim.x * blockDim.x) {
        float m = 0.f;
        for (int r = 0; r < P.R; ++r) {
            float p = P.sigma[r];
            for (int k = 0; k < P.N; ++k) p *= __ldg(P.U[k] + (int64_t)P.coords[(int64_t)k * P.nnz + e] * P.R + r);
            m += p;
        }
        a += (double)P.vals[e] * (double)m;
    }
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        P.out[blockIdx.x] = t;   // the CTAs' partials are summed in order on the host
    }
}

}  // namespace krp

using namespace krp;

namespace {

// Stable LSD radix sort of (key, perm) by key, 16-bit digits over `bits` bits.
void radix_sort(std::vector<uint64_t>& key, std::vector<uint32_t>& perm, int bits) {
    const size_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<uint32_t> p2(n);
    std::vector<size_t> cnt(65537);
    for (int shift = 0; shift < bits; shift += 16) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (size_t i = 0; i < n; ++i) ++cnt[((key[i] >> shift) & 0xffff) + 1];
        for (int d = 0; d < 65536; ++d) cnt[d + 1] += cnt[d];
        for (size_t i = 0; i < n; ++i) {
            const size_t dst = cnt[(key[i] >> shift) & 0xffff]++;
            k2[dst] = key[i];
            p2[dst] = perm[i];
        }
        key.swap(k2);
        perm.swap(p2);
    }
}

int bits_for(int64_t I) {
    int b = 1;
    while (b < 62 && ((int64_t)1 << b) < I) ++b;
    return b;
}

template <typename T>
bool dmalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

thread_local std::string g_tensor_error;

void free_lookup_scratch(krp_sptensor* t) {
    for (int q = 0; q < 2; ++q) {
        cudaFree(t->sk[q]);
        cudaFree(t->sv[q]);
        cudaFree(t->pk[q]);
        cudaFree(t->pv[q]);
        t->sk[q] = t->sv[q] = t->pk[q] = t->pv[q] = nullptr;
    }
    cudaFree(t->flag);
    cudaFree(t->useg);
    cudaFree(t->ufib);
    cudaFree(t->poff);
    cudaFree(t->cnt);
    cudaFree(t->uacc);
    cudaFree(t->pu);
    cudaFree(t->pn);
    cudaFree(t->hist);
    cudaFree(t->seg_part);
    cudaFree(t->seg_info);
    t->seg_part = nullptr;
    t->seg_info = nullptr;
    t->flag = t->pu = t->pn = t->hist = nullptr;
    t->useg = t->ufib = t->poff = t->cnt = nullptr;
    t->uacc = nullptr;
    t->lk_J = t->lk_pairs = t->lk_hist = t->lk_R = 0;
}

}  // namespace

extern "C" krp_status krp_sptensor_create(krp_sptensor** out, int N, const int64_t* I_host, int64_t nnz,
                                          const int32_t* const* coords_host, const float* vals_host,
                                          void* stream) {
    if (!out) return KRP_EINVAL;
    *out = nullptr;
    if (N < 2 || N > 16 || !I_host || !coords_host || !vals_host || nnz < 1 || nnz >= ((int64_t)1 << 32))
        return KRP_EINVAL;
    for (int k = 0; k < N; ++k)
        if (I_host[k] < 1 || I_host[k] >= ((int64_t)1 << 31) || !coords_host[k]) return KRP_EINVAL;
    for (int j = 0; j < N; ++j) {
        int b = 0;
        for (int k = 0; k < N; ++k)
            if (k != j) b += bits_for(I_host[k]);
        if (b > 63) return KRP_EINVAL;
    }
    for (int k = 0; k < N; ++k)
        for (int64_t e = 0; e < nnz; ++e)
            if (coords_host[k][e] < 0 || coords_host[k][e] >= I_host[k]) return KRP_EINVAL;
    krp_sptensor* t = new krp_sptensor();
    t->N = N;
    t->nnz = nnz;
    t->stream = (cudaStream_t)stream;
    t->I.assign(I_host, I_host + N);
    t->kbits.resize(N);
    for (int k = 0; k < N; ++k) t->kbits[k] = bits_for(I_host[k]);
    double n2 = 0.0;
    for (int64_t e = 0; e < nnz; ++e) n2 += (double)vals_host[e] * (double)vals_host[e];
    t->normT2 = n2;
    bool ok = dmalloc(&t->coords, (size_t)N * nnz) && dmalloc(&t->vals, (size_t)nnz);
    for (int k = 0; ok && k < N; ++k)
        ok = cudaMemcpy(t->coords + (size_t)k * nnz, coords_host[k], nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(t->vals, vals_host, nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    t->fkeys.assign(N, nullptr);
    t->fptr.assign(N, nullptr);
    t->fidx.assign(N, nullptr);
    t->fval.assign(N, nullptr);
    t->nfib.assign(N, 0);
    std::vector<uint64_t> key(nnz);
    std::vector<uint32_t> perm(nnz);
    for (int j = 0; ok && j < N; ++j) {
        int bits = 0;
        for (int64_t e = 0; e < nnz; ++e) {
            uint64_t kk = 0;
            for (int k = 0; k < N; ++k)
                if (k != j) kk = (kk << t->kbits[k]) | (uint64_t)(uint32_t)coords_host[k][e];
            key[e] = kk;
            perm[e] = (uint32_t)e;
        }
        for (int k = 0; k < N; ++k)
            if (k != j) bits += t->kbits[k];
        radix_sort(key, perm, bits);
        std::vector<uint64_t> fk;
        std::vector<int64_t> fp;
        std::vector<int32_t> fi(nnz);
        std::vector<float> fv(nnz);
        for (int64_t e = 0; e < nnz; ++e) {
            if (e == 0 || key[e] != key[e - 1]) {
                fk.push_back(key[e]);
                fp.push_back(e);
            }
            fi[e] = coords_host[j][perm[e]];
            fv[e] = vals_host[perm[e]];
        }
        fp.push_back(nnz);
        t->nfib[j] = (int64_t)fk.size();
        {   // fiber lengths as (length, count), longest first
            std::vector<int64_t> lens(fk.size());
            for (size_t f = 0; f < fk.size(); ++f) lens[f] = fp[f + 1] - fp[f];
            std::sort(lens.begin(), lens.end(), std::greater<int64_t>());
            std::vector<std::pair<int64_t, int64_t>> h;
            for (size_t f = 0; f < lens.size(); ++f) {
                if (h.empty() || h.back().first != lens[f])
                    h.push_back({lens[f], 1});
                else
                    ++h.back().second;
            }
            t->len_hist.push_back(std::move(h));
        }
        ok = dmalloc(&t->fkeys[j], fk.size()) && dmalloc(&t->fptr[j], fp.size()) && dmalloc(&t->fidx[j], (size_t)nnz) &&
             dmalloc(&t->fval[j], (size_t)nnz);
        ok = ok && cudaMemcpy(t->fkeys[j], fk.data(), fk.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t->fptr[j], fp.data(), fp.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t->fidx[j], fi.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t->fval[j], fv.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        krp_sptensor_destroy(t);
        return KRP_ENOMEM;
    }
    *out = t;
    return KRP_OK;
}

extern "C" void krp_sptensor_destroy(krp_sptensor* t) {
    if (!t) return;
    cudaStreamSynchronize(t->stream);
    cudaFree(t->coords);
    cudaFree(t->vals);
    for (int j = 0; j < (int)t->fkeys.size(); ++j) {
        cudaFree(t->fkeys[j]);
        cudaFree(t->fptr[j]);
        cudaFree(t->fidx[j]);
        cudaFree(t->fval[j]);
    }
    cudaFree(t->Y);
    free_lookup_scratch(t);
    delete t;
}

namespace krp {
// krp_solve_sparse, plus σ²[c] = Σ_i U_out[i, c]² when sumsq is non-null
krp_status solve_sparse_impl(krp_sampler* s, const krp_sptensor* tc, int j, int64_t J, const int32_t* idx,
                             const float* weight, const float* SA, float* U_out, int flags, double* sumsq) {
    if (!s || !tc || !idx || !weight || !SA || !U_out) return s ? fail(s, KRP_EINVAL, "null argument") : KRP_EINVAL;
    krp_sptensor* t = const_cast<krp_sptensor*>(tc);
    if (t->N != s->N || j < 0 || j >= s->N || J < 1 || J >= ((int64_t)1 << 31))
        return fail(s, KRP_EINVAL, "krp_solve_sparse: bad mode, J or tensor order");
    for (int k = 0; k < s->N; ++k)
        if (t->I[k] != s->I[k]) return fail(s, KRP_EINVAL, "krp_solve_sparse: tensor dims differ from the factors");
    const int R = s->R;
    const int RS = (R + 3) & ~3;   // Y's row stride: rows 16-byte aligned for Y M⁻¹
    const size_t ny = (size_t)s->I[j] * RS;
    if (ny > t->Y_floats) {
        cudaFree(t->Y);
        t->Y = nullptr;
        t->Y_floats = 0;
        if (!dmalloc(&t->Y, ny)) return fail(s, KRP_ENOMEM, "sparse Y scratch allocation failed");
        t->Y_floats = ny;
    }
    cudaError_t e = cudaMemsetAsync(t->Y, 0, ny * sizeof(float), s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "Y memset");
    LookupParams P{};
    P.fkeys = t->fkeys[j];
    P.fptr = t->fptr[j];
    P.fidx = t->fidx[j];
    P.fval = t->fval[j];
    P.nfib = t->nfib[j];
    for (int k = 0; k < s->N; ++k)
        if (k != j) {
            P.other[P.n_other] = k;
            P.kbits[P.n_other] = t->kbits[k];
            ++P.n_other;
        }
    P.idx = idx;
    P.weight = weight;
    P.SA = SA;
    P.J = J;
    P.R = R;
    P.Y = t->Y;
    P.RS = RS;
    // (fiber, nonzero) pairs a J-sample solve can read: the longest J fibers'
    // total length (at most nnz)
    int64_t pbound = 0, left = J;
    for (const auto& lc : t->len_hist[j]) {
        const int64_t take = std::min(left, lc.second);
        pbound += take * lc.first;
        left -= take;
        if (left == 0) break;
    }
    pbound = std::max<int64_t>(pbound, 1);
    const size_t nhist = std::max(radix_sort_hist_words(J), radix_sort_hist_words(pbound));
    if ((size_t)J > t->lk_J || (size_t)pbound > t->lk_pairs || nhist > t->lk_hist || (size_t)R > t->lk_R) {
        const size_t nJ = std::max<size_t>(J, t->lk_J), nP = std::max<size_t>(pbound, t->lk_pairs);
        const size_t nH = std::max(nhist, t->lk_hist), nR = std::max<size_t>(R, t->lk_R);
        free_lookup_scratch(t);
        bool ok = true;
        for (int q = 0; q < 2; ++q)
            ok = ok && dmalloc(&t->sk[q], nJ) && dmalloc(&t->sv[q], nJ) && dmalloc(&t->pk[q], nP) &&
                 dmalloc(&t->pv[q], nP);
        ok = ok && dmalloc(&t->flag, nJ + 1) && dmalloc(&t->useg, 2 * nJ) && dmalloc(&t->ufib, nJ) &&
             dmalloc(&t->poff, nJ + 1) && dmalloc(&t->cnt, 2) && dmalloc(&t->uacc, nJ * nR) &&
             dmalloc(&t->pu, nP) && dmalloc(&t->pn, nP) && dmalloc(&t->hist, nH);
        const size_t nC = std::max((nJ + SEG_CH_S - 1) / SEG_CH_S, (nP + SEG_CH - 1) / SEG_CH);   // chunks of the sums
        ok = ok && dmalloc(&t->seg_part, nC * 2 * nR) && dmalloc(&t->seg_info, nC * 4);
        if (!ok) {
            free_lookup_scratch(t);
            return fail(s, KRP_ENOMEM, "sparse lookup scratch allocation failed");
        }
        t->lk_J = nJ;
        t->lk_pairs = nP;
        t->lk_hist = nH;
        t->lk_R = nR;
    }
    const cudaStream_t cs = s->stream;
    const int grid = s->num_sms * 4;
    const uint32_t nfib = (uint32_t)t->nfib[j];
    int fbits = 1;
    while (fbits < 32 && ((uint64_t)1 << fbits) <= nfib) ++fbits;   // fiber ids 0 .. nfib
    const unsigned g0 = (unsigned)std::min<int64_t>((J + 256) / 256, (int64_t)s->num_sms * 8);
    // 1 - 2: samples by fiber, the distinct fibers' runs and summed rows
    fiber_find<<<g0, 256, 0, cs>>>(P, t->sk[0], t->sv[0]);
    count_launch();
    bool in1 = false;
    e = radix_sort_pairs(t->sk[0], t->sv[0], t->sk[1], t->sv[1], t->hist, J, nullptr, fbits, grid, &in1, cs);
    if (e != cudaSuccess) return cuda_check(s, e, "sample sort launch");
    const uint32_t* skey = t->sk[in1 ? 1 : 0];
    const uint32_t* sval = t->sv[in1 ? 1 : 0];
    run_heads<<<g0, 256, 0, cs>>>(skey, J, nfib, t->flag);
    count_launch();
    e = exclusive_scan_u32(t->flag, J + 1, cs);
    if (e != cudaSuccess) return cuda_check(s, e, "run scan launch");
    run_segments<<<g0, 256, 0, cs>>>(skey, J, nfib, t->flag, P.fptr, t->useg, t->ufib, t->poff, t->cnt);
    count_launch();
    const unsigned gs = (unsigned)(s->num_sms * 8);
    uint4* sinfo = reinterpret_cast<uint4*>(t->seg_info);
    SegSrc S2{};   // 2c: acc_u = Σ w_s SA[s, :]
    S2.key = skey;
    S2.sval = sval;
    S2.weight = weight;
    S2.scan = t->flag;
    S2.X = SA;
    S2.out = t->uacc;
    S2.R = R;
    S2.RO = R;
    seg_sums<true><<<gs, 256, 0, cs>>>(S2, t->cnt, t->useg, t->seg_part, sinfo);
    count_launch();
    seg_fix<true><<<gs, 256, 0, cs>>>(S2, t->cnt, t->useg, t->seg_part, sinfo);
    count_launch();
    // 3: the pairs, sorted by mode-j row
    e = exclusive_scan_i64(t->poff, t->cnt, t->cnt + 1, cs);
    if (e != cudaSuccess) return cuda_check(s, e, "pair scan launch");
    pair_fill<<<(unsigned)(s->num_sms * 8), 256, 0, cs>>>(P, t->ufib, t->poff, t->cnt, t->pk[0], t->pv[0], t->pu,
                                                        t->pn);
    count_launch();
    e = radix_sort_pairs(t->pk[0], t->pv[0], t->pk[1], t->pv[1], t->hist, pbound, t->cnt + 1, t->kbits[j], grid,
                         &in1, cs);
    if (e != cudaSuccess) return cuda_check(s, e, "pair sort launch");
    // 4: Y rows (the free pair of sort buffers takes the gathered fiber
    // indices and values)
    const int a1 = in1 ? 1 : 0, b1 = in1 ? 0 : 1;
    pair_gather<<<(unsigned)(s->num_sms * 8), 256, 0, cs>>>(P, t->pv[a1], t->pu, t->pn, t->cnt, t->pk[b1],
                                                           reinterpret_cast<float*>(t->pv[b1]));
    count_launch();
    SegSrc S4{};   // 4b: Y[i, :] = Σ v acc_u
    S4.key = t->pk[a1];
    S4.su = t->pk[b1];
    S4.sv = reinterpret_cast<const float*>(t->pv[b1]);
    S4.X = t->uacc;
    S4.out = t->Y;
    S4.R = R;
    S4.RO = RS;
    seg_sums<false><<<gs, 256, 0, cs>>>(S4, t->cnt, t->useg, t->seg_part, sinfo);
    count_launch();
    seg_fix<false><<<gs, 256, 0, cs>>>(S4, t->cnt, t->useg, t->seg_part, sinfo);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "fiber lookup launch");
    krp_status st = normal_inverse(s, J, SA, flags);
    if (st != KRP_OK) return st;
    const double* Minv = s->solve64 + (size_t)(2 * R * R + R * 128);
    // split-precision samplers apply M⁻¹ on the tensor cores (TF32x3) from R =
    // 64 (below, the SIMT product is the faster); FP32 samplers keep the SIMT
    // product
    if ((s->prec == KRP_PREC_BF16X3 || s->prec == KRP_PREC_TF32X3) && R >= 64 && minv_tc_supported(R))
        e = launch_minv_tc(t->Y, RS, Minv, s->I[j], R, U_out, sumsq, s->als_part, s->status, s->num_sms, s->stream);
    else
        e = launch_apply_minv(t->Y, RS, Minv, s->I[j], R, U_out, sumsq, s->als_part, s->num_sms, s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "apply_minv launch");
    return KRP_OK;
}
}  // namespace krp

extern "C" krp_status krp_solve_sparse(krp_sampler* s, const krp_sptensor* tc, int j, int64_t J,
                                       const int32_t* idx, const float* weight, const float* SA, float* U_out,
                                       int flags) {
    return solve_sparse_impl(s, tc, j, J, idx, weight, SA, U_out, flags, nullptr);
}

namespace krp {
krp_status als_buffers(krp_sampler* s, int64_t J, int32_t** idx, float** w, float** SA, double** sumsq);
}

extern "C" krp_status krp_cp_als_sweep(krp_sampler* s, const krp_sptensor* t, int64_t J, uint64_t seed,
                                       uint64_t draw_base, float* sigma) {
    if (!s || !t || !sigma) return s ? fail(s, KRP_EINVAL, "null argument") : KRP_EINVAL;
    int32_t* idx;
    float *w, *SA;
    double* sumsq;
    krp_status st = als_buffers(s, J, &idx, &w, &SA, &sumsq);
    if (st != KRP_OK) return st;
    const int R = s->R;
    for (int j = 0; j < s->N; ++j) {
        st = krp_sample(s, j, J, seed, draw_base + (uint64_t)j, idx, w, nullptr, SA);
        if (st != KRP_OK) return st;
        // U_j = Y M⁻¹ with its column sums of squares from the same pass
        st = solve_sparse_impl(s, t, j, J, idx, w, SA, s->U[j], KRP_PINV_FALLBACK, sumsq);
        if (st != KRP_OK) return st;
        const int64_t g2 = std::min<int64_t>((s->I[j] + 7) / 8, (int64_t)s->num_sms * 8);
        col_scale<<<(unsigned)g2, 256, 0, s->stream>>>(s->U[j], s->I[j], R, sumsq, sigma); count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(s, e, "normalise launch");
        st = build_tree(s, j, s->prec);
        if (st != KRP_OK) return st;
        s->has_factor[j] = 1;
    }
    return KRP_OK;
}

extern "C" krp_status krp_cp_fit(krp_sampler* s, const krp_sptensor* t, const float* sigma, double* fit_host) {
    if (!s || !t || !sigma || !fit_host) return s ? fail(s, KRP_EINVAL, "null argument") : KRP_EINVAL;
    if (t->N != s->N) return fail(s, KRP_EINVAL, "krp_cp_fit: tensor order differs");
    const int R = s->R, N = s->N;
    int32_t* idx;
    float *w, *SA;
    double* scratch;
    krp_status st = als_buffers(s, 1, &idx, &w, &SA, &scratch);
    if (st != KRP_OK) return st;
    double* inner = s->als_part + (size_t)s->num_sms * 2 * 128;   // one partial per CTA
    FitParams P{};
    for (int k = 0; k < N; ++k) P.U[k] = s->U[k];
    P.coords = t->coords;
    P.vals = t->vals;
    P.sigma = sigma;
    P.nnz = t->nnz;
    P.N = N;
    P.R = R;
    P.out = inner;
    const int64_t g = std::min<int64_t>((t->nnz + 255) / 256, (int64_t)s->num_sms * 8);
    fit_inner<<<(unsigned)g, 256, 0, s->stream>>>(P); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "fit launch");
    std::vector<float> roots((size_t)N * s->Tp), sg(R);
    std::vector<double> parts(g);
    for (int k = 0; k < N; ++k)
        cudaMemcpyAsync(roots.data() + (size_t)k * s->Tp, s->tree[k], s->Tp * 4, cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(sg.data(), sigma, R * 4, cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(parts.data(), inner, g * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "fit sync");
    double in_h = 0.0;
    for (int64_t b = 0; b < g; ++b) in_h += parts[b];
    // ||T̃||² = σᵀ (⊛_k G_k) σ from the trees' roots
    double m2 = 0.0;
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
            double g2 = (double)sg[a] * (double)sg[b];
            for (int k = 0; k < N; ++k)
                g2 *= (double)roots[(size_t)k * s->Tp + tri_index(std::min(a, b), std::max(a, b), R)];
            m2 += g2;
        }
    const double r2 = std::max(t->normT2 - 2.0 * in_h + m2, 0.0);
    *fit_host = 1.0 - sqrt(r2) / sqrt(t->normT2);
    return KRP_OK;
}
