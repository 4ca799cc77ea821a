// a1: segment-tree Gram build (Alg. 3 BuildSampler with F leaf rows, Y = [1];
// Eq. partial_gram; Lemma 3.2 point 1).
//
// Layout: factor U is I x R row-major FP32.  The tree T_{I,F} has L = 2^d
// leaves (ceil(I/F) padded with empty leaves); leaf b covers rows
// [bF, min((b+1)F, I)).  Heap numbering: root 1, children 2h, 2h+1, leaf b is
// node L + b.  Only the root (slot 0) and left children (slot h/2) are stored,
// each as a packed upper triangle with stride Tp floats (see common.cuh).
//
// Kernel 1 (tree_leaves_*): each CTA owns G groups of LB consecutive leaves,
// whose rows stream into shared memory with cp.async (three CTAs per SM
// overlap one another's staging and sums; the exact-decision leaves, one
// heavier CTA per SM, stage the next group while the current one is summed),
// and forms the leaf Grams G^v = U[S(v)]ᵀU[S(v)] (FP32 FMA with 4x4 register
// tiles on the upper triangle, or tcgen05 BF16x3 in tree_build_tc.cu).  Each thread then owns a fixed set of packed entries and
// sums them pairwise up the group (parent = left + right, Alg. 3),
// continuing across groups with a per-entry binary-counter stack, storing
// every left child it creates.  The CTA's subtree root goes to scratch.
// Kernel 2 (tree_up): the same pairwise sums over LBB nodes per CTA for the
// levels above, until the root.
//
// Exact-decision mode (KRP_PREC_EXACT): the leaf Grams are accumulated
// without rounding error (see leaf_grams_fp32), every stored slot keeps the
// low part of its double-float value in a second array (tree_lo), and the
// top levels are also written delta-encoded (build_dtop), for the descent's
// near-edge decisions.
#include "common.cuh"
#include "internal.h"
#include "tree_reduce.cuh"

#include <algorithm>

namespace krp {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage rows [row0, row0 + nrows) of U (zero beyond I) into sU (row stride R).
// VEC: 16-byte cp.async (needs R % 4 == 0 so every chunk is 16-byte aligned);
// otherwise 4-byte cp.async.  The caller commits and waits.
template <bool VEC>
__device__ __forceinline__ void stage_rows(float* sU, const float* __restrict__ U, int64_t I, int R,
                                           int64_t row0, int nrows) {
    const int64_t nf = (int64_t)nrows * R;
    const int64_t valid = max((int64_t)0, min(nf, (I - row0) * (int64_t)R));
    const float* src = U + row0 * (int64_t)R;
    if (VEC) {
        for (int64_t c = threadIdx.x; c < nf / 4; c += blockDim.x) {
            const int64_t off = 4 * c;
            const int bytes = (int)max((int64_t)0, min((int64_t)4, valid - off)) * 4;
            cp_async16(sU + off, bytes > 0 ? (const void*)(src + off) : (const void*)U, bytes);
        }
    } else {
        for (int64_t e = threadIdx.x; e < nf; e += blockDim.x)
            cp_async4(sU + e, e < valid ? (const void*)(src + e) : (const void*)U, e < valid ? 4 : 0);
    }
}

// Anchor of an exactly accumulated sum of products a_f b_f over one leaf:
// M = 1.5 * 2^e with 2^e > 4.5 sqrt(na) sqrt(nb) (na, nb the FP32 sums of
// squares of the two columns).  By Cauchy-Schwarz every partial sum lies
// within 2^e / 4 of 0, so M + partial stays in M's binade [2^e, 2^(e+1)),
// where FP32 numbers are multiples of one quantum ulp(M).
__device__ __forceinline__ float sum_anchor(float na, float nb) {
    int e;
    frexpf(4.5f * sqrtf(na) * sqrtf(nb), &e);
    return ldexpf(1.5f, e);
}

// Leaf Grams of LB leaves (F rows each) from sU into sG (LB x Tp), FP32 FMA,
// 4x4 register tiles over the upper triangle of 4-column blocks, two entries
// of a tile row per paired (f32x2) instruction.
// EXACT: each entry is accumulated on its anchor M (above), s = M + sum:
// t = fma(a, b, s) keeps a b to the quantum, s - t = -(what was kept) is
// exact (same binade), r = fma(a, b, s - t) is what was dropped (to 2^-24 of
// itself, |r| <= ulp(M)), and c accumulates r.  The entry is then (s - M) +
// c, written as a double-float (hi into sG, lo into sGlo): its error is at
// most F (F + 1) 2^-24 ulp(M) <= 9 F (F + 1) 2^-47 sqrt(G_ii G_jj), against
// FP32's 2^-24 F |partial sums|.
template <int LB, bool VEC, bool EXACT = false>
__device__ __forceinline__ void leaf_grams_fp32(const float* sU, float* sG, int R, int F, int Tp,
                                                float* sGlo = nullptr) {
    const int nt = (R + 3) >> 2;
    const int ntile = nt * (nt + 1) / 2;
    for (int task = threadIdx.x; task < LB * ntile; task += blockDim.x) {
        const int leaf = task / ntile;
        int t = task - leaf * ntile;
        int ti = 0;
        while (t >= nt - ti) {
            t -= nt - ti;
            ++ti;
        }
        const int tj = ti + t;
        const float* base = sU + (size_t)leaf * F * R;
        auto load = [&](int f, float* a, float* b) {
            if (VEC) {
                const float4 va = *reinterpret_cast<const float4*>(base + f * R + 4 * ti);
                const float4 vb = *reinterpret_cast<const float4*>(base + f * R + 4 * tj);
                a[0] = va.x; a[1] = va.y; a[2] = va.z; a[3] = va.w;
                b[0] = vb.x; b[1] = vb.y; b[2] = vb.z; b[3] = vb.w;
            } else {
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    a[x] = (4 * ti + x < R) ? base[f * R + 4 * ti + x] : 0.f;
                    b[x] = (4 * tj + x < R) ? base[f * R + 4 * tj + x] : 0.f;
                }
            }
        };
        // acc[x][h] holds entries (x, 2h) and (x, 2h + 1) of the tile
        float2 acc[4][2], cor[4][2];
        float na[4] = {0.f, 0.f, 0.f, 0.f}, nb[4] = {0.f, 0.f, 0.f, 0.f};
        if (EXACT) {
            float2 na2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, nb2[2] = {na2[0], na2[0]};
            for (int f = 0; f < F; ++f) {
                float a[4], b[4];
                load(f, a, b);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 ah = make_float2(a[2 * h], a[2 * h + 1]), bh = make_float2(b[2 * h], b[2 * h + 1]);
                    na2[h] = ffma2(ah, ah, na2[h]);
                    nb2[h] = ffma2(bh, bh, nb2[h]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                na[2 * h] = na2[h].x;
                na[2 * h + 1] = na2[h].y;
                nb[2 * h] = nb2[h].x;
                nb[2 * h + 1] = nb2[h].y;
            }
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                acc[x][h] = EXACT ? make_float2(sum_anchor(na[x], nb[2 * h]), sum_anchor(na[x], nb[2 * h + 1]))
                                  : make_float2(0.f, 0.f);
                cor[x][h] = make_float2(0.f, 0.f);
            }
        for (int f = 0; f < F; ++f) {
            float a[4], b[4];
            load(f, a, b);
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 ax = make_float2(a[x], a[x]), bh = make_float2(b[2 * h], b[2 * h + 1]);
                    if (EXACT) {
                        const float2 tt = ffma2(ax, bh, acc[x][h]);
                        const float2 nq = fsub2(acc[x][h], tt);
                        cor[x][h] = fadd2(cor[x][h], ffma2(ax, bh, nq));
                        acc[x][h] = tt;
                    } else {
                        acc[x][h] = ffma2(ax, bh, acc[x][h]);
                    }
                }
        }
        float* g = sG + (size_t)leaf * Tp;
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const int i = 4 * ti + x, j = 4 * tj + y;
                const float v = (y & 1) ? acc[x][y >> 1].y : acc[x][y >> 1].x;
                if (i <= j && j < R) {
                    if (EXACT) {
                        const float hi = v - sum_anchor(na[x], nb[y]);   // exact: same binade
                        float sh, sl;
                        two_sum(hi, (y & 1) ? cor[x][y >> 1].y : cor[x][y >> 1].x, sh, sl);
                        g[tri_index(i, j, R)] = sh;
                        sGlo[(size_t)leaf * Tp + tri_index(i, j, R)] = sl;
                    } else {
                        g[tri_index(i, j, R)] = v;
                    }
                }
            }
    }
}

// Write the staged rows [row0, row0 + nrows) back out to `dst` (the sampler's
// own copy of the factor), so that a factor update reads its source once.
template <bool VEC>
__device__ __forceinline__ void copy_rows_out(const float* sU, float* __restrict__ dst, int64_t I, int R,
                                              int64_t row0, int nrows) {
    const int64_t valid = max((int64_t)0, min((int64_t)nrows * R, (I - row0) * (int64_t)R));
    float* out = dst + row0 * (int64_t)R;
    if (VEC) {
        for (int64_t c = threadIdx.x; c < valid / 4; c += blockDim.x)
            reinterpret_cast<float4*>(out)[c] = reinterpret_cast<const float4*>(sU)[c];
        for (int64_t e = (valid / 4) * 4 + threadIdx.x; e < valid; e += blockDim.x) out[e] = sU[e];
    } else {
        for (int64_t e = threadIdx.x; e < valid; e += blockDim.x) out[e] = sU[e];
    }
}

// Block blk: leaves [blk G LB, (blk+1) G LB), subtree root to top slot blk.
// EXACT: exactly accumulated leaf Grams, low parts stored into tree_lo.
template <int LB, bool VEC, bool EXACT = false>
__device__ __forceinline__ void tree_leaves_fp32_body(const float* __restrict__ U, int64_t I, int R, int F, int64_t L,
                                                      int G, int Tp, float* __restrict__ tree,
                                                      float* __restrict__ top, float* __restrict__ copy_to,
                                                      int64_t blk, float* __restrict__ tree_lo = nullptr) {
    // DB: the exact-decision leaves (one CTA of heavier work per SM) stage the
    // next group while the current one is summed; the FP32 leaves keep one
    // stage and three CTAs per SM, whose staging overlaps the others' sums.
    constexpr bool DB = VEC && EXACT;
    extern __shared__ __align__(16) float smem[];
    const int rows = LB * F;
    const int T = tri_size(R);
    float* sU0 = smem;
    float* sU1 = sU0 + (size_t)rows * R;
    float* sG = (DB ? sU1 : sU0) + (size_t)rows * R;
    float* sGlo = EXACT ? sG + (size_t)LB * Tp : nullptr;
    float* stk = sG + (size_t)(EXACT ? 2 : 1) * LB * Tp;
    for (int e = threadIdx.x; e < LB * Tp; e += blockDim.x)
        if (e % Tp >= T) {  // packed tail stays zero
            sG[e] = 0.f;
            if (EXACT) sGlo[e] = 0.f;
        }
    const int64_t leaf0 = blk * G * LB;
    stage_rows<VEC>(sU0, U, I, R, leaf0 * F, rows);
    cp_async_commit();
    for (int g = 0; g < G; ++g) {
        float* cur = (DB && (g & 1)) ? sU1 : sU0;
        if (DB) {
            if (g + 1 < G) {
                stage_rows<VEC>((g & 1) ? sU0 : sU1, U, I, R, (leaf0 + (int64_t)(g + 1) * LB) * F, rows);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (copy_to) copy_rows_out<VEC>(cur, copy_to, I, R, (leaf0 + (int64_t)g * LB) * F, rows);
        leaf_grams_fp32<LB, VEC, EXACT>(cur, sG, R, F, Tp, sGlo);
        __syncthreads();
        if (EXACT) {   // each leaf's trace after its packed triangle (summed up the tree with the rest)
            for (int l = threadIdx.x; l < LB; l += blockDim.x) {
                float t = 0.f;
                for (int a = 0; a < R; ++a) t += sG[l * Tp + tri_index(a, a, R)];
                sG[l * Tp + T] = t;
            }
            __syncthreads();
        }
        reduce_group<LB, true, EXACT>(sG, stk, tree, top, L, leaf0 + (int64_t)g * LB, g, G, Tp, blk, sGlo, tree_lo);
        if (!DB && g + 1 < G) {
            __syncthreads();
            stage_rows<VEC>(sU0, U, I, R, (leaf0 + (int64_t)(g + 1) * LB) * F, rows);
            cp_async_commit();
        }
    }
}

template <int LB, bool VEC, bool EXACT>
__global__ void __launch_bounds__(288, EXACT ? 2 : 3) tree_leaves_fp32(const float* __restrict__ U, int64_t I, int R, int F,
                                                        int64_t L, int G, int Tp, float* __restrict__ tree,
                                                        float* __restrict__ top, float* __restrict__ copy_to,
                                                        float* __restrict__ tree_lo) {
    tree_leaves_fp32_body<LB, VEC, EXACT>(U, I, R, F, L, G, Tp, tree, top, copy_to, blockIdx.x, tree_lo);
}

// Entry e of node `node` of an input level as a double-float pair: the leaf
// kernel's (hi, lo) FP32 pairs as they are, FP64 values split exactly enough
// (hi = FP32 rounding, lo = FP32 rounding of the rest).
__device__ __forceinline__ void load_up(bool from_pairs, const float* __restrict__ in_pairs,
                                        const double* __restrict__ in64, int64_t node, int Tp, int e, float& hi,
                                        float& lo) {
    if (from_pairs) {
        hi = in_pairs[(node * 2) * Tp + e];
        lo = in_pairs[(node * 2 + 1) * Tp + e];
    } else {
        const double x = in64[node * Tp + e];
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
}

// Index of the entry of an ascending prefix array whose range holds x.
__device__ __forceinline__ int prefix_find(const int64_t* __restrict__ pre, int n, int64_t x) {
    int lo = 0, hi = n - 1;  // pre[0] = 0 <= x < pre[n]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Batched leaf kernel: CTA b builds block b - prefix[t] of tree t (the tree
// whose block range holds b), with LB leaves per group and the tree's own G.
template <int LB, bool VEC>
__global__ void __launch_bounds__(288, 3) tree_leaves_fp32_batch(const TreeDesc* __restrict__ trees,
                                                              const int64_t* __restrict__ prefix, int ntrees) {
    const int t = prefix_find(prefix, ntrees, blockIdx.x);
    const TreeDesc& d = trees[t];
    tree_leaves_fp32_body<LB, VEC>(d.src, d.I, d.R, d.F, d.L, d.G, d.Tp, d.tree, d.top,
                                   d.copy_to, (int64_t)blockIdx.x - prefix[t]);
}

// Batched level sums: CTA b sums `lbb` nodes of tree t's input level (t found
// as above) in the same pairwise order as tree_up<lbb>.
template <bool FROM_PAIRS>
__global__ void tree_up_batch(const UpDesc* __restrict__ ups, const int64_t* __restrict__ prefix, int ntrees) {
    const int t = prefix_find(prefix, ntrees, blockIdx.x);
    const UpDesc& u = ups[t];
    const int64_t cta = (int64_t)blockIdx.x - prefix[t];
    const int lbb = u.lbb, Tp = u.Tp;
    const int64_t first = cta * lbb;
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        float vh[16], vl[16];
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            vh[l] = vl[l] = 0.f;
            if (l < lbb) load_up(FROM_PAIRS, u.in_pairs, u.in64, first + l, Tp, e, vh[l], vl[l]);
        }
        int64_t h = u.n_in + first;
#pragma unroll
        for (int n = 16; n > 1; n >>= 1) {
            if (n > lbb) continue;
            h >>= 1;
#pragma unroll
            for (int l = 0; l < n / 2; ++l) {
                df_add(vh[2 * l], vl[2 * l], vh[2 * l + 1], vl[2 * l + 1], vh[l], vl[l]);
                store_node(u.tree, h + l, Tp, e, vh[l]);
            }
        }
        u.out[(size_t)cta * Tp + e] = (double)vh[0] + (double)vl[0];
    }
}

// Levels above the leaf kernel: LBB nodes per CTA from `in` (a full tree
// level with n_in nodes, heap ids n_in..2 n_in - 1; either the leaf kernel's
// (hi, lo) FP32 pairs or FP64 values) to one node per CTA in `out`, as the
// exact FP64 value of a double-float sum (the leaf kernel's in-CTA sums are
// double-float too, ~2^-44 relative; GB300 runs FP64 at ~1/64 of FP32, which
// made FP64 adds the bound of the first of these levels at large R).  Stores
// the FP32-rounded sum of every left child created.
template <int LBB, bool FROM_PAIRS>
__global__ void tree_up(const float* __restrict__ in_pairs, const double* __restrict__ in64, int64_t n_in, int Tp,
                        float* __restrict__ tree, double* __restrict__ out, float* __restrict__ tree_lo) {
    const int64_t first = (int64_t)blockIdx.x * LBB;
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        float vh[LBB], vl[LBB];
#pragma unroll
        for (int l = 0; l < LBB; ++l) load_up(FROM_PAIRS, in_pairs, in64, first + l, Tp, e, vh[l], vl[l]);
        int64_t h = n_in + first;
#pragma unroll
        for (int n = LBB; n > 1; n >>= 1) {
            h >>= 1;
#pragma unroll
            for (int l = 0; l < n / 2; ++l) {
                df_add(vh[2 * l], vl[2 * l], vh[2 * l + 1], vl[2 * l + 1], vh[l], vl[l]);
                store_node2(tree, tree_lo, h + l, Tp, e, vh[l], vl[l]);
            }
        }
        out[(size_t)blockIdx.x * Tp + e] = (double)vh[0] + (double)vl[0];
    }
}

// Exact FP64 Gram UᵀU for small factors (products of FP32 values are exact in
// FP64; sums in FP64): CTA (x, y) reduces row chunk x for packed entries
// y*256 .. y*256+255, one entry per thread, into partial x.
__global__ void __launch_bounds__(256) gram64_partial(const float* __restrict__ U, int64_t I, int R, int Tp,
                                                      int64_t rows_per_cta, double* __restrict__ part,
                                                      bool with_trace) {
    extern __shared__ __align__(16) float sU[];  // 64 x R
    const int T = tri_size(R);
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(I, r0 + rows_per_cta);
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    int ei = 0, ej = 0;
    if (e < T) {
        int rem = e;
        while (rem >= R - ei) {
            rem -= R - ei;
            ++ei;
        }
        ej = ei + rem;
    }
    double acc = 0.0;
    for (int64_t b = r0; b < r1; b += 64) {
        const int nr = (int)min((int64_t)64, r1 - b);
        __syncthreads();
        for (int x = threadIdx.x; x < 64 * R; x += blockDim.x) sU[x] = (x / R < nr) ? U[b * R + x] : 0.f;
        __syncthreads();
        if (e < T)
            for (int r = 0; r < nr; ++r) acc = fma((double)sU[r * R + ei], (double)sU[r * R + ej], acc);
        else if (e == T && with_trace)   // the trace after the packed triangle
            for (int x = 0; x < nr * R; ++x) acc = fma((double)sU[x], (double)sU[x], acc);
    }
    if (e < Tp) part[(size_t)blockIdx.x * Tp + e] = (e < T || (e == T && with_trace)) ? acc : 0.0;
}

// Sum the partials in a fixed order into the FP64 root; also refresh the
// stored FP32 root (slot 0) with the rounding of the exact value.
__global__ void gram64_finish(const double* __restrict__ part, int nparts, int Tp, double* __restrict__ root64,
                              float* __restrict__ slot0, float* __restrict__ slot0_lo) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Tp; e += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int p = 0; p < nparts; ++p) a += part[(size_t)p * Tp + e];
        root64[e] = a;
        slot0[e] = (float)a;
        if (slot0_lo) slot0_lo[e] = (float)(a - (double)(float)a);
    }
}

// Delta-encoded top of a tree for the exact-decision descent (levels < Ke):
// dtop = [root | D_1 | ... | D_{2^Ke - 1}] with the tree's slot numbering
// (slot c at offset c Tp), D_c = G_{2c} - alpha_c G_c (node_alpha) formed in
// double-float from the tree's (hi, lo) slots and rounded to FP32.  G_c of a
// right child is its parent's Gram minus its left sibling's, walked down from
// the root.  After the packed triangle each D slot holds kappa_c = max_ab
// |D_ab| / sqrt(g_a g_b) (g the root's diagonal), which bounds the descent's
// FP32 rounding error on w^T D_c; the root slot keeps its trace.  One CTA per
// slot.
__global__ void build_dtop(const float* __restrict__ tree, const float* __restrict__ tlo, int64_t I, int F,
                           int64_t L, int R, int Tp, float* __restrict__ dtop) {
    __shared__ unsigned kmax;   // kappa_c as FP32 bits (non-negative floats order as integers)
    const int64_t c = blockIdx.x;
    const int T = tri_size(R);
    if (threadIdx.x == 0) kmax = 0u;
    __syncthreads();
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        if (c == 0) {
            dtop[e] = tree[e];
            continue;
        }
        if (e >= T) {
            if (e > T) dtop[c * Tp + e] = 0.f;
            continue;
        }
        df G{tree[e], tlo[e]};
        const int dc = 63 - __clzll((unsigned long long)c);
        for (int t = 1; t <= dc; ++t) {
            const int64_t n = c >> (dc - t);
            const int64_t par = n >> 1;   // left child of par is stored at slot par
            const df gl{tree[par * Tp + e], tlo[par * Tp + e]};
            G = (n & 1) ? df_add(G, df_neg(gl)) : gl;
        }
        const df GL{tree[c * Tp + e], tlo[c * Tp + e]};
        const df D = df_add(GL, df_neg(df_mul_f(G, node_alpha(c, dc, L, F, I))));
        const float d = D.hi + D.lo;
        dtop[c * Tp + e] = d;
        int i = 0, rem = e;
        while (rem >= R - i) {
            rem -= R - i;
            ++i;
        }
        const float den = sqrtf(tree[tri_index(i, i, R)]) * sqrtf(tree[tri_index(i + rem, i + rem, R)]);
        const float k = den > 0.f ? fabsf(d) / den : (d != 0.f ? INFINITY : 0.f);
        atomicMax(&kmax, __float_as_uint(k));
    }
    __syncthreads();
    // a little above the largest ratio: covers the roundings of the ratio itself
    if (c > 0 && threadIdx.x == 0) dtop[c * Tp + T] = __uint_as_float(kmax) * 1.0001f;
}

cudaError_t launch_build_dtop(const krp_sampler* s, int j, cudaStream_t st) {
    const int Ke = s->Ke[j];
    build_dtop<<<(unsigned)((int64_t)1 << Ke), 256, 0, st>>>(s->tree[j], s->tree_lo[j], s->I[j], s->F, s->L[j],
                                                           s->R, s->Tp, s->dtop[j]);
    count_launch();
    return cudaGetLastError();
}

// BF16x3 and TF32x3 tensor-core leaf kernels (tree_build_tc.cu).
bool tree_tc_supported(int R, int F);
bool tree_tc_pipelined(int R, int F, const float* U);
void tree_tc_geometry(int R, int F, int64_t L, int Tp, bool pipelined, int* LB_out, int* G_out, size_t* smem_out,
                      bool tf32);
cudaError_t launch_tree_leaves_tc(const float* U, int64_t I, int R, int F, int64_t L, int LB, int G, int Tp,
                                  float* tree, float* top, float* copy_to, int* status, int64_t ctas, size_t smem,
                                  bool pipelined, int num_sms, cudaStream_t st, bool tf32);

namespace {

template <int LB, bool VEC, bool EXACT>
cudaError_t launch_leaves(const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp, float* tree,
                          float* top, float* copy_to, int64_t ctas, int threads, size_t smem, cudaStream_t st,
                          float* tree_lo) {
    auto k = tree_leaves_fp32<LB, VEC, EXACT>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<(unsigned)ctas, threads, smem, st>>>(U, I, R, F, L, G, Tp, tree, top, copy_to, tree_lo); count_launch();
    return cudaGetLastError();
}

template <int LB>
cudaError_t dispatch_vec(bool vec, const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp,
                         float* tree, float* top, float* copy_to, int64_t ctas, int threads, size_t smem,
                         cudaStream_t st, float* tree_lo) {
    if (tree_lo)
        return vec ? launch_leaves<LB, true, true>(U, I, R, F, L, G, Tp, tree, top, copy_to, ctas, threads, smem, st,
                                                   tree_lo)
                   : launch_leaves<LB, false, true>(U, I, R, F, L, G, Tp, tree, top, copy_to, ctas, threads, smem,
                                                    st, tree_lo);
    return vec ? launch_leaves<LB, true, false>(U, I, R, F, L, G, Tp, tree, top, copy_to, ctas, threads, smem, st,
                                                nullptr)
               : launch_leaves<LB, false, false>(U, I, R, F, L, G, Tp, tree, top, copy_to, ctas, threads, smem, st,
                                                 nullptr);
}

}  // namespace

// Leaf-kernel geometry: LB leaves per group (power of two, <= 16, <= L, one
// group of rows <= 32 KB), G groups per CTA (power of two, <= 8).  Exact
// leaves keep a second LB x Tp array of low parts and stay within 110 KB, so
// that two CTAs share an SM.
void tree_geometry(int R, int F, int64_t L, int Tp, bool vec, int* LB_out, int* G_out, int* threads_out,
                   size_t* smem_out, bool exact = false) {
    const size_t leaf_bytes = (size_t)F * R * 4;
    int LB = 1;
    while (LB < 16 && (int64_t)LB * 2 <= L && (size_t)LB * 2 * leaf_bytes <= 32 * 1024) LB *= 2;
    const int nt = (R + 3) / 4;
    const int ntile = nt * (nt + 1) / 2;
    int threads = std::min(288, std::max(64, ((LB * ntile + 31) / 32) * 32));
    const int64_t groups = L / LB;
    int G = 1;
    auto smem_of = [&](int g) {
        int lv = 0;
        while ((1 << lv) < g) ++lv;
        return (size_t)(vec && exact ? 2 : 1) * LB * leaf_bytes + (size_t)(exact ? 2 : 1) * LB * Tp * 4 +
               (size_t)2 * (lv + 1) * Tp * 4;
    };
    const size_t cap = exact ? 110 * 1024 : 160 * 1024;
    while (G < 8 && (int64_t)G * 2 <= groups && smem_of(G * 2) <= cap) G *= 2;
    *LB_out = LB;
    *G_out = G;
    *threads_out = threads;
    *smem_out = smem_of(G);
}

cudaError_t launch_leaves_batch(const TreeDesc* trees_dev, const int64_t* block_prefix_dev, int ntrees,
                                int64_t nblocks, int LB, int Rmax, int Fmax, int Tpmax, int Gmax, bool vec,
                                cudaStream_t st) {
    int lv = 0;
    while ((1 << lv) < Gmax) ++lv;
    const size_t leaf_bytes = (size_t)Fmax * Rmax * 4;
    const size_t smem = (size_t)LB * leaf_bytes + (size_t)LB * Tpmax * 4 + (size_t)2 * (lv + 1) * Tpmax * 4;
    cudaError_t e = cudaSuccess;
#define KRP_LB(LBV)                                                                                              \
    {                                                                                                            \
        auto k = vec ? tree_leaves_fp32_batch<LBV, true> : tree_leaves_fp32_batch<LBV, false>;                   \
        if (smem > 48 * 1024) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e == cudaSuccess) {                                                                                  \
            k<<<(unsigned)nblocks, 288, smem, st>>>(trees_dev, block_prefix_dev, ntrees);                         \
            count_launch();                                                                                      \
            e = cudaGetLastError();                                                                              \
        }                                                                                                        \
    }
    switch (LB) {
        case 1: KRP_LB(1) break;
        case 2: KRP_LB(2) break;
        case 4: KRP_LB(4) break;
        default: KRP_LB(8) break;
    }
#undef KRP_LB
    return e;
}

cudaError_t launch_up_batch(const UpDesc* ups_dev, const int64_t* cta_prefix_dev, int ntrees, int64_t nctas,
                            int Tpmax, bool from_pairs, cudaStream_t st) {
    const int threads = std::min(512, std::max(64, ((Tpmax + 31) / 32) * 32));
    if (from_pairs)
        tree_up_batch<true><<<(unsigned)nctas, threads, 0, st>>>(ups_dev, cta_prefix_dev, ntrees);
    else
        tree_up_batch<false><<<(unsigned)nctas, threads, 0, st>>>(ups_dev, cta_prefix_dev, ntrees);
    count_launch();
    return cudaGetLastError();
}

krp_status build_tree(krp_sampler* s, int j, int precision, const float* src) {
    // src: rows to build from; if it is not the sampler's copy, the leaf kernel
    // also writes them into s->U[j].
    float* copy_to = (src && src != s->U[j]) ? s->U[j] : nullptr;
    if (!src) src = s->U[j];
    const int R = s->R, F = s->F, Tp = s->Tp;
    const int64_t I = s->I[j], L = s->L[j];
    const bool vec = (R % 4) == 0;
    // exact-decision samplers build every tree with exactly accumulated leaves
    float* tree_lo = s->exact ? s->tree_lo[j] : nullptr;
    // BF16x3 takes the tensor cores where the pipelined kernel applies (F R a
    // multiple of 4, its stages fitting); elsewhere (R = 25, F = R = 128) the
    // FP32 leaves are faster and more accurate.  TF32x3 always takes the
    // non-pipelined tensor-core kernel.
    const bool tf32 = precision == KRP_PREC_TF32X3;
    const bool tc_pipe = !s->exact && precision == KRP_PREC_BF16X3 && tree_tc_pipelined(R, F, src);
    const bool tc = !s->exact && (tc_pipe || (tf32 && tree_tc_supported(R, F)));
    int LB, G, threads = 128;
    size_t smem;
    if (tc)
        tree_tc_geometry(R, F, L, Tp, tc_pipe, &LB, &G, &smem, tf32);
    else
        tree_geometry(R, F, L, Tp, vec, &LB, &G, &threads, &smem, s->exact);
    const int64_t ctas = L / ((int64_t)LB * G);
    const int T = tri_size(R);
    const bool exact_root = (double)I * T <= (double)(1 << 22);
    const int nparts = exact_root ? (int)std::min<int64_t>((I + 255) / 256, 512) : 0;
    // scratch (floats): leaf-kernel roots as (hi, lo) pairs, then FP64 space for
    // two ping-pong levels or the exact-root partials
    const size_t pairs = (size_t)ctas * 2 * Tp;
    const size_t f64 = std::max<size_t>((size_t)2 * (ctas / 2 + 2) * Tp, (size_t)nparts * Tp);
    const size_t need = pairs + 2 * f64;
    if (need > s->build_scratch_floats) {
        if (s->build_scratch) cudaFree(s->build_scratch);
        s->build_scratch = nullptr;
        s->build_scratch_floats = 0;
        if (cudaMalloc(&s->build_scratch, need * sizeof(float)) != cudaSuccess)
            return fail(s, KRP_ENOMEM, "tree build scratch allocation failed");
        s->build_scratch_floats = need;
    }
    float* top = s->build_scratch;
    double* up0 = reinterpret_cast<double*>(s->build_scratch + pairs);  // pairs is even: 8-byte aligned
    double* up1 = up0 + (size_t)(ctas / 2 + 2) * Tp;
    if (tc) {
        const cudaError_t e = launch_tree_leaves_tc(src, I, R, F, L, LB, G, Tp, s->tree[j], top, copy_to, s->status,
                                                    ctas, smem, tc_pipe, s->num_sms, s->stream, tf32);
        if (e != cudaSuccess) return cuda_check(s, e, "tensor-core tree leaf kernel launch");
    } else {
        cudaError_t e;
        switch (LB) {
            case 1: e = dispatch_vec<1>(vec, src, I, R, F, L, G, Tp, s->tree[j], top, copy_to, ctas, threads, smem, s->stream, tree_lo); break;
            case 2: e = dispatch_vec<2>(vec, src, I, R, F, L, G, Tp, s->tree[j], top, copy_to, ctas, threads, smem, s->stream, tree_lo); break;
            case 4: e = dispatch_vec<4>(vec, src, I, R, F, L, G, Tp, s->tree[j], top, copy_to, ctas, threads, smem, s->stream, tree_lo); break;
            case 8: e = dispatch_vec<8>(vec, src, I, R, F, L, G, Tp, s->tree[j], top, copy_to, ctas, threads, smem, s->stream, tree_lo); break;
            default: e = dispatch_vec<16>(vec, src, I, R, F, L, G, Tp, s->tree[j], top, copy_to, ctas, threads, smem, s->stream, tree_lo); break;
        }
        if (e != cudaSuccess) return cuda_check(s, e, "tree leaf kernel launch");
    }
    // levels above the leaf kernel, in FP64, down to the FP64 root
    int64_t n = ctas;
    const int up_threads = std::min(512, std::max(64, ((Tp + 31) / 32) * 32));
    bool first = true;
    const double* in64 = nullptr;
    double* outs[2] = {up0, up1};
    int which = 0;
    do {
        const int64_t lbb = std::min<int64_t>(16, n);
        const unsigned grid = (unsigned)(n / lbb);
        double* out = (n / lbb == 1) ? s->root64[j] : outs[which];
#define KRP_UP(LBBV)                                                                                          \
    if (first)                                                                                                \
        tree_up<LBBV, true><<<grid, up_threads, 0, s->stream>>>(top, nullptr, n, Tp, s->tree[j], out, tree_lo); \
    else                                                                                                      \
        tree_up<LBBV, false><<<grid, up_threads, 0, s->stream>>>(nullptr, in64, n, Tp, s->tree[j], out, tree_lo);
        switch (lbb) {
            case 1: KRP_UP(1) break;
            case 2: KRP_UP(2) break;
            case 4: KRP_UP(4) break;
            case 8: KRP_UP(8) break;
            default: KRP_UP(16) break;
        }
#undef KRP_UP
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(s, e, "tree up kernel launch");
        in64 = out;
        which ^= 1;
        first = false;
        n /= lbb;
    } while (n > 1);
    // small factors: exact FP64 root Gram (replaces the summed one)
    if (exact_root) {
        const int64_t rpc = (I + nparts - 1) / nparts;
        const dim3 grid(nparts, (Tp + 255) / 256);
        gram64_partial<<<grid, 256, 64 * R * 4, s->stream>>>(s->U[j], I, R, Tp, rpc, up0, tree_lo != nullptr);
        count_launch();
        gram64_finish<<<(Tp + 255) / 256, 256, 0, s->stream>>>(up0, nparts, Tp, s->root64[j], s->tree[j], tree_lo);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(s, e, "exact root Gram launch");
    }
    if (s->exact) {
        const cudaError_t e = launch_build_dtop(s, j, s->stream);
        if (e != cudaSuccess) return cuda_check(s, e, "delta-encoded top launch");
    }
    return KRP_OK;
}

}  // namespace krp
