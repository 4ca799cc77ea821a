// Shared by the leaf kernels of the segment-tree build (Alg. 3): storing a
// node's packed triangle, double-float addition, and the pairwise sums of one
// group of leaf Grams continued across groups with a binary-counter stack.
#pragma once

#include "common.cuh"

namespace krp {

__device__ __forceinline__ void store_node(float* __restrict__ tree, int64_t h, int Tp, int e, float v) {
    if (tree_stored(h)) tree[tree_slot(h) * Tp + e] = v;
}
// The same with the low part of a double-float value into `tree_lo` (the
// exact-decision mode's second array), when given.
__device__ __forceinline__ void store_node2(float* __restrict__ tree, float* __restrict__ tree_lo, int64_t h, int Tp,
                                           int e, float hi, float lo) {
    if (tree_stored(h)) {
        tree[tree_slot(h) * Tp + e] = hi;
        if (tree_lo) tree_lo[tree_slot(h) * Tp + e] = lo;
    }
}

// Double-float addition (Knuth TwoSum, then a fast renormalisation): the pair
// (hi, lo) carries the sum to about 2^-44 relative, so that the sums above the
// leaves add no rounding error of their own; hi is the FP32-rounded sum.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
    const float s = ah + bh;
    const float bb = s - ah;
    const float err = (ah - (s - bb)) + (bh - bb);
    const float t = err + al + bl;
    h = s + t;
    l = t - (h - s);
}

// Pairwise sums of one group's LB leaf Grams (entry e), then the binary-counter
// merge across the CTA's groups, in double-float (DF) or plain FP32 (for leaf
// Grams that carry ~1e-5 error of their own, where the sums' 2^-24 per level
// is immaterial).  GDF = false keeps DF for the merge across groups and the
// levels above but sums inside a group in FP32: the few roundings of each
// group's sum are independent across the many groups of a tree, so they reach
// the root as ~2^-24 / sqrt(groups) relative, the size of the leaves' own FP32
// error there.  Stores the FP32 value of every left child created (and its low
// part into tree_lo, if given); the subtree root of the G groups (the CTA's,
// or the block `top_slot` of a persistent CTA) goes to top as (hi, lo).
// sGlo: the leaf Grams' low parts (exactly accumulated leaves), or nullptr.
template <int LB, bool DF = true, bool GDF = DF>
__device__ __forceinline__ void reduce_group(const float* sG, float* stk, float* __restrict__ tree,
                                             float* __restrict__ top, int64_t L, int64_t first_leaf,
                                             int g, int G, int Tp, int64_t top_slot,
                                             const float* sGlo = nullptr, float* __restrict__ tree_lo = nullptr) {
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        float vh[LB], vl[LB];
#pragma unroll
        for (int l = 0; l < LB; ++l) {
            vh[l] = sG[l * Tp + e];
            vl[l] = sGlo ? sGlo[l * Tp + e] : 0.f;
        }
        int64_t h = L + first_leaf;
#pragma unroll
        for (int l = 0; l < LB; ++l) store_node2(tree, tree_lo, h + l, Tp, e, vh[l], vl[l]);
#pragma unroll
        for (int n = LB; n > 1; n >>= 1) {
            h >>= 1;
#pragma unroll
            for (int l = 0; l < n / 2; ++l) {
                if (GDF)
                    df_add(vh[2 * l], vl[2 * l], vh[2 * l + 1], vl[2 * l + 1], vh[l], vl[l]);
                else
                    vh[l] = vh[2 * l] + vh[2 * l + 1];
                store_node2(tree, tree_lo, h + l, Tp, e, vh[l], vl[l]);
            }
        }
        float hi = vh[0], lo = vl[0];
        int idx = g, lvl = 0;
        while (idx & 1) {
            if (DF)
                df_add(stk[(2 * lvl) * Tp + e], stk[(2 * lvl + 1) * Tp + e], hi, lo, hi, lo);
            else
                hi = stk[(2 * lvl) * Tp + e] + hi;
            h >>= 1;
            idx >>= 1;
            ++lvl;
            store_node2(tree, tree_lo, h, Tp, e, hi, lo);
        }
        if (G > 1) {   // with one group the stack is never read (and may have no space)
            stk[(2 * lvl) * Tp + e] = hi;
            stk[(2 * lvl + 1) * Tp + e] = lo;
        }
        if (g == G - 1) {
            top[((size_t)top_slot * 2) * Tp + e] = hi;
            top[((size_t)top_slot * 2 + 1) * Tp + e] = lo;
        }
    }
}

}  // namespace krp
