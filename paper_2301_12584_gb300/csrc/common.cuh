// Shared device helpers for libkrpls (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/krpls.h"

namespace krp {

// ---------------------------------------------------------------------------
// Packed upper-triangle layout of a symmetric R x R node matrix: row i holds
// columns j = i..R-1, rows concatenated.  T = R(R+1)/2 entries; each node is
// stored with a stride Tp = T rounded up to a multiple of 8 floats (32-byte
// sectors, 16-byte vector loads), the tail zero-filled.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int tri_size(int R) { return R * (R + 1) / 2; }
__host__ __device__ __forceinline__ int tri_stride(int R) { return (tri_size(R) + 7) & ~7; }
__host__ __device__ __forceinline__ int tri_index(int i, int j, int R) {
    return i * R - (i * (i - 1)) / 2 + (j - i);
}

// Storage slot of heap node h (root 1, children 2h, 2h+1): the root is slot 0
// and a left child h (even) is slot h/2.  Right children are not stored; a
// descent only reads left children (Alg. 4).
__host__ __device__ __forceinline__ int64_t tree_slot(int64_t h) { return h == 1 ? 0 : h >> 1; }
__host__ __device__ __forceinline__ bool tree_stored(int64_t h) { return h == 1 || (h & 1) == 0; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64
// multiplies, word permutation and key xor; the key is bumped by two Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// (2*(x>>9)+1) * 2^-24: an open-interval uniform exact in FP32 and FP64.
__device__ __forceinline__ float u32_to_unit(uint32_t x) {
    return (float)(2u * (x >> 9) + 1u) * 5.9604644775390625e-8f;
}

// ---------------------------------------------------------------------------
// Device status word: the first failure wins, later ones are dropped.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Butterfly sum: every lane ends with the bitwise-identical total (each step
// adds two equal partials in either order), so branch decisions that depend
// on it are warp-uniform.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}
// Two FP32 fused multiply-adds in one instruction: (a.x b.x + c.x, a.y b.y + c.y).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    uint64_t d;
    const uint64_t ua = *reinterpret_cast<uint64_t*>(&a), ub = *reinterpret_cast<uint64_t*>(&b),
                   uc = *reinterpret_cast<uint64_t*>(&c);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(ua), "l"(ub), "l"(uc));
    return *reinterpret_cast<float2*>(&d);
}
// Paired FP32 add / subtract (one instruction each, round to nearest).
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    uint64_t d;
    const uint64_t ua = *reinterpret_cast<uint64_t*>(&a), ub = *reinterpret_cast<uint64_t*>(&b);
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(ua), "l"(ub));
    return *reinterpret_cast<float2*>(&d);
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    uint64_t d;
    const uint64_t ua = *reinterpret_cast<uint64_t*>(&a), ub = *reinterpret_cast<uint64_t*>(&b);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(ua), "l"(ub));
    return *reinterpret_cast<float2*>(&d);
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is an unevaluated pair hi + lo of FP32
// numbers with |lo| <= ulp(hi)/2 (about 48 significant bits).  Error-free
// transformations: TwoSum (Knuth) and TwoProduct via FMA.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ df df_add(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    df r;
    r.hi = s + e;
    r.lo = e - (r.hi - s);
    return r;
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
// (double-float) + (float)
__device__ __forceinline__ df df_add_f(df a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    e += a.lo;
    df r;
    r.hi = s + e;
    r.lo = e - (r.hi - s);
    return r;
}
// (float) x (double-float)
__device__ __forceinline__ df df_mul_f(df a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    df r;
    r.hi = p + e;
    r.lo = e - (r.hi - p);
    return r;
}
// a <= b
__device__ __forceinline__ bool df_le(df a, df b) {
    const df d = df_add(a, df_neg(b));
    return d.hi < 0.f || (d.hi == 0.f && d.lo <= 0.f);
}
// a * b = p + e exactly (TwoProduct by FMA).
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = a * b;
    return df{p, fmaf(a, b, -p)};
}
// (double-float) x (double-float), about 2^-44 relative.
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    df r;
    r.hi = p + e;
    r.lo = e - (r.hi - p);
    return r;
}

// ---------------------------------------------------------------------------
// Rows of heap node h at depth t of a tree with L leaves of F rows over I
// rows (Sec. 3.1: leaf b holds rows [bF, min((b+1)F, I)), padding leaves are
// empty), and the share alpha_c = rows(2c) / rows(c) of node c's left child,
// rounded to FP32 (1/2 for every full node).  The exact-decision mode stores
// the top levels of a tree as D_c = G_{2c} - alpha_c G_c, so that the FP32
// rounding falls on the small deviation of a child from its share of the
// parent rather than on the child's whole Gram.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t node_rows(int64_t h, int t, int64_t L, int F, int64_t I) {
    const int64_t span = L >> t;
    const int64_t b0 = (h - ((int64_t)1 << t)) * span;
    const int64_t lo = b0 * F < I ? b0 * F : I;
    const int64_t hi = (b0 + span) * F < I ? (b0 + span) * F : I;
    return hi - lo;
}
__host__ __device__ __forceinline__ float node_alpha(int64_t c, int t, int64_t L, int F, int64_t I) {
    const int64_t n = node_rows(c, t, L, F, I);
    return n > 0 ? (float)node_rows(2 * c, t + 1, L, F, I) / (float)n : 0.5f;
}
// Top levels delta-encoded in exact-decision mode (decisions at depth < KRP_EXACT_TOP).
constexpr int KRP_EXACT_TOP = 10;
// Margin of the exact-decision mode, relative to the stage total C, added to
// the FP32 path's modelled error terms: a decision whose gap |tau - low -
// m(L(c))| is within both is re-taken from double-float masses.
constexpr float KRP_EXACT_BAND = 5e-10f;

// Butterfly sum of a double-float over the warp; every lane gets the same pair
// (TwoSum gives the same exact error for either operand order).
__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, v.hi, m);
        const float ol = __shfl_xor_sync(0xffffffffu, v.lo, m);
        float s, e;
        two_sum(v.hi, oh, s, e);
        e += v.lo + ol;
        v.hi = s + e;
        v.lo = e - (v.hi - s);
    }
    return v;
}

}  // namespace krp
