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
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

}  // namespace krp
