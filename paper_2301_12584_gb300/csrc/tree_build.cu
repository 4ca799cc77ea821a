// a1: segment-tree Gram build (Alg. 3 BuildSampler with F leaf rows, Y = [1];
// Eq. partial_gram; Lemma 3.2 point 1).
//
// Layout: factor U is I x R row-major FP32.  The tree T_{I,F} has L = 2^d
// leaves (ceil(I/F) padded with empty leaves); leaf b covers rows
// [bF, min((b+1)F, I)).  Heap numbering: root 1, children 2h, 2h+1, leaf b is
// node L + b.  Only the root (slot 0) and left children (slot h/2) are stored,
// each as a packed upper triangle with stride Tp floats (see common.cuh).
//
// Kernel 1 (tree_leaves_*): each CTA owns G groups of LB consecutive leaves.
// Rows of the next group stream into shared memory with cp.async while the
// current group's leaf Grams G^v = U[S(v)]ᵀU[S(v)] are formed (FP32 FMA with
// 4x4 register tiles on the upper triangle, or tcgen05 BF16x3 in
// tree_build_tc.cu).  Each thread then owns a fixed set of packed entries and
// sums them pairwise up the group (parent = left + right, Alg. 3 line 7),
// continuing across groups with a per-entry binary-counter stack, storing
// every left child it creates.  The CTA's subtree root goes to scratch.
// Kernel 2 (tree_up): the same pairwise sums over LBB nodes per CTA for the
// levels above, until the root.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace krp {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage rows [row0, row0 + nrows) of U (zero beyond I) into sU (row stride R).
// VEC: 16-byte cp.async (needs R % 4 == 0 so every chunk is 16-byte aligned);
// otherwise plain synchronous loads.
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
        for (int64_t e = threadIdx.x; e < nf; e += blockDim.x) sU[e] = e < valid ? src[e] : 0.f;
    }
}

// Leaf Grams of LB leaves (F rows each) from sU into sG (LB x Tp), FP32 FMA,
// 4x4 register tiles over the upper triangle of 4-column blocks.
template <int LB, bool VEC>
__device__ __forceinline__ void leaf_grams_fp32(const float* sU, float* sG, int R, int F, int Tp) {
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
        float acc[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
        const float* base = sU + (size_t)leaf * F * R;
        for (int f = 0; f < F; ++f) {
            float a[4], b[4];
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
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
        float* g = sG + (size_t)leaf * Tp;
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const int i = 4 * ti + x, j = 4 * tj + y;
                if (i <= j && j < R) g[tri_index(i, j, R)] = acc[x][y];
            }
    }
}

__device__ __forceinline__ void store_node(float* __restrict__ tree, int64_t h, int Tp, int e, float v) {
    if (tree_stored(h)) tree[tree_slot(h) * Tp + e] = v;
}

// Pairwise sums of one group's LB leaf Grams (entry e), then the binary-counter
// merge across the CTA's groups.  Stores every left child created.
template <int LB>
__device__ __forceinline__ void reduce_group(const float* sG, float* stk, float* __restrict__ tree,
                                             float* __restrict__ top, int64_t L, int64_t first_leaf,
                                             int g, int G, int Tp) {
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        float v[LB];
#pragma unroll
        for (int l = 0; l < LB; ++l) v[l] = sG[l * Tp + e];
        int64_t h = L + first_leaf;
#pragma unroll
        for (int l = 0; l < LB; ++l) store_node(tree, h + l, Tp, e, v[l]);
#pragma unroll
        for (int n = LB; n > 1; n >>= 1) {
            h >>= 1;
#pragma unroll
            for (int l = 0; l < n / 2; ++l) {
                v[l] = v[2 * l] + v[2 * l + 1];
                store_node(tree, h + l, Tp, e, v[l]);
            }
        }
        float val = v[0];
        int idx = g, lvl = 0;
        while (idx & 1) {
            val = stk[lvl * Tp + e] + val;
            h >>= 1;
            idx >>= 1;
            ++lvl;
            store_node(tree, h, Tp, e, val);
        }
        stk[lvl * Tp + e] = val;
        if (g == G - 1) top[(size_t)blockIdx.x * Tp + e] = val;
    }
}

template <int LB, bool VEC>
__global__ void __launch_bounds__(512) tree_leaves_fp32(const float* __restrict__ U, int64_t I, int R, int F,
                                                        int64_t L, int G, int Tp, float* __restrict__ tree,
                                                        float* __restrict__ top) {
    extern __shared__ __align__(16) float smem[];
    const int rows = LB * F;
    const int T = tri_size(R);
    float* sU0 = smem;
    float* sU1 = sU0 + (size_t)rows * R;
    float* sG = (VEC ? sU1 : sU0) + (size_t)rows * R;
    float* stk = sG + (size_t)LB * Tp;
    for (int e = threadIdx.x; e < LB * Tp; e += blockDim.x)
        if (e % Tp >= T) sG[e] = 0.f;  // packed tail stays zero
    const int64_t leaf0 = (int64_t)blockIdx.x * G * LB;
    stage_rows<VEC>(sU0, U, I, R, leaf0 * F, rows);
    if (VEC) cp_async_commit();
    for (int g = 0; g < G; ++g) {
        float* cur = (VEC && (g & 1)) ? sU1 : sU0;
        if (VEC) {
            if (g + 1 < G) {
                stage_rows<VEC>((g & 1) ? sU0 : sU1, U, I, R, (leaf0 + (int64_t)(g + 1) * LB) * F, rows);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
        }
        __syncthreads();
        leaf_grams_fp32<LB, VEC>(cur, sG, R, F, Tp);
        __syncthreads();
        reduce_group<LB>(sG, stk, tree, top, L, leaf0 + (int64_t)g * LB, g, G, Tp);
        if (!VEC && g + 1 < G) {
            __syncthreads();
            stage_rows<VEC>(sU0, U, I, R, (leaf0 + (int64_t)(g + 1) * LB) * F, rows);
        }
    }
}

// Levels above the leaf kernel: LBB nodes per CTA from `in` (a full tree level
// with n_in nodes, heap ids n_in..2 n_in - 1) to one node per CTA in `out`.
template <int LBB>
__global__ void tree_up(const float* __restrict__ in, int64_t n_in, int Tp, float* __restrict__ tree,
                        float* __restrict__ out) {
    const int64_t first = (int64_t)blockIdx.x * LBB;
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        float v[LBB];
#pragma unroll
        for (int l = 0; l < LBB; ++l) v[l] = in[(first + l) * Tp + e];
        int64_t h = n_in + first;
#pragma unroll
        for (int n = LBB; n > 1; n >>= 1) {
            h >>= 1;
#pragma unroll
            for (int l = 0; l < n / 2; ++l) {
                v[l] = v[2 * l] + v[2 * l + 1];
                store_node(tree, h + l, Tp, e, v[l]);
            }
        }
        out[(size_t)blockIdx.x * Tp + e] = v[0];
    }
}

// BF16x3 tensor-core leaf kernel (tree_build_tc.cu); returns false if the
// shape is not supported there (caller falls back to FP32).
bool launch_tree_leaves_tc(krp_sampler* s, int j, int LB, int G, int64_t ctas, float* top, size_t smem_fp32);

namespace {

template <int LB, bool VEC>
cudaError_t launch_leaves(const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp, float* tree,
                          float* top, int64_t ctas, int threads, size_t smem, cudaStream_t st) {
    auto k = tree_leaves_fp32<LB, VEC>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<(unsigned)ctas, threads, smem, st>>>(U, I, R, F, L, G, Tp, tree, top); count_launch();
    return cudaGetLastError();
}

template <int LB>
cudaError_t dispatch_vec(bool vec, const float* U, int64_t I, int R, int F, int64_t L, int G, int Tp,
                         float* tree, float* top, int64_t ctas, int threads, size_t smem, cudaStream_t st) {
    return vec ? launch_leaves<LB, true>(U, I, R, F, L, G, Tp, tree, top, ctas, threads, smem, st)
               : launch_leaves<LB, false>(U, I, R, F, L, G, Tp, tree, top, ctas, threads, smem, st);
}

}  // namespace

// Leaf-kernel geometry: LB leaves per group (power of two, <= 16, <= L, one
// group of rows <= 32 KB), G groups per CTA (power of two, <= 8).
void tree_geometry(int R, int F, int64_t L, int Tp, bool vec, int* LB_out, int* G_out, int* threads_out,
                   size_t* smem_out) {
    const size_t leaf_bytes = (size_t)F * R * 4;
    int LB = 1;
    while (LB < 16 && (int64_t)LB * 2 <= L && (size_t)LB * 2 * leaf_bytes <= 32 * 1024) LB *= 2;
    const int nt = (R + 3) / 4;
    const int ntile = nt * (nt + 1) / 2;
    int threads = std::min(512, std::max(64, ((LB * ntile + 31) / 32) * 32));
    const int64_t groups = L / LB;
    int G = 1;
    auto smem_of = [&](int g) {
        int lv = 0;
        while ((1 << lv) < g) ++lv;
        return (size_t)(vec ? 2 : 1) * LB * leaf_bytes + (size_t)LB * Tp * 4 + (size_t)(lv + 1) * Tp * 4;
    };
    while (G < 8 && (int64_t)G * 2 <= groups && smem_of(G * 2) <= 160 * 1024) G *= 2;
    *LB_out = LB;
    *G_out = G;
    *threads_out = threads;
    *smem_out = smem_of(G);
}

krp_status build_tree(krp_sampler* s, int j, int precision) {
    const int R = s->R, F = s->F, Tp = s->Tp;
    const int64_t I = s->I[j], L = s->L[j];
    const bool vec = (R % 4) == 0;
    int LB, G, threads;
    size_t smem;
    tree_geometry(R, F, L, Tp, vec, &LB, &G, &threads, &smem);
    const int64_t ctas = L / ((int64_t)LB * G);
    const size_t need = (size_t)(ctas + ctas / 2 + 2) * Tp;
    if (need > s->build_scratch_floats) {
        if (s->build_scratch) cudaFree(s->build_scratch);
        s->build_scratch = nullptr;
        s->build_scratch_floats = 0;
        if (cudaMalloc(&s->build_scratch, need * sizeof(float)) != cudaSuccess)
            return fail(s, KRP_ENOMEM, "tree build scratch allocation failed");
        s->build_scratch_floats = need;
    }
    float* top = s->build_scratch;
    float* top2 = top + (size_t)ctas * Tp;
    bool done = false;
    if (precision == KRP_PREC_BF16X3) done = launch_tree_leaves_tc(s, j, LB, G, ctas, top, smem);
    if (!done) {
        cudaError_t e;
        switch (LB) {
            case 1: e = dispatch_vec<1>(vec, s->U[j], I, R, F, L, G, Tp, s->tree[j], top, ctas, threads, smem, s->stream); break;
            case 2: e = dispatch_vec<2>(vec, s->U[j], I, R, F, L, G, Tp, s->tree[j], top, ctas, threads, smem, s->stream); break;
            case 4: e = dispatch_vec<4>(vec, s->U[j], I, R, F, L, G, Tp, s->tree[j], top, ctas, threads, smem, s->stream); break;
            case 8: e = dispatch_vec<8>(vec, s->U[j], I, R, F, L, G, Tp, s->tree[j], top, ctas, threads, smem, s->stream); break;
            default: e = dispatch_vec<16>(vec, s->U[j], I, R, F, L, G, Tp, s->tree[j], top, ctas, threads, smem, s->stream); break;
        }
        if (e != cudaSuccess) return cuda_check(s, e, "tree leaf kernel launch");
    }
    int64_t n = ctas;
    const int up_threads = std::min(512, std::max(64, ((Tp + 31) / 32) * 32));
    while (n > 1) {
        const int64_t lbb = std::min<int64_t>(16, n);
        const unsigned grid = (unsigned)(n / lbb);
        switch (lbb) {
            case 2: tree_up<2><<<grid, up_threads, 0, s->stream>>>(top, n, Tp, s->tree[j], top2); count_launch(); break;
            case 4: tree_up<4><<<grid, up_threads, 0, s->stream>>>(top, n, Tp, s->tree[j], top2); count_launch(); break;
            case 8: tree_up<8><<<grid, up_threads, 0, s->stream>>>(top, n, Tp, s->tree[j], top2); count_launch(); break;
            default: tree_up<16><<<grid, up_threads, 0, s->stream>>>(top, n, Tp, s->tree[j], top2); count_launch(); break;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(s, e, "tree up kernel launch");
        std::swap(top, top2);
        n /= lbb;
    }
    return KRP_OK;
}

}  // namespace krp
