// Single-element updates of a factor (UpdateSampler, App. A "Efficient
// single-element updates"): U_j[r, c] := u_new changes, in the leaf holding
// row r, only row and column c of its Gram — by d x (x the old row, d =
// u_new - U_j[r, c]) plus d² on the diagonal — and every ancestor, the sum of
// its two children, by the same row and column.  So one update touches R
// entries of each stored node on the leaf's root path (the root and the left
// children among its ancestors; right children are not stored) and of the
// FP64 root: O(R log(I/F)) work.
//
// One CTA applies the n updates in order (an update may read a row that an
// earlier one changed); per update its threads spread over (node, entry).
#include "common.cuh"
#include "internal.h"

namespace krp {
namespace {

// tree_lo (exact-decision mode, else null): the slots' low parts; each stored
// entry then takes the change in double-float, (hi, lo) + change.
__global__ void __launch_bounds__(256) update_entries(float* __restrict__ U, float* __restrict__ tree,
                                                      float* __restrict__ tree_lo,
                                                      double* __restrict__ root64, int64_t I, int R, int F,
                                                      int64_t L, int depth, int Tp, int64_t n,
                                                      const int32_t* __restrict__ rows,
                                                      const int32_t* __restrict__ cols,
                                                      const float* __restrict__ vals, int* __restrict__ status) {
    __shared__ double dv[128];   // change of row / column c: d x[k], and 2 d x[c] + d² at k = c
    __shared__ int64_t slots[64];
    __shared__ int nslots;
    for (int64_t q = 0; q < n; ++q) {
        const int64_t r = rows[q];
        const int c = cols[q];
        const bool ok = r >= 0 && r < I && c >= 0 && c < R;  // uniform across the CTA
        if (!ok) {
            if (threadIdx.x == 0) set_status(status, KRP_EINVAL);
            continue;
        }
        const double d = (double)vals[q] - (double)U[r * R + c];
        for (int k = threadIdx.x; k < R; k += blockDim.x) {
            const double x = (double)U[r * R + k];
            dv[k] = k == c ? 2.0 * d * x + d * d : d * x;
        }
        if (threadIdx.x == 0) {
            int m = 0;
            for (int64_t h = L + r / F; h >= 1; h >>= 1)
                if (tree_stored(h)) slots[m++] = tree_slot(h);
            nslots = m;
        }
        __syncthreads();
        const int m = nslots;
        for (int t = threadIdx.x; t < m * R; t += blockDim.x) {
            const int node = t / R, k = t % R;
            const int e = k < c ? tri_index(k, c, R) : tri_index(c, k, R);
            const int64_t at = slots[node] * (int64_t)Tp + e;
            if (tree_lo) {
                const double v = (double)tree[at] + (double)tree_lo[at] + dv[k];
                const float hi = (float)v;
                tree[at] = hi;
                tree_lo[at] = (float)(v - (double)hi);
            } else {
                tree[at] += (float)dv[k];
            }
        }
        for (int k = threadIdx.x; k < R; k += blockDim.x)
            root64[k < c ? tri_index(k, c, R) : tri_index(c, k, R)] += dv[k];
        if (tree_lo) {   // exact-decision trees: the trace after the packed triangle changes by dv[c]
            const int T = tri_size(R);
            for (int node = threadIdx.x; node < m; node += blockDim.x) {
                const int64_t at = slots[node] * (int64_t)Tp + T;
                const double v = (double)tree[at] + (double)tree_lo[at] + dv[c];
                const float hi = (float)v;
                tree[at] = hi;
                tree_lo[at] = (float)(v - (double)hi);
            }
            if (threadIdx.x == 0) root64[T] += dv[c];
        }
        __syncthreads();
        if (threadIdx.x == 0) U[r * R + c] = vals[q];
        __syncthreads();
    }
    (void)depth;
}

}  // namespace
}  // namespace krp

using namespace krp;

extern "C" krp_status krp_update_entries(krp_sampler* s, int j, int64_t n, const int32_t* rows, const int32_t* cols,
                                         const float* values) {
    if (!s) return fail(nullptr, KRP_EINVAL, "krp_update_entries: NULL sampler");
    if (j < 0 || j >= s->N) return fail(s, KRP_EINVAL, "krp_update_entries: j out of range");
    if (n < 0 || (n > 0 && (!rows || !cols || !values)))
        return fail(s, KRP_EINVAL, "krp_update_entries: need n >= 0 and device rows, cols, values");
    if (!s->has_factor[j]) return fail(s, KRP_ESTATE, "krp_update_entries: factor not set");
    if (n == 0) return KRP_OK;
    update_entries<<<1, 256, 0, s->stream>>>(s->U[j], s->tree[j], s->exact ? s->tree_lo[j] : nullptr, s->root64[j],
                                             s->I[j], s->R, s->F, s->L[j], s->depth[j], s->Tp, n, rows, cols, values,
                                             s->status);
    count_launch();
    s->last_exclude = -2;  // the per-draw preparation depends on G_j
    krp_status st = cuda_check(s, cudaGetLastError(), "krp_update_entries launch");
    if (st == KRP_OK && s->exact) st = cuda_check(s, launch_build_dtop(s, j, s->stream), "delta-encoded top launch");
    return st;
}
