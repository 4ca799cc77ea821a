// Dispatch of the batched conditional descent (a4 + a5, a6 fused): R <= 32
// runs descent_fast.cu's warp-per-sample kernel; 32 < R <= 128 descent_team.cu's
// team-per-sample kernel (the default, faster on GB300) or descent_nm.cu's
// node-major batches or descent_nmtc.cu's level-synchronous node-major form
// with the masses on the tensor cores (krp_set_descent_form); all follow the sampling loop of Alg. 2 with the
// loops exchanged as in App. A.6 and Alg. 4 on E_k and Z_k.  Also the
// sampled-row gather (a6) as a separate kernel.
#include "common.cuh"
#include "internal.h"

#include <math.h>

namespace krp {

krp_status launch_descent(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id,
                          int32_t* idx, float* weight, float* logq, float* SA, float* trace, int64_t n_trace) {
    cudaError_t fe = cudaSuccess;
    if (launch_descent_fast(s, exclude_j, J, seed, draw_id, idx, weight, logq, SA, trace, n_trace, &fe))
        return fe == cudaSuccess ? KRP_OK : cuda_check(s, fe, "descent launch");
    if (s->descent_form == KRP_DESCENT_NODE_MAJOR_TC &&
        launch_descent_nmtc(s, exclude_j, J, seed, draw_id, idx, weight, logq, SA, trace, n_trace, &fe))
        return fe == cudaSuccess ? KRP_OK : cuda_check(s, fe, "descent launch");
    if (s->descent_form == KRP_DESCENT_NODE_MAJOR &&
        launch_descent_nm(s, exclude_j, J, seed, draw_id, idx, weight, logq, SA, trace, n_trace, &fe))
        return fe == cudaSuccess ? KRP_OK : cuda_check(s, fe, "descent launch");
    if (launch_descent_team(s, exclude_j, J, seed, draw_id, idx, weight, logq, SA, trace, n_trace, &fe))
        return fe == cudaSuccess ? KRP_OK : cuda_check(s, fe, "descent launch");
    return fail(s, KRP_EINVAL, "descent: R outside 1..128");
}

// ---------------------------------------------------------------------------
// a6: sampled-row gather SA[s,:] = w_s * prod_k U_k[idx[k][s], :]
// (warp per sample, lanes over columns).
// ---------------------------------------------------------------------------
struct GatherParams {
    const float* U[16];
    int incl[16];
    int n_incl;
    int R;
    int64_t J;
    const int32_t* idx;
    const float* weight;
    float* SA;
};

__global__ void __launch_bounds__(256) krp_gather_kernel(GatherParams P) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < P.J; s += warps) {
        const float w = P.weight[s];
        for (int a = lane; a < P.R; a += 32) {
            float v = w;
            for (int pi = 0; pi < P.n_incl; ++pi) {
                const int k = P.incl[pi];
                const int64_t row = P.idx[(int64_t)k * P.J + s];
                v *= __ldg(P.U[k] + row * P.R + a);
            }
            P.SA[s * P.R + a] = v;
        }
    }
}

krp_status launch_gather(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx, const float* weight,
                         float* SA) {
    GatherParams P{};
    for (int k = 0; k < s->N; ++k) {
        P.U[k] = s->U[k];
        if (k != exclude_j) P.incl[P.n_incl++] = k;
    }
    P.R = s->R;
    P.J = J;
    P.idx = idx;
    P.weight = weight;
    P.SA = SA;
    const int64_t need = (J + 7) / 8;
    const int64_t grid = need < (int64_t)s->num_sms * 8 ? need : (int64_t)s->num_sms * 8;
    krp_gather_kernel<<<(unsigned)grid, 256, 0, s->stream>>>(P); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "gather launch");
    return KRP_OK;
}

}  // namespace krp
