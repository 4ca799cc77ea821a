// Internal host-side declarations shared by the libkrpls translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/krpls.h"

struct krp_sampler {
    int N = 0, R = 0, F = 0, prec = 0;
    cudaStream_t stream = nullptr;
    int T = 0, Tp = 0;          // packed triangle size and node stride (floats)
    int Rp = 1, dE = 0;         // eigencomponent tree: leaves (R padded to 2^dE)
    int num_sms = 0;
    std::vector<int64_t> I, L;  // rows and padded leaf count per factor
    std::vector<int> depth;     // log2 L
    std::vector<float*> U;      // factor copies, I_k x R
    std::vector<float*> tree;   // L_k slots x Tp
    std::vector<double*> root64;  // FP64 root Gram G_k (packed upper, Tp) per factor
    std::vector<char> has_factor;
    // per-draw sampler state (written by the prep kernels)
    double* G64 = nullptr;      // N x R x R : FP64 copies of the root Grams
    double* Gplus64 = nullptr;  // R x R
    double* lam64 = nullptr;    // N x R      eigenvalues of G_{>k} (ascending)
    double* V64 = nullptr;      // N x R x R  eigenvectors (column u)
    double* work64 = nullptr;   // prep scratch: N x (2 R x R) FP64
    float* Gplus32 = nullptr;   // Tp packed upper triangle of G⁺
    float* etree = nullptr;     // N x Rp x Tp : eigencomponent trees E_k
    float* V32 = nullptr;       // N x R x R : row u = eigenvector u of G_{>k}
    float* V32lo = nullptr;     // N x R x R : FP32 residual V - V32 (double-float eigenvectors)
    int* rank_dev = nullptr;    // rank(A) of the last prep
    int* status = nullptr;      // device status word
    // scratch
    float* build_scratch = nullptr;
    size_t build_scratch_floats = 0;
    float* solve_scratch = nullptr;
    size_t solve_scratch_floats = 0;
    double* solve64 = nullptr;  // FP64 solve work (2 R*R + 128 R) then M⁻¹ (R*R)
    // STS-CP sweep buffers (allocated on first use)
    int32_t* als_idx = nullptr;
    float* als_w = nullptr;
    float* als_SA = nullptr;
    double* als_sumsq = nullptr;
    int64_t als_J = 0;
    std::string last_error;
    int last_exclude = -2;      // exclude_j of the last prep (for inspection)
};

struct krp_sptensor {
    int N = 0;
    int64_t nnz = 0;
    cudaStream_t stream = nullptr;
    std::vector<int64_t> I;
    int32_t* coords = nullptr;         // N x nnz (device), original order
    float* vals = nullptr;             // nnz (device), original order
    // per mode j: fibers of mode j sorted by the key of the other modes
    std::vector<uint64_t*> fkeys;      // nf_j keys (ascending)
    std::vector<int64_t*> fptr;        // nf_j + 1 offsets
    std::vector<int32_t*> fidx;        // nnz: mode-j coordinate, fiber order
    std::vector<float*> fval;          // nnz: value, fiber order
    std::vector<int64_t> nfib;
    std::vector<int> kbits;            // bits per mode in the packed key
    double normT2 = 0.0;               // ||T||_F^2 (host, FP64)
    float* Y = nullptr;                // scratch: max I_j x R
    size_t Y_floats = 0;
};

namespace krp {

krp_status fail(krp_sampler* s, krp_status code, const std::string& msg);
// Process-wide count of kernel launches made by this library.
void count_launch();
int64_t launch_counter();
krp_status cuda_check(krp_sampler* s, cudaError_t e, const char* what);

// a1: build factor j's segment tree from s->U[j] (FP32 or BF16x3 Grams).
krp_status build_tree(krp_sampler* s, int j, int precision, const float* src = nullptr);
// a2 + a3: G, G⁺, G_{>k}, eigendecompositions, E_k trees for the given exclusion.
krp_status sampler_prep(krp_sampler* s, int exclude_j);
// a4 + a5 (+a6 fused): the batched conditional descent.
krp_status launch_descent(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed,
                          uint64_t draw_id, int32_t* idx, float* weight, float* logq, float* SA,
                          float* trace = nullptr, int64_t n_trace = 0);
// R <= 32 path of the descent (descent_fast.cu); false if R is out of range.
bool launch_descent_fast(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err);
cudaError_t launch_wait_timeout_probe(krp_sampler* s, int tries);
// a6: gather
krp_status launch_gather(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx,
                         const float* weight, float* SA);
// a8: normal equations (M = SAᵀSA, Z = SAᵀ diag(w) B) + FP64 Cholesky solve.
krp_status dense_solve(krp_sampler* s, int64_t J, const float* SA, const float* weight,
                       const float* B_rows, int nrhs, float* X, int flags);
// a8 (sparse): M⁻¹ into s->solve64 (FP64, R x R), from SA.
krp_status normal_inverse(krp_sampler* s, int64_t J, const float* SA, int flags);

}  // namespace krp
