// Internal host-side declarations shared by the libkrpls translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/krpls.h"

struct krp_sampler {
    int N = 0, R = 0, F = 0, prec = 0;
    int descent_form = 0;       // KRP_DESCENT_* for 32 < R <= 128
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
    // exact-decision mode (KRP_PREC_EXACT): every tree slot's low part, and the
    // delta-encoded top levels [root | D_1 .. D_{2^Ke - 1}] (the tree's slot numbering)
    int exact = 0;
    std::vector<float*> tree_lo;  // L_k slots x Tp
    std::vector<float*> dtop;     // 2^Ke_k slots x Tp
    std::vector<int> Ke;          // delta-encoded levels: min(KRP_EXACT_TOP, depth_k)
    unsigned long long* nexact = nullptr;  // device count of exact re-decisions (row stages)
    // per-draw sampler state (written by the prep kernels)
    double* G64 = nullptr;      // N x R x R : FP64 copies of the root Grams
    double* Gplus64 = nullptr;  // R x R
    double* lam64 = nullptr;    // N x R      eigenvalues of G_{>k} (ascending)
    double* V64 = nullptr;      // N x R x R  eigenvectors (column u)
    double* work64 = nullptr;   // prep scratch: (N + 1) x 6 R x R FP64 (per included factor six
                                // R x R matrices of the eigen-refinement), then 256 doubles (scales)
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
    double* als_part = nullptr;   // per-CTA partial sums (column norms, fit), summed in a fixed order
    int64_t als_J = 0;
    // workspace of the tensor-core node-major descent (allocated on first use)
    char* nm_ws = nullptr;
    size_t nm_ws_bytes = 0;
    std::string last_error;
    int last_exclude = -2;      // exclude_j of the last prep (for inspection)
    // a captured sequence of this sampler's calls (krp_capture_begin / _end)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool capturing = false;
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
    // per mode, the fibers' lengths as (length, count) pairs, longest first:
    // the longest J fibers bound the (fiber, nonzero) pairs a J-sample solve reads
    std::vector<std::vector<std::pair<int64_t, int64_t>>> len_hist;
    // lookup scratch of the deterministic solve (sized for lk_J samples and
    // lk_pairs pairs): the samples sorted by fiber; per distinct sampled fiber
    // its run of samples, fiber id, summed w_s SA[s, :] and the scan of the
    // fiber lengths; the (fiber, nonzero) pairs sorted by mode-j row
    uint32_t* sk[2] = {nullptr, nullptr};
    uint32_t* sv[2] = {nullptr, nullptr};
    uint32_t* flag = nullptr;    // J + 1
    int64_t* useg = nullptr;     // 2 J
    int64_t* ufib = nullptr;     // J
    int64_t* poff = nullptr;     // J + 1
    int64_t* cnt = nullptr;      // distinct sampled fibers, pairs
    float* uacc = nullptr;       // J x R
    uint32_t* pk[2] = {nullptr, nullptr};
    uint32_t* pv[2] = {nullptr, nullptr};
    uint32_t* pu = nullptr;      // per pair: distinct-fiber index
    uint32_t* pn = nullptr;      // per pair: nonzero (fiber order)
    uint32_t* hist = nullptr;
    float* seg_part = nullptr;   // per chunk of sorted positions: 2 x R partial sums
    uint32_t* seg_info = nullptr;   // per chunk: 4 words
    size_t lk_J = 0, lk_pairs = 0, lk_hist = 0, lk_R = 0;
};

namespace krp {

// ---------------------------------------------------------------------------
// Kernel parameter blocks shared between the single-problem launches and the
// batched ones (batch.cu), which keep one block per problem in device memory.
// ---------------------------------------------------------------------------
struct PrepParams {
    const double* roots[16];  // FP64 root Gram G_k of each factor (packed upper)
    int incl[16];             // included factors, ascending
    int n_incl;
    int extra_refine;         // eigen-refinement steps beyond the first (samplers: 1; batches: 0)
};

struct PrepItem {  // everything prep_pinv / prep_eig read and write for one problem
    PrepParams P;
    int N, exclude, R, Rp, dE, Tp;
    double* G64;
    double* Gplus64;
    float* Gplus32;
    int* rank;
    int* status;
    double* gwork;
    double* lam64;
    double* V64;
    float* V32;
    float* V32lo;
    float* etree;
};

struct FastParams {  // the R <= 32 descent of one problem
    const float* U[16];
    const float* tree[16];
    const float* tlo[16];     // exact-decision mode: tree low parts
    const float* dtop[16];    // exact-decision mode: delta-encoded top levels
    int Ke[16];               // exact-decision mode: delta-encoded levels
    const float* etree[16];
    const float* Vhi[16];
    const float* Vlo[16];
    int64_t I[16];
    int64_t L[16];
    int depth[16];
    int incl[16];
    int n_incl;
    int R, F, T, Tp, Rp, dE;
    const float* Gplus32;
    const int* rank;
    int* status;
    uint32_t key0, key1, draw;
    int64_t J;
    int32_t* idx;
    float* weight;
    float* logq;
    float* SA;
    float* trace;
    int64_t n_trace;
    unsigned long long* nexact;   // exact-decision mode: count of exact re-decisions (may be null)
};

struct FastCall {  // per-call arguments of the batched descent
    uint32_t key0, key1, draw;
    int N;
    int64_t J;
    int32_t* idx;            // [P][N][J]
    float* weight;           // [P][J]
    float* SA;               // problem p at SA + J * row_off[p], rows of R_p floats
    const int64_t* row_off;  // device, prefix sums of R_p
};

struct TreeDesc {  // one factor tree of one problem, for the batched build
    const float* src;      // rows to build from
    float* copy_to;        // the sampler's copy of the factor (written if != src), or nullptr
    float* tree;
    float* top;            // (hi, lo) pairs of the leaf kernel's block roots
    double* up[2];         // FP64 levels above the leaf kernel
    double* root64;
    int64_t I, L;
    int R, F, Tp, G;       // G groups of the batch's LB leaves per leaf-kernel block
};

struct UpDesc {  // one tree in one pass of the batched level sums
    const float* in_pairs;  // first pass: the leaf kernel's (hi, lo) pairs
    const double* in64;     // later passes: FP64 nodes
    double* out;
    float* tree;
    int64_t n_in;           // nodes of the input level (heap ids n_in .. 2 n_in - 1)
    int lbb;                // nodes summed per CTA (1..16)
    int Tp;
};

struct SolveItem {  // one problem of the batched dense solve
    int R;
    int nparts;
    int64_t row_off;  // SA rows of this problem start at SA + J * row_off
    int64_t x_off;    // X of this problem at X + x_off * nrhs
    float* part;      // nparts x (T + R nrhs) partials
};

struct PlantItem {  // one problem of the planted right-hand side (included factors only)
    const float* U[16];
    int64_t I[16];
    int krow[16];      // row of idx holding factor m's indices
    int N, R;
    int64_t row_off;   // X of this problem at X + row_off * nrhs
};

krp_status fail(krp_sampler* s, krp_status code, const std::string& msg);
// Process-wide count of kernel launches made by this library.
void count_launch();
int64_t launch_counter();
krp_status cuda_check(krp_sampler* s, cudaError_t e, const char* what);

// a1: build factor j's segment tree from s->U[j] (FP32 or BF16x3 Grams; exact
// leaves and low parts in an exact-decision sampler).
krp_status build_tree(krp_sampler* s, int j, int precision, const float* src = nullptr);
// The delta-encoded top of factor j's tree from its (hi, lo) slots (exact mode).
cudaError_t launch_build_dtop(const krp_sampler* s, int j, cudaStream_t st);
// a2 + a3: G, G⁺, G_{>k}, eigendecompositions, E_k trees for the given exclusion.
krp_status sampler_prep(krp_sampler* s, int exclude_j);
// a4 + a5 (+a6 fused): the batched conditional descent.
krp_status launch_descent(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed,
                          uint64_t draw_id, int32_t* idx, float* weight, float* logq, float* SA,
                          float* trace = nullptr, int64_t n_trace = 0);
// R <= 32 path of the descent (descent_fast.cu); false if R is out of range.
bool launch_descent_fast(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err);
// 32 < R <= 128 path (descent_team.cu): TMA-staged teams of warps; false if R is out of range.
bool launch_descent_team(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err);
// 32 < R <= 128 node-major path (descent_nm.cu): CTA batches advanced level by
// level; false if R is out of range or no batch fits the shared memory.
bool launch_descent_nmtc(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err);
bool launch_descent_nm(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
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

// Batched launches (one launch per phase for many problems; batch.cu).
void prep_item_for(const krp_sampler* s, int exclude_j, PrepItem* it);
cudaError_t launch_prep_batch(const PrepItem* items_dev, int P, int n_incl, int Rmax, cudaStream_t st);
void fast_params_for(const krp_sampler* s, int exclude_j, FastParams* P);
cudaError_t launch_descent_fast_batch(const FastParams* table_dev, const FastCall& call, int P, int ctas_per_problem,
                                      cudaStream_t st);
cudaError_t launch_leaves_batch(const TreeDesc* trees_dev, const int64_t* block_prefix_dev, int ntrees,
                                int64_t nblocks, int LB, int Rmax, int Fmax, int Tpmax, int Gmax, bool vec,
                                cudaStream_t st);
cudaError_t launch_up_batch(const UpDesc* ups_dev, const int64_t* cta_prefix_dev, int ntrees, int64_t nctas,
                            int Tpmax, bool from_pairs, cudaStream_t st);
cudaError_t launch_solve_batch(const SolveItem* items_dev, int P, int max_parts, int Rmax, int64_t J,
                               const float* SA, const float* weight, const float* B, int nrhs, int flags, float* X,
                               int* status, cudaStream_t st);
cudaError_t launch_planted(const PlantItem* items_dev, int P, int64_t J, const int32_t* idx, int N_idx,
                           const float* X_true, int nrhs, float sigma, uint64_t seed, float* B, cudaStream_t st);

}  // namespace krp
