/*
 * krpls.h — C ABI of libkrpls, exact leverage-score sampling from Khatri-Rao
 * products and the sketched least-squares solves it feeds (CP-ALS), for
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Bharadwaj, Malik, Murray, Grigori, Buluç, Demmel, "Fast Exact
 * Leverage Score Sampling from Khatri-Rao Products with Applications to
 * Tensor Decomposition", NeurIPS 2023 (arXiv 2301.12584).
 *
 * Conventions for every call below
 *   - Matrices are row-major and contiguous.  Factor U_k is I_k x R, FP32.
 *   - Pointers are DEVICE pointers unless the parameter name ends in _host
 *     or the comment says "host or device" (those accept pinned/pageable
 *     host memory or device memory; the copy is made with cudaMemcpyDefault).
 *   - All work is enqueued asynchronously on the CUDA stream passed to
 *     krp_create (0 = legacy default stream).  Output buffers are valid
 *     after that stream is synchronised (e.g. by krp_sync_status).
 *   - The caller owns every buffer it passes in.  The sampler owns copies of
 *     the factors, the segment trees, and all scratch.  No call allocates
 *     device memory except krp_create, krp_sptensor_create and the first
 *     call that needs a larger scratch buffer (documented per call).
 *   - Errors: arguments the host can check return immediately with a
 *     negative krp_status and leave no work enqueued.  Conditions found on
 *     the device (zero or non-finite probability mass, a singular normal
 *     matrix) set a device status word that krp_sync_status returns and
 *     clears.  krp_last_error gives a message for the most recent failure.
 *   - No call prints, aborts or throws across the ABI.
 */
#ifndef KRPLS_H
#define KRPLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct krp_sampler krp_sampler;     /* opaque */
typedef struct krp_sptensor krp_sptensor;   /* opaque */

typedef enum {
    KRP_OK = 0,
    KRP_EINVAL = -1,      /* bad argument (host-checked)                         */
    KRP_ENOMEM = -2,      /* device allocation failed                            */
    KRP_ECUDA = -3,       /* a CUDA runtime call failed                          */
    KRP_EZERO = -4,       /* total probability mass is zero (A == 0, or U_k unset)*/
    KRP_ESINGULAR = -5,   /* normal matrix not positive definite                 */
    KRP_ENUMERIC = -6,    /* NaN or Inf probability mass seen on the device      */
    KRP_ETIMEOUT = -7,    /* a bounded device wait gave up (no hang)             */
    KRP_ESTATE = -8       /* call made in the wrong state (e.g. factor not set)  */
} krp_status;

typedef enum {
    KRP_PREC_FP32 = 0,    /* segment-tree Grams by FP32 FMA                      */
    KRP_PREC_BF16X3 = 1,  /* Grams on tcgen05 tensor cores, BF16 hi/lo split,    */
                          /* three products, FP32 accumulate                     */
    KRP_PREC_EXACT = 2,   /* exact decisions (sampler-wide, at krp_create, R <= 32): */
                          /* leaf Grams accumulated without rounding error, every */
                          /* tree slot kept as a double-float (hi, lo) pair, the  */
                          /* top tree levels also stored as deviations from their */
                          /* share of the parent, and every descent decision whose */
                          /* FP32 gap lies within its error terms (+5e-10 C) of a */
                          /* bin edge re-taken from double-float masses (Alg. 4   */
                          /* in near-FP64 arithmetic)                             */
    KRP_PREC_TF32X3 = 3   /* Grams on tcgen05 tensor cores, TF32 hi/lo split     */
                          /* (~22 significant bits), three products, FP32         */
                          /* accumulate; the sparse solve's Y M^-1 as TF32x3 too  */
} krp_precision;

#define KRP_PINV_FALLBACK 1  /* krp_solve_*: if Cholesky fails, use the FP64
                                eigen-pseudo-inverse instead of failing       */

/* ------------------------------------------------------------------------
 * Construction (Thm 1.1 part 1; Alg. 1 ConstructKRPSampler; Alg. 3
 * BuildSampler; Lemma 3.2).
 *
 * krp_create: a sampler for N factors U_k (I_host[k] x R).  F is the leaf
 * size of each factor's segment tree T_{I_k,F} (F = 0 selects F = R, the
 * paper's choice for the row samplers Z_k).  The tree's leaf count is
 * ceil(I_k/F) padded to a power of two with empty leaves.  Limits:
 * 1 <= N <= 16, 1 <= R <= 128, 1 <= I_k < 2^31, 1 <= F <= 4*R.
 * `stream` is a cudaStream_t (may be NULL).  Allocates all factor, tree and
 * sampler storage.  On failure *out is set to NULL.
 * precision = KRP_PREC_EXACT makes the whole sampler draw as the FP64 Alg. 2/4
 * would (indices equal to an FP64 replay except where a uniform lies within
 * ~1e-12 of a bin edge): it needs R <= 32 (KRP_EINVAL otherwise), allocates a
 * second array the size of each tree plus 2^10 slots per factor, builds
 * every tree with exact leaves whatever precision krp_set_factor_prec names.
 * ---------------------------------------------------------------------- */
krp_status krp_create(krp_sampler** out, int N, const int64_t* I_host, int R, int F,
                      int precision, void* stream);

/* Release everything the sampler owns (NULL is a no-op).  Synchronises the
 * sampler's stream first. */
void krp_destroy(krp_sampler* s);

/* Full-factor update (Thm 1.1 part 1; Alg. 1).  Copies U (I_j x R,
 * host or device) into the sampler and rebuilds Z_j: leaf partial Grams
 * G^v = U[S(v)]ᵀ U[S(v)] and their sums up the tree (Eq. partial_gram),
 * whose root is G_j = U_jᵀ U_j.  Returns KRP_EINVAL for j out of range. */
krp_status krp_set_factor(krp_sampler* s, int j, const float* U);

/* Same as krp_set_factor with an explicit precision for this rebuild. */
krp_status krp_set_factor_prec(krp_sampler* s, int j, const float* U, int precision);

/* Single-element updates (App. A, UpdateSampler): for q = 0..n-1 in order,
 * U_j[rows[q], cols[q]] := values[q] (rows, cols int32 and values FP32, device
 * arrays of n entries).  Each update changes row and column cols[q] of the
 * stored Grams on the leaf-to-root path of its row and of the FP64 root:
 * O(R log(I_j/F)) work instead of a rebuild.  An out-of-range (row, col) is
 * skipped and sets KRP_EINVAL on the device status.  FP32 tree entries take
 * the FP32-rounded change, so after many updates a rebuild (krp_set_factor)
 * restores the build's rounding.  The next krp_sample_draw needs a new
 * krp_sample_prepare (krp_sample does both). */
krp_status krp_update_entries(krp_sampler* s, int j, int64_t n, const int32_t* rows, const int32_t* cols,
                              const float* values);

/* ------------------------------------------------------------------------
 * Sampling (Thm 1.1 part 2; Alg. 2 KRPSample; Alg. 4 RowSample; Thm 3.1).
 *
 * Draws J i.i.d. row indices of A = ⊙_{k != exclude_j} U_k from the exact
 * leverage-score distribution (Eq. leverage_definition), factors taken in
 * ascending k.  Per draw the sampler forms G = ⊛ G_k and G⁺ (FP64,
 * eigen-pseudo-inverse with cutoff R*2^-52*lam_max), and for each included k
 * G_{>k} = G⁺ ⊛ ⊛_{m>k} G_m (Eq. G_geq_k_defn), its eigendecomposition
 * (FP64, eigenvalues ascending, negatives clamped to 0) and the eigencomponent
 * sampler E_k (Alg. 2).  Each sample then descends E_k and Z_k for
 * each k (two-stage draw, Eqs. first_dist and second_conditional_dist).
 *
 * Uniforms: Philox4x32-10 with key (seed lo32, seed hi32) and counter
 * (sample index d, draw_id lo32, position of k among included factors, 0);
 * word 0 drives the eigencomponent stage and word 1 the row stage, each
 * mapped to (2*(x>>9)+1)*2^-24.
 *
 * Outputs (device):
 *   idx     int32 [N][J] (row k holds the index into U_k; row exclude_j is
 *           left untouched).
 *   weight  float [J], w_s = 1/sqrt(J q_s) with q_s = ℓ_s / rank(A) (Sec. 2.1).
 *   logq    float [J] or NULL: log q_s.
 *   SA      float [J][R] or NULL: the sketched design rows w_s ⊛_k U_k[s_k,:]
 *           (fused gather; same values as krp_gather).
 * Requires every included factor set (else KRP_ESTATE).  J >= 1, J < 2^31.
 * exclude_j = -1 includes every factor.  Device-side failures (zero or
 * non-finite mass) are reported by krp_sync_status.
 * ---------------------------------------------------------------------- */
krp_status krp_sample(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed,
                      uint64_t draw_id, int32_t* idx, float* weight, float* logq, float* SA);

/* krp_sample split in two, for callers that time or overlap the phases:
 * krp_sample_prepare does the per-draw work that does not depend on the
 * samples (the set-up of Alg. 2: G, G⁺, G_{>k}, eigendecompositions, E_k) for
 * one exclusion; krp_sample_draw then runs the descent (its sampling loop) and may be
 * called several times (other J, seed or draw_id) while no factor changes.
 * krp_sample_draw returns KRP_ESTATE if the last prepare was for another
 * exclude_j or a factor was set since. */
krp_status krp_sample_prepare(krp_sampler* s, int exclude_j);
krp_status krp_sample_draw(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id,
                           int32_t* idx, float* weight, float* logq, float* SA);

/* Form of the descent for 32 < R <= 128 (no effect at R <= 32): the same
 * draws up to the rounding of the masses (flips only where a uniform lies
 * within ~1e-6 of a bin edge; ~1e-5 for the tensor-core form at R = 128).
 *   KRP_DESCENT_AUTO (default) and KRP_DESCENT_TEAM: one team of warps per
 *     sample, two tree levels per fetch, the sample's quadratic-form weights
 *     kept in registers for a whole tree;
 *   KRP_DESCENT_NODE_MAJOR: each CTA advances a batch of up to 32 samples
 *     level by level together, grouping them by the node they sit at so that
 *     every distinct node is fetched once per batch (shared upper levels cost
 *     one fetch per CTA, deeper ones stream through a ring of copies across
 *     the batch); the weights are formed per sample and level.
 *   KRP_DESCENT_NODE_MAJOR_TC (App. A.10's level-synchronous batches): all J
 *     samples advance one tree level at a time, grouped by node; for each
 *     group of up to 128 samples with vectors H (128 x R) the left child's
 *     masses come from D = H G_v on the tcgen05 tensor cores (split TF32,
 *     m_s = Σ_j D[s, j] H[s, j]) and the leaf's row weights from
 *     D = H U_leafᵀ; decisions within 1e-6 C of an edge are re-taken in
 *     double-float.  Faster than TEAM from R ~ 96 up, but its split-TF32
 *     masses are less exact: at R = 128 it flips about twice as many draws
 *     within 1e-5 C of a bin edge.  Needs F <= 128 and a device workspace of about
 *     J (3 R + 24) floats; where that does not hold (or no workspace can be
 *     allocated, e.g. during a graph capture) the team form runs instead.
 * KRP_EINVAL for another value. */
#define KRP_DESCENT_AUTO 0
#define KRP_DESCENT_TEAM 1
#define KRP_DESCENT_NODE_MAJOR 2
#define KRP_DESCENT_NODE_MAJOR_TC 3
krp_status krp_set_descent_form(krp_sampler* s, int form);

/* Sampled-row gather: SA[s,:] = weight[s] * ⊛_{k != exclude_j} U_k[idx[k][s], :]
 * (the rows of S·A, Sec. 2.1).  idx/weight as produced by krp_sample.  Indices
 * are not range-checked on the device; pass krp_sample's output. */
krp_status krp_gather(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx,
                      const float* weight, float* SA);

/* Dense sketched solve X = argmin ||SA X - SB||_F (Thm 2.1) by the normal
 * equations: M = SAᵀSA and Z = SAᵀ SB formed in FP32 with an FP64 final
 * reduction, FP64 Cholesky of M, X = M⁻¹ Z.  SB[s,:] = weight[s] * B_rows[s,:]
 * where B_rows (J x nrhs) are the caller's unweighted rows of B at the sampled
 * tuples.  X is R x nrhs (device).  1 <= nrhs <= 64.  If M is not positive
 * definite: with flags & KRP_PINV_FALLBACK, X = M⁺ Z (FP64 eigen-pseudo-inverse);
 * otherwise the device status becomes KRP_ESINGULAR and X is zero.  The first
 * call with a larger J or nrhs than any before may allocate scratch. */
krp_status krp_solve_dense(krp_sampler* s, int64_t J, const float* SA, const float* weight,
                           const float* B_rows, int nrhs, float* X, int flags);

/* krp_solve_dense without any device allocation (no counterpart in the paper;
 * it is the same Thm 2.1 solve, by the same kernels).  For callers that may
 * not allocate device memory: a host framework that owns all of it through its
 * own pool, or a loop under a memory budget where an allocation could fail or
 * stall the device.  Needs no sampler.
 *   J: sampled rows, 1 <= J < 2^31.  R: 1..32.  nrhs: 1..16.
 *   SA (J x R), weight (J), B_rows (J x nrhs), X (R x nrhs out): device,
 *   row-major FP32, caller-owned, as for krp_solve_dense.
 *   status: caller-owned device int; the call sets it to zero on `stream`
 *   before its kernels, which raise it to KRP_ESINGULAR (X zero) if M is not
 *   positive definite and flags lacks KRP_PINV_FALLBACK.
 *   stream: cudaStream_t (NULL = legacy default stream).
 * Scratch: a fixed 2.13 MB array in the library's device image (512 partial
 * sums of SAᵀSA and SAᵀSB), needing no initial value.  R > 32 or nrhs > 16 is
 * rejected with KRP_EINVAL (message in krp_last_error(NULL)).  Every call
 * looks up the array's device address in the current context; the first call
 * in a context may load the library's device code there, so make it before
 * capturing any stream.  All calls
 * on one device share the array: calls that overlap in time (other streams,
 * other host threads) race on it and must be serialised by the caller.
 * Returns KRP_OK once both kernels are enqueued. */
krp_status krp_solve_dense_noalloc(int64_t J, int R, const float* SA, const float* weight, const float* B_rows,
                                   int nrhs, float* X, int flags, int* status, void* stream);

/* ------------------------------------------------------------------------
 * Sparse tensors and STS-CP (Sec. 3.3; Alg. 6 CP-ALS; App. A.9).
 *
 * krp_sptensor_create: an N-mode sparse tensor with dims I_host and nnz
 * nonzeros; coords_host[k] (host, int32, nnz entries each) and vals_host
 * (host, FP32).  Builds, for every mode j, an index of the mode-j fibers:
 * nonzeros sorted by a key packing the other modes' coordinates, with the
 * fiber start offsets.  Duplicated coordinates must not occur.  The index
 * lives on the device; the sort runs on the host (as in the paper's
 * preprocessing).  Requires Σ_{k != j} ceil(log2 I_k) <= 63 for every j.
 * ---------------------------------------------------------------------- */
krp_status krp_sptensor_create(krp_sptensor** out, int N, const int64_t* I_host, int64_t nnz,
                               const int32_t* const* coords_host, const float* vals_host,
                               void* stream);
void krp_sptensor_destroy(krp_sptensor* t);

/* Sketched mode-j least-squares solve of Alg. 6 against the tensor's matricization:
 * Y = SBᵀ SA (I_j x R; each sampled tuple's mode-j fiber is looked up in the
 * index and its nonzeros scattered with weight w_s), M = SAᵀSA, U_out = Y M⁻¹
 * (M⁻¹ from FP64 Cholesky).  idx/weight/SA from krp_sample(exclude_j = j).
 * U_out: I_j x R (device).  Allocates scratch on first use. */
krp_status krp_solve_sparse(krp_sampler* s, const krp_sptensor* t, int j, int64_t J,
                            const int32_t* idx, const float* weight, const float* SA,
                            float* U_out, int flags);

/* One STS-CP sweep (one pass of Alg. 6's loop) over all modes j = 0..N-1: draw J
 * samples excluding j (draw id draw_base + j), solve for U_j, set
 * sigma[i] = ||U_j[:,i]||_2, normalise U_j's columns, and rebuild Z_j.
 * sigma: R floats (device), holds the last mode's norms.  The sampler's
 * factors are the ALS state. */
krp_status krp_cp_als_sweep(krp_sampler* s, const krp_sptensor* t, int64_t J, uint64_t seed,
                            uint64_t draw_base, float* sigma);

/* CP fit 1 - ||T~ - T||_F / ||T||_F (Sec. 4.3) of the sampler's factors
 * with weights sigma (device, R floats) against tensor t.  Result written to
 * *fit_host after an internal stream synchronisation. */
krp_status krp_cp_fit(krp_sampler* s, const krp_sptensor* t, const float* sigma, double* fit_host);

/* ------------------------------------------------------------------------
 * Status, inspection.
 * ---------------------------------------------------------------------- */
/* Synchronise the sampler's stream, return and clear the device status word
 * (KRP_OK if no device-side failure), or KRP_ECUDA if the sync failed. */
krp_status krp_sync_status(krp_sampler* s);

/* Number of CUDA kernels this library has launched in the process so far
 * (all samplers; for accounting in benchmarks). */
int64_t krp_launch_count(void);

/* Exact-decision samplers (KRP_PREC_EXACT): number of row-stage descents that
 * have switched to double-float masses since krp_create (a decision or a leaf
 * scan within the near-edge band of Alg. 4's cutoffs; at most one per sample
 * and included factor), written to *count_host after a stream
 * synchronisation.  Zero for other samplers.  No counterpart in the paper. */
krp_status krp_exact_count(krp_sampler* s, int64_t* count_host);

/* Test hook for the device-side wait bound (no counterpart in the paper): the
 * descent's TMA waits give up after a bounded number of suspending tries and
 * set KRP_ETIMEOUT instead of hanging.  This launches one warp that waits on a
 * barrier nothing completes, with `tries` (1..1000) tries of up to ~0.1 ms
 * each; krp_sync_status then returns KRP_ETIMEOUT and the context stays usable. */
krp_status krp_debug_wait_timeout(krp_sampler* s, int tries);

/* Test hook for the stable radix sort behind krp_solve_sparse (no
 * counterpart in the paper): sorts n (key, value) pairs of device uint32
 * arrays in place by the low `bits` bits of the keys (1..32), equal keys in
 * their input order.  Allocates temporary arrays; synchronous on `stream`. */
krp_status krp_debug_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, void* stream);

/* Message for the most recent failure on this sampler; never NULL. */
const char* krp_last_error(const krp_sampler* s);

/* krp_sample (without logq/SA) that also records, for samples 0..n_trace-1,
 * every branch the descent evaluated (Alg. 4): trace (device,
 * float) is laid out [n_trace][n_included][2 stages: eigencomponent, row][66]
 * with [0] = root mass C and, for level l = 0..depth-1, [2+2l] = mass of the
 * left child m(L(c)) and [3+2l] = mass of the current node m(c) (the right
 * child inherits m(c) - m(L(c))).  The left-branch probability at level l is
 * [2+2l]/[3+2l].  For tests; same draws as krp_sample with the same
 * arguments. */
krp_status krp_debug_trace(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id,
                           int32_t* idx, float* weight, float* trace, int64_t n_trace);

/* Tree geometry of factor j: padded leaf count L, depth d = log2 L, and the
 * node stride (floats) of the stored upper triangles. */
krp_status krp_tree_info(const krp_sampler* s, int j, int64_t* L_host, int* depth_host,
                         int* node_stride_host);

/* Copy factor j's segment tree to host memory (L * node_stride floats).
 * Slot 0 is the root G_j; slot v/2 holds the left child v (v even) in heap
 * numbering (root 1, children 2v, 2v+1, leaf b = node L + b).  Each slot is
 * the upper triangle of G^v packed row by row, then zero padding.  Synchronous. */
krp_status krp_get_tree(const krp_sampler* s, int j, float* out_host, int64_t n_floats);

/* Exact-decision samplers (KRP_PREC_EXACT): copy factor j's low parts (the
 * slot layout of krp_get_tree, L * node_stride floats: slot value = tree +
 * low part, a double-float) and/or its delta-encoded top (2^Ke *
 * node_stride floats, Ke = min(10, depth), in the tree's slot numbering: the
 * root, then for slot c = 1 .. 2^Ke - 1 the FP32 rounding of G_{2c} - alpha_c
 * G_c with alpha_c = rows(2c) / rows(c) rounded to FP32) to host; NULL skips
 * either.
 * KRP_EINVAL for other samplers or short buffers.  Synchronous. */
krp_status krp_get_tree_exact(const krp_sampler* s, int j, float* lo_host, int64_t n_lo, float* dtop_host,
                              int64_t n_dtop);

/* Copy the sampler's copy of factor j (I_j x R row-major FP32, n_floats >=
 * I_j R) to host memory: what krp_set_factor stored, or what the last
 * krp_cp_als_sweep (or krp_update_entries) left there.  KRP_EINVAL if factor j
 * was never set.  Synchronous. */
krp_status krp_get_factor(const krp_sampler* s, int j, float* out_host, int64_t n_floats);

/* After krp_sample: copy the FP64 eigendecomposition of G_{>k} used for
 * included factor k (lam: R values ascending, V: R x R row-major with
 * eigenvector u in column u), the FP64 G⁺ (R x R) and rank(A).  Any pointer
 * may be NULL.  Synchronous. */
krp_status krp_get_prep(const krp_sampler* s, int k, double* lam_host, double* V_host,
                        double* Gplus_host, int* rank_host);

/* Least-squares accuracy (Sec. 4.2).
 * krp_kron_rows: B_rows[s] = Π_{k != exclude_j} c_k[idx[k][s]], the entries of
 * b = c_1 ⊗ ... ⊗ c_N at the sampled tuples (black-box access: b is never
 * formed).  c_host[k]: device pointer to c_k (I_k floats; NULL allowed for
 * k = exclude_j); B_rows: J floats (device).
 * krp_sketch_distortion: D(S, A) = kappa(SQ) - 1 (Eq. distortion_defn) for the
 * sketch SA (J x R, device, e.g. krp_sample's SA) of A = ⊙_{k != exclude_j} U_k,
 * without forming A or a basis of its range: kappa(SQ) = kappa(SA V Σ⁻¹) with
 * AᵀA = ⊛ U_kᵀU_k = V Σ² Vᵀ (appendix on computing sketch distortion), from
 * FP32 partial sums of SAᵀSA and FP64 eigendecompositions.  Needs a
 * preparation (krp_sample / krp_sample_prepare) since the last factor change;
 * writes D (inf if SQ is rank-deficient) and rank(A) to host; synchronous. */
krp_status krp_kron_rows(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx, const float* const* c_host,
                         float* B_rows);
krp_status krp_sketch_distortion(krp_sampler* s, int exclude_j, int64_t J, const float* SA, double* D_host,
                                 int* rank_host);

/* CUDA-graph capture of a sampler's calls (no counterpart in the paper):
 * between krp_capture_begin and krp_capture_end the sampler's calls on its
 * stream are recorded, not run (end reports the node count); krp_replay runs
 * the recorded sequence again with the arguments given at capture (e.g. one
 * whole STS-CP sweep, krp_cp_als_sweep).  The sampler must have been created
 * with its own stream.  Make each call once before capturing, so that no
 * scratch grows during capture; calls that synchronise (krp_sync_status,
 * krp_cp_fit, copies to host) must not be captured. */
krp_status krp_capture_begin(krp_sampler* s);
krp_status krp_capture_end(krp_sampler* s, int64_t* nodes_host);
krp_status krp_replay(krp_sampler* s);

/* ------------------------------------------------------------------------
 * Planted right-hand side (a synthetic workload; no counterpart in the paper).
 *
 * krp_planted_rows: B_rows[s, c] = a_s · X_true[:, c] + sigma * xi(s, c) for the
 * sampled tuples s of krp_sample (idx, same exclude_j), where a_s =
 * ⊛_{k != exclude_j} U_k[idx[k][s], :] is row s of A.  X_true: R x nrhs (device,
 * row-major); B_rows: J x nrhs (device).  xi is a standard normal by Box–Muller
 * from Philox4x32-10 with key (seed lo32, seed hi32) and counter (lin lo32,
 * lin hi32, c, 0x9E3779B9), lin = the C-order linear index of the tuple over
 * the included factors mod 2^64, so repeated tuples get the same noise.
 * 1 <= nrhs <= 64.  Asynchronous on the sampler's stream.
 * ---------------------------------------------------------------------- */
krp_status krp_planted_rows(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx, const float* X_true,
                            int nrhs, float sigma, uint64_t seed, float* B_rows);

/* ------------------------------------------------------------------------
 * Batches of independent problems: every phase of the path (tree builds,
 * preparation, descent, planted right-hand side, dense solve) as one launch
 * over all P problems (Alg. 1-4 and Thm 2.1 applied to each problem), and
 * the whole sequence capturable as one CUDA graph.
 *
 * krp_batch_create: a batch over P existing samplers (not owned; they must
 * outlive the batch), all with the same N, R <= 32, F <= 32 and every factor
 * set.  No factor is excluded.  `stream` (a cudaStream_t, not NULL if the
 * batch is to be captured) carries all batch work; the samplers' own streams
 * are not used.  Allocates the per-problem parameter tables and scratch.
 *
 * Packed layouts (device): idx [P][N][J] int32; weight [P][J]; SA: problem p's
 * J x R_p rows at SA + J * Roff[p]; B_rows [P][J][nrhs]; X_true and X: problem
 * p's R_p x nrhs at X + Roff[p] * nrhs, where Roff[p] = R_0 + ... + R_{p-1}.
 *
 * krp_batch_set_sources: U_host[p * N + k] = device pointer to problem p's new
 * factor k (I_k x R_p) or NULL for "rebuild from the sampler's copy"; U_host
 * NULL = all NULL.  The next krp_batch_build copies each given factor into
 * its sampler while building.  Updates a device table in place (synchronous),
 * so a captured graph uses the sources bound when it runs.  Not while capturing.
 * krp_batch_build: rebuild every tree (FP32 Grams, Alg. 3).
 * krp_batch_sample: per problem, the preparation of Alg. 2 and J samples (the
 * per-problem uniforms of krp_sample with the same seed and draw_id); SA may
 * be NULL.  krp_batch_planted_rows / krp_batch_solve_dense: krp_planted_rows
 * and krp_solve_dense for every problem (1 <= nrhs <= 16 for the solve).
 * krp_batch_sync_status: synchronise; the first device status found (batch,
 * then samplers), cleared.
 * krp_batch_capture_begin / _end: record the batch calls made in between on
 * the batch stream into a CUDA graph instead of running them (end reports
 * the graph's node count); run each call once before capturing, so that no
 * scratch needs to grow during capture.  krp_batch_replay: launch that graph.
 * krp_batch_set_tuning: descent CTAs per problem (1..64).  krp_batch_autotune:
 * time the sampling phase for 1, 2, 4, 8, 16 CTAs per problem at this J and
 * keep the fastest (allocates and frees temporary outputs; synchronous).
 * ---------------------------------------------------------------------- */
typedef struct krp_batch krp_batch;
krp_status krp_batch_create(krp_batch** out, krp_sampler* const* samplers_host, int P, void* stream);
void krp_batch_destroy(krp_batch* b);
krp_status krp_batch_set_sources(krp_batch* b, const float* const* U_host);
krp_status krp_batch_build(krp_batch* b);
krp_status krp_batch_sample(krp_batch* b, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx, float* weight,
                            float* SA);
krp_status krp_batch_planted_rows(krp_batch* b, int64_t J, const int32_t* idx, const float* X_true, int nrhs,
                                  float sigma, uint64_t seed, float* B_rows);
krp_status krp_batch_solve_dense(krp_batch* b, int64_t J, const float* SA, const float* weight, const float* B_rows,
                                 int nrhs, float* X, int flags);
krp_status krp_batch_sync_status(krp_batch* b);
krp_status krp_batch_capture_begin(krp_batch* b);
krp_status krp_batch_capture_end(krp_batch* b, int64_t* nodes_host);
krp_status krp_batch_replay(krp_batch* b);
krp_status krp_batch_set_tuning(krp_batch* b, int descent_ctas_per_problem);
krp_status krp_batch_autotune(krp_batch* b, int64_t J, int* best_host);
const char* krp_batch_last_error(const krp_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* KRPLS_H */
