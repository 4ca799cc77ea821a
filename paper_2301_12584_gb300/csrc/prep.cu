// a2 + a3: per-draw sampler preparation (the set-up steps of Alg. 2; Eq. G_geq_k_defn;
// Eq. first_dist; Sec. 3.2).
//
// prep_pinv (1 CTA): G = ⊛_{k incl} G_k from the trees' FP32 roots, in FP64;
//   G⁺ by FP64 Cholesky inverse when the exact 1-norm condition number of the
//   result is <= 1e10 (then no eigenvalue is near the pseudo-inverse cutoff and
//   G⁺ = G⁻¹), otherwise by the FP64 Jacobi eigen-pseudo-inverse with cutoff
//   R * 2^-52 * lam_max.  rank(A) = number of kept eigenvalues.
// prep_eig (one CTA per included factor k): G_{>k} = G⁺ ⊛ ⊛_{m>k incl} G_m,
//   its eigendecomposition (cyclic Jacobi with round-robin pairs, in FP32 or
//   FP64), eigenvalues ascending with negatives clamped to zero, and the
//   eigencomponent tree E_k = BuildSampler(√Λ Vᵀ, F = 1, Y = G_k): leaf u holds
//   λ_u V_u V_uᵀ, internal nodes the pairwise sums, every stored node
//   multiplied entrywise by G_k so that its mass for history h is hᵀ P^v h.
#include "common.cuh"
#include "internal.h"
#include "jacobi.cuh"

#include <math.h>

namespace krp {

// Rank of each eigenvalue in ascending order (ties by index) -> position.
__device__ void ascending_positions(const double* lam, int n, int* pos) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int r = 0;
        for (int j = 0; j < n; ++j) r += (lam[j] < lam[i]) || (lam[j] == lam[i] && j < i);
        pos[i] = r;
    }
}


// Block-wide sum of one double per thread (fixed order, every thread gets it).
__device__ double block_sum(double v, double* red) {
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition of an n x n FP64 matrix A (row-major), one CTA:
// cyclic Jacobi in FP32 on A / max|A| (fast on GB300, whose FP64 rate is low),
// then one FP64 refinement step of Ogita & Aishima ("Iterative refinement for
// symmetric eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018):
//   Rm = I - XᵀX, S = Xᵀ A X, λ_i = S_ii / (1 - Rm_ii),
//   E_ij = (S_ij + λ_j Rm_ij) / (λ_j - λ_i) if |λ_i - λ_j| > δ else Rm_ij / 2,
//   δ = 2 (||S - diag λ||_F + ||A||_F ||Rm||_F),  X <- X + X E,
// which takes FP32-accurate eigenpairs to about 1e-14.
// On exit X holds the eigenvectors in its columns and lam the eigenvalues
// (unsorted).  Work: Af, Vf (n*n floats), As, S, T, Rm (n*n doubles), cs/pr.
// ---------------------------------------------------------------------------
struct EigWork {
    float* Af;
    float* Vf;
    double* As;
    double* S;
    double* T;
    double* Rm;
    float* csf;
    int* pr;
    double* red;
};

// Scale A by max |A| into w.As (FP64) and w.Af (FP32), FP32 Jacobi, X = the
// FP32 eigenvectors in FP64.  Returns the scale.
__device__ double eig_fp32_start(const double* __restrict__ A, int n, double* __restrict__ X, EigWork w) {
    const int nn = n * n;
    double mx = 0.0;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) mx = fmax(mx, fabs(A[e]));
    __shared__ double s_mx;
    if (threadIdx.x == 0) s_mx = 0.0;
    __syncthreads();
    // block max through atomics on a shared double (as bits; values are >= 0)
    atomicMax(reinterpret_cast<unsigned long long*>(&s_mx), __double_as_longlong(mx));
    __syncthreads();
    const double scale = s_mx > 0.0 ? s_mx : 1.0;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const double a = A[e] / scale;
        w.As[e] = a;
        w.Af[e] = (float)a;
    }
    __syncthreads();
    jacobi_eig<float>(w.Af, w.Vf, n, w.csf, w.pr, w.red, 30, 4e-7);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) X[e] = (double)w.Vf[e];
    __syncthreads();
    return scale;
}

// steps: refinement steps (each roughly squares the eigenvectors' error, down to
// FP64 rounding over the eigenvalue gaps).
__device__ void eig_fp32_refined(const double* __restrict__ A, int n, double* __restrict__ X, double* __restrict__ lam,
                                 EigWork w, int steps = 1) {
    const int nn = n * n;
    const double scale = eig_fp32_start(A, n, X, w);
    for (int step = 0; step < steps; ++step) {
        // Rm = I - XᵀX ; T = As X
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double r = (i == j) ? 1.0 : 0.0, t = 0.0;
            for (int k = 0; k < n; ++k) {
                r -= X[k * n + i] * X[k * n + j];
                t += w.As[i * n + k] * X[k * n + j];
            }
            w.Rm[e] = r;
            w.T[e] = t;
        }
        __syncthreads();
        // S = Xᵀ T
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += X[k * n + i] * w.T[k * n + j];
            w.S[e] = acc;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = w.S[i * n + i] / (1.0 - w.Rm[i * n + i]);
        __syncthreads();
        double off = 0.0, an = 0.0, rn = 0.0;
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            const double sd = w.S[e] - (i == j ? lam[i] : 0.0);
            off += sd * sd;
            an += w.As[e] * w.As[e];
            rn += w.Rm[e] * w.Rm[e];
        }
        off = block_sum(off, w.red);
        an = block_sum(an, w.red);
        rn = block_sum(rn, w.red);
        const double delta = 2.0 * (sqrt(off) + sqrt(an) * sqrt(rn));
        // E into T
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double E;
            if (i == j)
                E = 0.5 * w.Rm[e];
            else if (fabs(lam[i] - lam[j]) > delta)
                E = (w.S[e] + lam[j] * w.Rm[e]) / (lam[j] - lam[i]);
            else
                E = 0.5 * w.Rm[e];
            w.T[e] = E;
        }
        __syncthreads();
        // X <- X + X E (into S, then copy)
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double acc = X[e];
            for (int k = 0; k < n; ++k) acc += X[i * n + k] * w.T[k * n + j];
            w.S[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nn; e += blockDim.x) X[e] = w.S[e];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] *= scale;
    __syncthreads();
}

// Shared-memory carve-up for eig_fp32_refined plus extras; FP64 matrices go to
// `gwork` (global) when `gwork` is non-null.
__device__ EigWork carve(char* base, int n, double* gwork, double** X, double** A64, double** lam, int** pos) {
    const int nn = n * n;
    EigWork w;
    char* p = base;
    w.red = reinterpret_cast<double*>(p);
    p += 64 * 8;
    *lam = reinterpret_cast<double*>(p);
    p += (size_t)n * 8;
    *pos = reinterpret_cast<int*>(p);
    p += (size_t)((n + 1) & ~1) * 4;
    w.pr = reinterpret_cast<int*>(p);
    p += (size_t)2 * (n / 2 + 1) * 4 + 8;
    w.csf = reinterpret_cast<float*>(p);
    p += (size_t)2 * (n / 2 + 1) * 4 + 8;
    p = reinterpret_cast<char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    w.Af = reinterpret_cast<float*>(p);
    p += (size_t)nn * 4;
    w.Vf = reinterpret_cast<float*>(p);
    p += (size_t)nn * 4;
    p = reinterpret_cast<char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    double* d = gwork ? gwork : reinterpret_cast<double*>(p);
    w.As = d;
    w.S = d + nn;
    w.T = d + 2 * (size_t)nn;
    w.Rm = d + 3 * (size_t)nn;
    *X = d + 4 * (size_t)nn;
    *A64 = d + 5 * (size_t)nn;
    return w;
}

__host__ size_t carve_smem_bytes(int n, bool fp64_in_smem) {
    const size_t nn = (size_t)n * n;
    size_t b = 64 * 8 + (size_t)n * 8 + (size_t)((n + 1) & ~1) * 4 + 2 * ((size_t)2 * (n / 2 + 1) * 4 + 8) + 32;
    b += 2 * nn * 4 + 16;
    if (fp64_in_smem) b += 6 * nn * 8;
    return b;
}

// ---------------------------------------------------------------------------
// prep_pinv (one CTA): G = ⊛ G_k (FP64), G⁺ and rank.
// Well-conditioned G (exact 1-norm condition number <= 1e10, so no eigenvalue
// is near the cutoff): G⁺ = G⁻¹ from an FP64 Cholesky factor.  Otherwise the
// eigen-pseudo-inverse with cutoff R * 2^-52 * lam_max.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prep_pinv_body(const PrepParams& P, int N, int exclude, int R, int Tp,
                                               double* __restrict__ G64, double* __restrict__ Gplus64,
                                               float* __restrict__ Gplus32, int* __restrict__ rank_out,
                                               int* __restrict__ status, double* __restrict__ gwork) {
    extern __shared__ __align__(16) char smp[];
    const int RR = R * R;
    double *X, *A64, *lam;
    int* pos;
    EigWork w = carve(smp, R, gwork, &X, &A64, &lam, &pos);
    double* G = A64;        // R x R
    double* Lm = w.S;       // Cholesky factor (lower)
    double* Li = w.T;       // L⁻¹ (lower)
    double* Gi = w.Rm;      // G⁻¹
    __shared__ double s_inv[128];
    __shared__ double s_c1[128], s_c2[128];
    __shared__ int flag;
    for (int e = threadIdx.x; e < RR; e += blockDim.x) G[e] = 1.0;
    for (int k = 0; k < N; ++k) {
        const double* rt = P.roots[k];
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            const int i = e / R, j = e % R;
            const double v = rt[tri_index(min(i, j), max(i, j), R)];
            G64[(size_t)k * RR + e] = v;
            if (k != exclude) G[e] *= v;
        }
    }
    if (threadIdx.x == 0) flag = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += blockDim.x) Lm[e] = G[e];
    __syncthreads();
    for (int c = 0; c < R; ++c) {
        if (threadIdx.x == 0) {
            const double d = Lm[c * R + c];
            if (!(d > 0.0)) flag = 1;
            const double l = d > 0.0 ? sqrt(d) : 1.0;
            Lm[c * R + c] = l;
            s_inv[c] = 1.0 / l;
        }
        __syncthreads();
        const double ic = s_inv[c];
        for (int i = c + 1 + threadIdx.x; i < R; i += blockDim.x) Lm[i * R + c] *= ic;
        __syncthreads();
        const int n = R - c - 1;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = c + 1 + e / n, j = c + 1 + e % n;
            if (j <= i) Lm[i * R + j] -= Lm[i * R + c] * Lm[j * R + c];
        }
        __syncthreads();
    }
    if (!flag) {
        for (int col = threadIdx.x; col < R; col += blockDim.x) {   // L⁻¹, column by column
            for (int i = 0; i < R; ++i) {
                double acc = (i == col) ? 1.0 : 0.0;
                for (int k = col; k < i; ++k) acc -= Lm[i * R + k] * Li[k * R + col];
                Li[i * R + col] = (i >= col) ? acc * s_inv[i] : 0.0;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {        // G⁻¹ = L⁻ᵀ L⁻¹
            const int i = e / R, j = e % R;
            double acc = 0.0;
            for (int k = max(i, j); k < R; ++k) acc += Li[k * R + i] * Li[k * R + j];
            Gi[e] = acc;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < R; j += blockDim.x) {         // column abs sums
            double ca = 0.0, cb = 0.0;
            for (int i = 0; i < R; ++i) {
                ca += fabs(G[i * R + j]);
                cb += fabs(Gi[i * R + j]);
            }
            s_c1[j] = ca;
            s_c2[j] = cb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int j = 0; j < R; ++j) {
                a = fmax(a, s_c1[j]);
                b = fmax(b, s_c2[j]);
            }
            if (!(a * b <= 1e10)) flag = 1;
        }
        __syncthreads();
    }
    int rank = R;
    if (!flag) {
        for (int e = threadIdx.x; e < RR; e += blockDim.x) Gplus64[e] = Gi[e];
    } else {
        eig_fp32_refined(G, R, X, lam, w);
        // The refinement's eigenvalues are first-order estimates from the
        // unrefined vectors: a cluster of zero eigenvalues comes out near
        // 1e-14 lambda_max, above the cutoff R 2^-52 lambda_max, and would be
        // inverted.  Rayleigh quotients of the refined vectors are accurate to
        // ~eps^2 there.  (T = G X into w.T, free after the refinement.)
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            const int i = e / R, j = e % R;
            double acc = 0.0;
            for (int k = 0; k < R; ++k) acc = fma(G[i * R + k], X[k * R + j], acc);
            w.T[e] = acc;
        }
        __syncthreads();
        for (int u = threadIdx.x; u < R; u += blockDim.x) {
            double num = 0.0, den = 0.0;
            for (int i = 0; i < R; ++i) {
                num = fma(X[i * R + u], w.T[i * R + u], num);
                den = fma(X[i * R + u], X[i * R + u], den);
            }
            lam[u] = den > 0.0 ? num / den : 0.0;
        }
        __syncthreads();
        double lmax = 0.0;
        for (int i = 0; i < R; ++i) lmax = fmax(lmax, lam[i]);
        const double cut = R * 2.220446049250313e-16 * lmax;
        rank = 0;
        for (int i = 0; i < R; ++i) rank += lam[i] > cut;
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            const int i = e / R, j = e % R;
            double acc = 0.0;
            for (int u = 0; u < R; ++u)
                if (lam[u] > cut) acc += X[i * R + u] * X[j * R + u] / lam[u];
            Gplus64[e] = acc;
        }
    }
    __syncthreads();
    // FP32 copy of G⁺ scaled by 2^-gexp (gexp from its largest entry, kept in
    // rank_out[1]): G⁺ ~ 1 / Π_k ||U_k||² leaves the FP32 range for many or
    // large factors, while the weights need only hᵀ G⁺ h up to that factor
    double gm = 0.0;
    for (int e = threadIdx.x; e < RR; e += blockDim.x) gm = fmax(gm, fabs(Gplus64[e]));
    for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if ((threadIdx.x & 31) == 0) s_c1[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, s_c1[q]);
        s_c1[0] = m;
    }
    __syncthreads();
    const int gexp = (s_c1[0] > 0.0 && isfinite(s_c1[0])) ? ilogb(s_c1[0]) : 0;
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        float v = 0.f;
        if (e < tri_size(R)) {
            int i = 0, rem = e;
            while (rem >= R - i) {
                rem -= R - i;
                ++i;
            }
            v = (float)ldexp(Gplus64[i * R + i + rem], -gexp);
        }
        Gplus32[e] = v;
    }
    if (threadIdx.x == 0) {
        rank_out[0] = rank;
        rank_out[1] = gexp;
        if (rank == 0) set_status(status, KRP_EZERO);
    }
}

// ---------------------------------------------------------------------------
// prep_eig: one CTA per included factor k: G_{>k}, its eigendecomposition
// (eig_fp32_refined), eigenvalues ascending with negatives clamped to zero,
// eigenvectors as FP64 columns, FP32 rows and FP32 residual rows (E_k is
// built from them by prep_etree).
// ---------------------------------------------------------------------------
// Eigenvalues clamped to >= 0 and put in ascending order; eigenvectors as
// FP64 columns, FP32 rows and FP32 residual rows (the outputs of prep_eig).
__device__ __forceinline__ void eig_output(int k, int R, const double* __restrict__ X, double* lam, int* pos,
                                           double* __restrict__ lam64, double* __restrict__ V64,
                                           float* __restrict__ V32, float* __restrict__ V32lo) {
    const int RR = R * R;
    for (int i = threadIdx.x; i < R; i += blockDim.x) lam[i] = fmax(lam[i], 0.0);
    __syncthreads();
    ascending_positions(lam, R, pos);
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        const int row = e / R, u = e % R;   // X[row][u], eigenvector u in column u
        const int o = pos[u];
        const double v = X[e];
        V64[(size_t)k * RR + row * R + o] = v;
        const float vh = (float)v;
        V32[(size_t)k * RR + o * R + row] = vh;   // row o = eigenvector
        V32lo[(size_t)k * RR + o * R + row] = (float)(v - (double)vh);
    }
    for (int u = threadIdx.x; u < R; u += blockDim.x) lam64[(size_t)k * R + pos[u]] = lam[u];
}

// split: stop after the FP32 Jacobi, leaving As and X in gwork and the scale
// in scales[p]; the refinement then runs over many CTAs (refine_* below).
__device__ __forceinline__ void prep_eig_body(const PrepParams& P, int N, int R, int Rp, int dE, int Tp,
                                              const double* __restrict__ G64, const double* __restrict__ Gplus64,
                                              double* __restrict__ lam64, double* __restrict__ V64,
                                              float* __restrict__ V32, float* __restrict__ V32lo,
                                              float* __restrict__ etree, double* __restrict__ gwork, int p,
                                              bool split = false, double* __restrict__ scales = nullptr) {
    extern __shared__ __align__(16) char smp[];
    const int RR = R * R;
    const int n_incl = P.n_incl;
    const int k = P.incl[p];
    double *X, *A64, *lam;
    int* pos;
    EigWork w = carve(smp, R, gwork ? gwork + (size_t)p * 6 * RR : nullptr, &X, &A64, &lam, &pos);
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {     // G_{>k} = G⁺ ⊛ ⊛_{m>k} G_m
        double v = Gplus64[e];
        for (int q = p + 1; q < n_incl; ++q) v *= G64[(size_t)P.incl[q] * RR + e];
        A64[e] = v;
    }
    __syncthreads();
    if (split) {
        const double scale = eig_fp32_start(A64, R, X, w);
        if (threadIdx.x == 0) scales[p] = scale;
        return;
    }
    eig_fp32_refined(A64, R, X, lam, w, 1 + P.extra_refine);
    eig_output(k, R, X, lam, pos, lam64, V64, V32, V32lo);
}

// ---------------------------------------------------------------------------
// The Ogita–Aishima refinement step of eig_fp32_refined for R > 32, spread
// over CTAs: GB300 runs FP64 at ~1/64 of FP32, so the four R x R products on
// one SM dominate the preparation there.  Per included factor p the work area
// holds six R x R FP64 matrices: [0] As (scaled G_{>k}), [1] S, [2] T,
// [3] Rm, [4] X, [5] the input (then λ).  Steps: T = As X and Rm = I - XᵀX;
// S = Xᵀ T; λ, δ and E (into [2]) in one CTA per factor; X + X E (into [1]);
// then the outputs of eig_output.
// ---------------------------------------------------------------------------
constexpr int RG_TILE = 16;

// C = eye I + sign op(A) B + Add, on 16 x 16 output tiles; matrices are
// indices into the factor's six (Add: -1 for none); op(A) = Aᵀ if transA.
__global__ void __launch_bounds__(RG_TILE * RG_TILE) refine_gemm(double* __restrict__ work, int n, int iA, int iB,
                                                                 int iC, int iAdd, int transA, int eye,
                                                                 double sign) {
    const size_t RR = (size_t)n * n;
    double* base = work + (size_t)blockIdx.z * 6 * RR;
    const double* A = base + iA * RR;
    const double* B = base + iB * RR;
    double* C = base + iC * RR;
    const double* Add = iAdd >= 0 ? base + iAdd * RR : nullptr;
    __shared__ double sA[RG_TILE][RG_TILE + 1], sB[RG_TILE][RG_TILE + 1];
    const int ty = threadIdx.x / RG_TILE, tx = threadIdx.x % RG_TILE;
    const int i = blockIdx.y * RG_TILE + ty, j = blockIdx.x * RG_TILE + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < n; k0 += RG_TILE) {
        const int ia = blockIdx.y * RG_TILE + ty, ka = k0 + tx;   // op(A)[ia][ka]
        sA[ty][tx] = (ia < n && ka < n) ? (transA ? A[(size_t)ka * n + ia] : A[(size_t)ia * n + ka]) : 0.0;
        const int kb = k0 + ty;
        sB[ty][tx] = (kb < n && j < n) ? B[(size_t)kb * n + j] : 0.0;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < RG_TILE; ++kk) acc = fma(sA[ty][kk], sB[kk][tx], acc);
        __syncthreads();
    }
    if (i < n && j < n)
        C[(size_t)i * n + j] = (eye && i == j ? 1.0 : 0.0) + sign * acc + (Add ? Add[(size_t)i * n + j] : 0.0);
}

// λ_i = S_ii / (1 - Rm_ii), δ, and E into slot [2] (one CTA per factor).
__global__ void __launch_bounds__(1024) refine_mid(double* __restrict__ work, int n) {
    __shared__ double red[64];
    __shared__ double lam[128];
    const size_t RR = (size_t)n * n;
    double* base = work + (size_t)blockIdx.x * 6 * RR;
    const double *As = base, *S = base + RR, *Rm = base + 3 * RR;
    double* E = base + 2 * RR;
    double* lam_out = base + 5 * RR;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        lam[i] = S[(size_t)i * n + i] / (1.0 - Rm[(size_t)i * n + i]);
        lam_out[i] = lam[i];
    }
    __syncthreads();
    double off = 0.0, an = 0.0, rn = 0.0;
    for (size_t e = threadIdx.x; e < RR; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const double sd = S[e] - (i == j ? lam[i] : 0.0);
        off += sd * sd;
        an += As[e] * As[e];
        rn += Rm[e] * Rm[e];
    }
    off = block_sum(off, red);
    an = block_sum(an, red);
    rn = block_sum(rn, red);
    const double delta = 2.0 * (sqrt(off) + sqrt(an) * sqrt(rn));
    for (size_t e = threadIdx.x; e < RR; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        double v;
        if (i == j)
            v = 0.5 * Rm[e];
        else if (fabs(lam[i] - lam[j]) > delta)
            v = (S[e] + lam[j] * Rm[e]) / (lam[j] - lam[i]);
        else
            v = 0.5 * Rm[e];
        E[e] = v;
    }
}

// The refined X (slot [1]) and λ (slot [5]) times the scale, to the outputs.
__global__ void __launch_bounds__(1024) refine_finish(const __grid_constant__ PrepParams P, double* __restrict__ work,
                                                      int n, const double* __restrict__ scales,
                                                      double* __restrict__ lam64, double* __restrict__ V64,
                                                      float* __restrict__ V32, float* __restrict__ V32lo) {
    __shared__ double lam[128];
    __shared__ int pos[128];
    const size_t RR = (size_t)n * n;
    const int p = blockIdx.x;
    const double* base = work + (size_t)p * 6 * RR;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = base[5 * RR + i] * scales[p];
    __syncthreads();
    eig_output(P.incl[p], n, base + RR, lam, pos, lam64, V64, V32, V32lo);
}

// ---------------------------------------------------------------------------
// E_k (a3) from the sorted eigenpairs that prep_eig wrote: per packed entry
// e = (i, j) (one thread each, CTAs spread over the entries), leaves
// u = 0..Rp-1 hold λ_u V[i,u] V[j,u] (zero for u >= R); binary-counter
// pairwise sums up the tree; stored nodes multiplied by G_k[i,j].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void etree_body(int k, int R, int Rp, int Tp, const double* __restrict__ G64,
                                           const double* __restrict__ lam64, const double* __restrict__ V64,
                                           float* __restrict__ etree, int e) {
    const int RR = R * R;
    const double* lk = lam64 + (size_t)k * R;
    const double* Vk = V64 + (size_t)k * RR;
    const double* Gk = G64 + (size_t)k * RR;
    float* et = etree + (size_t)k * Rp * Tp;
    const int T = tri_size(R);
    // E_k's masses are compared only with each other, so its nodes carry a
    // power-of-two scale that keeps them near 1 in FP32 (λ_max(G_{>k}) can
    // be ~2^-144 for the last of many factors)
    __shared__ double s_esc;
    if (threadIdx.x == 0) {
        double gkmax = 0.0;
        for (int i = 0; i < R; ++i) gkmax = fmax(gkmax, Gk[i * R + i]);
        const double emag = lk[R - 1] * gkmax;
        s_esc = (emag > 0.0 && isfinite(emag)) ? ldexp(1.0, -ilogb(emag)) : 1.0;
    }
    __syncthreads();
    const double esc = s_esc;
    if (e >= Tp) return;
    if (e >= T) {
        for (int sl = 0; sl < Rp; ++sl) et[(size_t)sl * Tp + e] = 0.f;
        return;
    }
    int i = 0, rem = e;
    while (rem >= R - i) {
        rem -= R - i;
        ++i;
    }
    const int j = i + rem;
    const double gij = Gk[i * R + j] * esc;
    double stk[8];
    for (int u = 0; u < Rp; ++u) {
        double val = (u < R) ? lk[u] * Vk[i * R + u] * Vk[j * R + u] : 0.0;
        int64_t h = Rp + u;
        if (tree_stored(h)) et[tree_slot(h) * Tp + e] = (float)(val * gij);
        int idx = u, lvl = 0;
        while (idx & 1) {
            val = stk[lvl] + val;
            h >>= 1;
            idx >>= 1;
            ++lvl;
            if (tree_stored(h)) et[tree_slot(h) * Tp + e] = (float)(val * gij);
        }
        stk[lvl] = val;
    }
}

constexpr int ETREE_THREADS = 128;

size_t carve_smem_bytes(int n, bool fp64_in_smem);

__global__ void __launch_bounds__(1024) prep_pinv(const __grid_constant__ PrepParams P, int N, int exclude, int R,
                                                 int Tp, double* __restrict__ G64, double* __restrict__ Gplus64,
                                                 float* __restrict__ Gplus32, int* __restrict__ rank_out,
                                                 int* __restrict__ status, double* __restrict__ gwork) {
    prep_pinv_body(P, N, exclude, R, Tp, G64, Gplus64, Gplus32, rank_out, status, gwork);
}

__global__ void __launch_bounds__(1024) prep_eig(const __grid_constant__ PrepParams P, int N, int R, int Rp, int dE,
                                                int Tp, const double* __restrict__ G64,
                                                const double* __restrict__ Gplus64, double* __restrict__ lam64,
                                                double* __restrict__ V64, float* __restrict__ V32,
                                                float* __restrict__ V32lo, float* __restrict__ etree,
                                                double* __restrict__ gwork, int split, double* __restrict__ scales) {
    prep_eig_body(P, N, R, Rp, dE, Tp, G64, Gplus64, lam64, V64, V32, V32lo, etree, gwork, blockIdx.x, split != 0,
                  scales);
}

// grid (entry blocks, included factors)
__global__ void __launch_bounds__(ETREE_THREADS) prep_etree(const __grid_constant__ PrepParams P, int R, int Rp, int Tp,
                                                            const double* __restrict__ G64,
                                                            const double* __restrict__ lam64,
                                                            const double* __restrict__ V64, float* __restrict__ etree) {
    etree_body(P.incl[blockIdx.y], R, Rp, Tp, G64, lam64, V64, etree, blockIdx.x * ETREE_THREADS + threadIdx.x);
}

// Batched forms: CTA b of prep_pinv_batch prepares problem b; CTA b of
// prep_eig_batch the included factor b % n_incl of problem b / n_incl.
__global__ void __launch_bounds__(256) prep_pinv_batch(const PrepItem* __restrict__ items) {
    const PrepItem& it = items[blockIdx.x];
    prep_pinv_body(it.P, it.N, it.exclude, it.R, it.Tp, it.G64, it.Gplus64, it.Gplus32, it.rank, it.status,
                   it.gwork);
}
__global__ void __launch_bounds__(256) prep_eig_batch(const PrepItem* __restrict__ items, int n_incl) {
    const PrepItem& it = items[blockIdx.x / n_incl];
    const int p = blockIdx.x % n_incl;
    prep_eig_body(it.P, it.N, it.R, it.Rp, it.dE, it.Tp, it.G64, it.Gplus64, it.lam64, it.V64, it.V32, it.V32lo,
                  it.etree, it.gwork ? it.gwork + (size_t)p * 6 * it.R * it.R : nullptr, p);
}
// grid (entry blocks of the largest Tp, problems x included factors)
__global__ void __launch_bounds__(ETREE_THREADS) prep_etree_batch(const PrepItem* __restrict__ items, int n_incl) {
    const PrepItem& it = items[blockIdx.y / n_incl];
    if ((int)(blockIdx.x * ETREE_THREADS) >= it.Tp) return;   // uniform across the CTA
    etree_body(it.P.incl[blockIdx.y % n_incl], it.R, it.Rp, it.Tp, it.G64, it.lam64, it.V64, it.etree,
               blockIdx.x * ETREE_THREADS + threadIdx.x);
}

void prep_item_for(const krp_sampler* s, int exclude_j, PrepItem* it) {
    PrepItem& x = *it;
    x = PrepItem{};
    x.P.n_incl = 0;
    for (int k = 0; k < s->N; ++k) {
        x.P.roots[k] = s->root64[k];
        if (k != exclude_j) x.P.incl[x.P.n_incl++] = k;
    }
    x.N = s->N;
    x.exclude = exclude_j;
    x.R = s->R;
    x.Rp = s->Rp;
    x.dE = s->dE;
    x.Tp = s->Tp;
    x.G64 = s->G64;
    x.Gplus64 = s->Gplus64;
    x.Gplus32 = s->Gplus32;
    x.rank = s->rank_dev;
    x.status = s->status;
    x.gwork = carve_smem_bytes(s->R, true) <= 200 * 1024 ? nullptr : s->work64;
    x.lam64 = s->lam64;
    x.V64 = s->V64;
    x.V32 = s->V32;
    x.V32lo = s->V32lo;
    x.etree = s->etree;
}

cudaError_t launch_prep_batch(const PrepItem* items_dev, int P, int n_incl, int Rmax, cudaStream_t st) {
    const bool in_smem = carve_smem_bytes(Rmax, true) <= 200 * 1024;
    const size_t smem = carve_smem_bytes(Rmax, in_smem);
    cudaFuncSetAttribute(prep_pinv_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(prep_eig_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prep_pinv_batch<<<P, 256, smem, st>>>(items_dev); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prep_eig_batch<<<P * n_incl, 256, smem, st>>>(items_dev, n_incl); count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int tpmax = (tri_size(Rmax) + 7) & ~7;
    prep_etree_batch<<<dim3((tpmax + ETREE_THREADS - 1) / ETREE_THREADS, P * n_incl), ETREE_THREADS, 0, st>>>(
        items_dev, n_incl);
    count_launch();
    return cudaGetLastError();
}

krp_status sampler_prep(krp_sampler* s, int exclude_j) {
    const int R = s->R, N = s->N;
    PrepParams P{};
    P.n_incl = 0;
    // a second refinement step takes the eigenvectors to FP64 rounding over
    // the eigenvalue gaps (one step leaves ~1e-8 where the gaps are ~1e-4 of
    // lambda_max, enough to move the eigencomponent stage's branch
    // probabilities by ~1e-4)
    P.extra_refine = 1;
    for (int k = 0; k < N; ++k) {
        P.roots[k] = s->root64[k];
        if (k != exclude_j) P.incl[P.n_incl++] = k;
    }
    const bool in_smem = carve_smem_bytes(R, true) <= 200 * 1024;
    const size_t smem = carve_smem_bytes(R, in_smem);
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(prep_pinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(prep_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    // one CTA per R x R problem: more threads hide the rotation steps'
    // shared-memory latency once R is past a warp's width
    const int nt = R > 32 ? 1024 : 256;
    prep_pinv<<<1, nt, smem, s->stream>>>(P, N, exclude_j, R, s->Tp, s->G64, s->Gplus64, s->Gplus32, s->rank_dev,
                                         s->status, in_smem ? nullptr : s->work64); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "prep_pinv launch");
    // R > 32 with the FP64 work in global memory: the refinement step over many CTAs
    const bool split = R > 32 && !in_smem;
    double* scales = s->work64 + (size_t)6 * R * R * (N + 1);   // the area's 256-double tail
    prep_eig<<<P.n_incl, nt, smem, s->stream>>>(P, N, R, s->Rp, s->dE, s->Tp, s->G64, s->Gplus64, s->lam64, s->V64,
                                               s->V32, s->V32lo, s->etree, in_smem ? nullptr : s->work64,
                                               split ? 1 : 0, scales); count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "prep_eig launch");
    if (split) {
        const int nt16 = (R + RG_TILE - 1) / RG_TILE;
        const dim3 g(nt16, nt16, P.n_incl);
        double* w = s->work64;
        refine_gemm<<<g, RG_TILE * RG_TILE, 0, s->stream>>>(w, R, 0, 4, 2, -1, 0, 0, 1.0);    // T = As X
        refine_gemm<<<g, RG_TILE * RG_TILE, 0, s->stream>>>(w, R, 4, 4, 3, -1, 1, 1, -1.0);   // Rm = I - XᵀX
        refine_gemm<<<g, RG_TILE * RG_TILE, 0, s->stream>>>(w, R, 4, 2, 1, -1, 1, 0, 1.0);    // S = Xᵀ T
        refine_mid<<<P.n_incl, 1024, 0, s->stream>>>(w, R);                                    // λ, δ, E
        refine_gemm<<<g, RG_TILE * RG_TILE, 0, s->stream>>>(w, R, 4, 2, 1, 4, 0, 0, 1.0);     // X + X E
        refine_finish<<<P.n_incl, 1024, 0, s->stream>>>(P, w, R, scales, s->lam64, s->V64, s->V32, s->V32lo);
        for (int q = 0; q < 6; ++q) count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(s, e, "prep refinement launch");
    }
    prep_etree<<<dim3((s->Tp + ETREE_THREADS - 1) / ETREE_THREADS, P.n_incl), ETREE_THREADS, 0, s->stream>>>(
        P, R, s->Rp, s->Tp, s->G64, s->lam64, s->V64, s->etree);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "prep_etree launch");
    s->last_exclude = exclude_j;
    return KRP_OK;
}

}  // namespace krp
