// a2 + a3: per-draw sampler preparation (Alg. 2 lines 1-5; Eq. G_geq_k_defn;
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

struct PrepParams {
    const double* roots[16];  // FP64 root Gram G_k of each factor (packed upper)
    int incl[16];            // included factors, ascending
    int n_incl;
};

// ---------------------------------------------------------------------------
// prep_pinv: G, G⁺, rank.  The three R x R FP64 work matrices live in shared
// memory when they fit (R <= 64), else in the global buffer gbuf.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) prep_pinv(PrepParams P, int N, int exclude, int R, int Tp,
                                                 double* __restrict__ G64, double* __restrict__ Gplus64,
                                                 float* __restrict__ Gplus32, int* __restrict__ rank_out,
                                                 int* __restrict__ status, double* __restrict__ gbuf) {
    extern __shared__ __align__(16) double sm[];
    const int RR = R * R;
    double* red = sm;                        // 64
    double* cs = red + 64;                   // 2*(R/2+1)
    int* pr = (int*)(cs + 2 * (R / 2 + 1));  // 2*(R/2+1)
    double* G = gbuf ? gbuf : (double*)(pr + 2 * (R / 2 + 1) + 2);  // R x R
    double* W = G + RR;                      // R x R  (Cholesky factor / eigenvectors)
    double* Ginv = W + RR;                   // R x R
    __shared__ int flag;
    __shared__ double s_norm, s_inorm;
    // G_k in FP64 (full symmetric) for every factor; G = Hadamard of included
    for (int e = threadIdx.x; e < RR; e += blockDim.x) G[e] = 1.0;
    for (int k = 0; k < N; ++k) {
        const double* rt = P.roots[k];
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            const int i = e / R, j = e % R;
            const double v = rt ? rt[tri_index(min(i, j), max(i, j), R)] : 0.0;
            G64[(size_t)k * RR + e] = v;
            if (k != exclude) G[e] *= v;
        }
    }
    if (threadIdx.x == 0) flag = 0;
    __syncthreads();
    // Cholesky G = L Lᵀ (right-looking, column by column), L in W (lower).
    for (int e = threadIdx.x; e < RR; e += blockDim.x) W[e] = G[e];
    __syncthreads();
    for (int c = 0; c < R; ++c) {
        if (threadIdx.x == 0) {
            const double d = W[c * R + c];
            if (!(d > 0.0)) flag = 1;
            W[c * R + c] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double dc = W[c * R + c];
        for (int i = c + 1 + threadIdx.x; i < R; i += blockDim.x) W[i * R + c] /= dc;
        __syncthreads();
        for (int e = threadIdx.x; e < (R - c - 1) * (R - c - 1); e += blockDim.x) {
            const int i = c + 1 + e / (R - c - 1), j = c + 1 + e % (R - c - 1);
            if (j <= i) W[i * R + j] -= W[i * R + c] * W[j * R + c];
        }
        __syncthreads();
    }
    if (!flag) {
        // L⁻¹ column by column (forward substitution), into Ginv (lower).
        for (int col = threadIdx.x; col < R; col += blockDim.x) {
            for (int i = 0; i < R; ++i) {
                double acc = (i == col) ? 1.0 : 0.0;
                for (int k = col; k < i; ++k) acc -= W[i * R + k] * Ginv[k * R + col];
                Ginv[i * R + col] = (i >= col) ? acc / W[i * R + i] : 0.0;
            }
        }
        __syncthreads();
        // G⁻¹ = L⁻ᵀ L⁻¹ ; reuse W as output
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            const int i = e / R, j = e % R;
            double acc = 0.0;
            for (int k = max(i, j); k < R; ++k) acc += Ginv[k * R + i] * Ginv[k * R + j];
            W[e] = acc;
        }
        __syncthreads();
        // exact 1-norm condition number ||G||_1 ||G⁻¹||_1
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int j = 0; j < R; ++j) {
                double ca = 0.0, cb = 0.0;
                for (int i = 0; i < R; ++i) {
                    ca += fabs(G[i * R + j]);
                    cb += fabs(W[i * R + j]);
                }
                a = fmax(a, ca);
                b = fmax(b, cb);
            }
            s_norm = a;
            s_inorm = b;
            if (!(a * b <= 1e10)) flag = 1;
        }
        __syncthreads();
    }
    int rank = R;
    if (!flag) {
        for (int e = threadIdx.x; e < RR; e += blockDim.x) Gplus64[e] = W[e];
    } else {
        // eigen-pseudo-inverse in FP64
        for (int e = threadIdx.x; e < RR; e += blockDim.x) Ginv[e] = G[e];
        __syncthreads();
        jacobi_eig<double>(Ginv, W, R, cs, pr, red, 30, 1e-14);
        __shared__ double lam_max;
        if (threadIdx.x == 0) {
            double mx = 0.0;
            for (int i = 0; i < R; ++i) mx = fmax(mx, Ginv[i * R + i]);
            lam_max = mx;
        }
        __syncthreads();
        const double cut = R * 2.220446049250313e-16 * lam_max;
        rank = 0;
        for (int i = 0; i < R; ++i) rank += Ginv[i * R + i] > cut;
        for (int e = threadIdx.x; e < RR; e += blockDim.x) {
            const int i = e / R, j = e % R;
            double acc = 0.0;
            for (int u = 0; u < R; ++u) {
                const double l = Ginv[u * R + u];
                if (l > cut) acc += W[i * R + u] * W[j * R + u] / l;
            }
            Gplus64[e] = acc;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        float v = 0.f;
        if (e < tri_size(R)) {
            // row i, column j of packed entry e
            int i = 0, rem = e;
            while (rem >= R - i) {
                rem -= R - i;
                ++i;
            }
            const int j = i + rem;
            v = (float)Gplus64[i * R + j];
        }
        Gplus32[e] = v;
    }
    if (threadIdx.x == 0) {
        *rank_out = rank;
        if (rank == 0) set_status(status, KRP_EZERO);
    }
}

// ---------------------------------------------------------------------------
// prep_eig: one CTA per included factor.
// ---------------------------------------------------------------------------
template <typename Scalar>
__global__ void __launch_bounds__(256) prep_eig(PrepParams P, int N, int R, int Rp,
                                                int dE, int Tp, const double* __restrict__ G64,
                                                const double* __restrict__ Gplus64, double* __restrict__ lam64,
                                                double* __restrict__ V64, float* __restrict__ V32,
                                                float* __restrict__ V32lo, float* __restrict__ etree) {
    extern __shared__ __align__(16) double sm[];
    const int RR = R * R;
    const int p = blockIdx.x;
    const int n_incl = P.n_incl;
    const int k = P.incl[p];
    Scalar* A = (Scalar*)sm;            // R x R
    Scalar* V = A + RR;                 // R x R  (2 R*R Scalars: 8-byte aligned end)
    double* lam = (double*)(V + RR);
    int* pos = (int*)(lam + R);
    double* red = (double*)(pos + R + (R & 1));
    Scalar* cs = (Scalar*)(red + 64);
    int* pr = (int*)(cs + 2 * (R / 2 + 1));
    // G_{>k} = G⁺ ⊛ ⊛_{m>k, m included} G_m
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        double v = Gplus64[e];
        for (int q = p + 1; q < n_incl; ++q) v *= G64[(size_t)P.incl[q] * RR + e];
        A[e] = (Scalar)v;
    }
    __syncthreads();
    jacobi_eig<Scalar>(A, V, R, cs, pr, red, 30, sizeof(Scalar) == 8 ? 1e-14 : 1e-6);
    for (int i = threadIdx.x; i < R; i += blockDim.x) lam[i] = fmax((double)A[i * R + i], 0.0);
    __syncthreads();
    ascending_positions(lam, R, pos);
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        const int row = e / R, u = e % R;   // V[row][u], eigenvector u in column u
        const int o = pos[u];
        V64[(size_t)k * RR + row * R + o] = (double)V[e];
        const double v = (double)V[e];
        const float vh = (float)v;
        V32[(size_t)k * RR + o * R + row] = vh;   // row o = eigenvector
        V32lo[(size_t)k * RR + o * R + row] = (float)(v - (double)vh);
    }
    for (int u = threadIdx.x; u < R; u += blockDim.x) lam64[(size_t)k * R + pos[u]] = lam[u];
    __syncthreads();
    // E_k: per packed entry e=(i,j), leaves u = 0..Rp-1 hold λ_u V[i,u] V[j,u]
    // (zero for u >= R); binary-counter pairwise sums up the tree; stored
    // nodes multiplied by G_k[i,j].  Reads the sorted eigenpairs from global.
    const double* lk = lam64 + (size_t)k * R;
    const double* Vk = V64 + (size_t)k * RR;
    const double* Gk = G64 + (size_t)k * RR;
    float* et = etree + (size_t)k * Rp * Tp;
    const int T = tri_size(R);
    for (int e = threadIdx.x; e < Tp; e += blockDim.x) {
        if (e >= T) {
            for (int sl = 0; sl < Rp; ++sl) et[(size_t)sl * Tp + e] = 0.f;
            continue;
        }
        int i = 0, rem = e;
        while (rem >= R - i) {
            rem -= R - i;
            ++i;
        }
        const int j = i + rem;
        const double gij = Gk[i * R + j];
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
}

krp_status sampler_prep(krp_sampler* s, int exclude_j) {
    const int R = s->R, N = s->N;
    PrepParams P{};
    P.n_incl = 0;
    for (int k = 0; k < N; ++k) {
        P.roots[k] = s->root64[k];
        if (k != exclude_j) P.incl[P.n_incl++] = k;
    }
    const size_t mats = (size_t)3 * R * R * 8;
    const size_t small = 64 * 8 + 2 * (R / 2 + 1) * 8 + 2 * (R / 2 + 1) * 4 + 16;
    const bool pinv_smem = mats + small <= 200 * 1024;
    const size_t sm1 = small + (pinv_smem ? mats : 0);
    if (sm1 > 48 * 1024) cudaFuncSetAttribute(prep_pinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    prep_pinv<<<1, 256, sm1, s->stream>>>(P, N, exclude_j, R, s->Tp, s->G64, s->Gplus64, s->Gplus32,
                                          s->rank_dev, s->status, pinv_smem ? nullptr : s->work64); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "prep_pinv launch");
    // Eigendecompositions of G_{>k}: FP64 Jacobi while the two R x R FP64
    // matrices fit in shared memory (R <= 64), FP32 Jacobi above that.
    const bool fp64 = (size_t)2 * R * R * 8 <= 96 * 1024;
    const size_t sc = fp64 ? 8 : 4;
    const size_t sm2 = 2 * (size_t)R * R * sc + (size_t)R * 8 + (size_t)(R + 2) * 4 + 64 * 8 +
                       2 * (R / 2 + 1) * sc + 2 * (R / 2 + 1) * 4 + 64;
    if (fp64) {
        if (sm2 > 48 * 1024)
            cudaFuncSetAttribute(prep_eig<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        prep_eig<double><<<P.n_incl, 256, sm2, s->stream>>>(P, N, R, s->Rp, s->dE, s->Tp, s->G64, s->Gplus64,
                                                           s->lam64, s->V64, s->V32, s->V32lo, s->etree); count_launch();
    } else {
        if (sm2 > 48 * 1024)
            cudaFuncSetAttribute(prep_eig<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        prep_eig<float><<<P.n_incl, 256, sm2, s->stream>>>(P, N, R, s->Rp, s->dE, s->Tp, s->G64, s->Gplus64,
                                                          s->lam64, s->V64, s->V32, s->V32lo, s->etree); count_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "prep_eig launch");
    s->last_exclude = exclude_j;
    return KRP_OK;
}

}  // namespace krp
