// a8: sketched least-squares solve by the normal equations (Thm 2.1; the
// O(JR^2) solve of App. A.9):  M = SAᵀSA,  Z = SAᵀ SB with SB = diag(w) B,
// FP64 Cholesky M = L Lᵀ, X = M⁻¹ Z.  If Cholesky fails, optionally the FP64
// eigen-pseudo-inverse (cutoff R * 2^-52 * lam_max): X = M⁺ Z.
//
// normal_partial: grid-strided CTAs each reduce a contiguous chunk of rows
// into FP32 partial sums of the upper triangle of M and of Z (rows staged in
// shared memory, one output per thread slot).  Each chunk is first scaled by
// a power of two 2^-e (e from its largest entry, stored in part_exp) so that
// the FP32 sums neither overflow nor underflow when the weights
// 1/sqrt(J q) are far from 1 (many factors: q ~ 2^-144 at N = 9, I = 2^16).
// normal_solve (one CTA): FP64 sum of the partials times 2^(2e) in a fixed
// order, Cholesky, triangular solves.  A single problem's sum runs first, in
// the same order, over many CTAs (normal_reduce; GB300's FP64 rate is ~1/64 of
// FP32 per SM), and normal_solve_sums starts from it.
#include "common.cuh"
#include "internal.h"
#include "jacobi.cuh"

#include <math.h>

#include <algorithm>

namespace krp {

constexpr int SOLVE_ROWS = 32;  // rows per shared-memory tile

// Z columns: B_rows (J x nrhs) weighted by w; with B_rows == nullptr Z is not formed.
// CTA (px, py): rows [px rows_per_cta, (px+1) rows_per_cta), outputs chunk py.
__device__ __forceinline__ void normal_partial_body(const float* __restrict__ SA, const float* __restrict__ w,
                                                    const float* __restrict__ B, int64_t J, int R, int nrhs,
                                                    int64_t rows_per_cta, float* __restrict__ part,
                                                    float* __restrict__ part_exp, int px, int py) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float s_max[32];
    float* sA = sm;                          // SOLVE_ROWS x R
    float* sB = sA + SOLVE_ROWS * R;         // SOLVE_ROWS x nrhs
    const int T = tri_size(R);
    const int nout = T + R * nrhs;
    constexpr int MAXO = 8;                  // outputs per thread; py selects the output chunk
    float acc[MAXO];
    int oi[MAXO], oj[MAXO];
#pragma unroll
    for (int o = 0; o < MAXO; ++o) {
        acc[o] = 0.f;
        const int id = (py * MAXO + o) * blockDim.x + threadIdx.x;
        oi[o] = -1;
        oj[o] = 0;
        if (id < T) {
            int i = 0, rem = id;
            while (rem >= R - i) {
                rem -= R - i;
                ++i;
            }
            oi[o] = i;
            oj[o] = i + rem;
        } else if (id < nout) {
            oi[o] = (id - T) / nrhs;
            oj[o] = -1 - (id - T) % nrhs;  // negative: a column of Z
        }
    }
    const int64_t r0 = (int64_t)px * rows_per_cta;
    const int64_t r1 = min(J, r0 + rows_per_cta);
    // the chunk's scale 2^-ex from its largest |SA| and |w B| entry
    float mx = 0.f;
    for (int64_t e = threadIdx.x; e < (r1 - r0) * R; e += blockDim.x) mx = fmaxf(mx, fabsf(SA[r0 * R + e]));
    if (B)
        for (int64_t e = threadIdx.x; e < (r1 - r0) * nrhs; e += blockDim.x)
            mx = fmaxf(mx, fabsf(w[r0 + e / nrhs] * B[r0 * nrhs + e]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmaxf(m, s_max[q]);
        s_max[0] = m;
    }
    __syncthreads();
    const int ex = (s_max[0] > 0.f && isfinite(s_max[0])) ? ilogbf(s_max[0]) : 0;
    const float sc = ldexpf(1.f, -ex);  // exact power of two (-126 <= ex <= 127)
    if (part_exp && py == 0 && threadIdx.x == 0) part_exp[px] = (float)ex;
    for (int64_t base = r0; base < r1; base += SOLVE_ROWS) {
        const int nr = (int)min((int64_t)SOLVE_ROWS, r1 - base);
        __syncthreads();
        for (int e = threadIdx.x; e < SOLVE_ROWS * R; e += blockDim.x)
            sA[e] = (e / R < nr) ? SA[(base + e / R) * R + e % R] * sc : 0.f;
        if (B)
            for (int e = threadIdx.x; e < SOLVE_ROWS * nrhs; e += blockDim.x) {
                const int r = e / nrhs;
                sB[e] = (r < nr) ? (w[base + r] * B[(base + r) * nrhs + e % nrhs]) * sc : 0.f;
            }
        __syncthreads();
#pragma unroll
        for (int o = 0; o < MAXO; ++o) {
            if (oi[o] < 0) continue;
            const int i = oi[o], j = oj[o];
            float a = acc[o];
            if (j >= 0) {
                for (int r = 0; r < nr; ++r) a = fmaf(sA[r * R + i], sA[r * R + j], a);
            } else {
                const int c = -1 - j;
                for (int r = 0; r < nr; ++r) a = fmaf(sA[r * R + i], sB[r * nrhs + c], a);
            }
            acc[o] = a;
        }
    }
#pragma unroll
    for (int o = 0; o < MAXO; ++o) {
        const int id = (py * MAXO + o) * blockDim.x + threadIdx.x;
        if (id < nout) part[(size_t)px * nout + id] = acc[o];
    }
}

// part_exp: one float per partial (the chunk's exponent), e.g. right after the
// nparts x nout partials.
__global__ void __launch_bounds__(256) normal_partial(const float* __restrict__ SA, const float* __restrict__ w,
                                                      const float* __restrict__ B, int64_t J, int R, int nrhs,
                                                      int64_t rows_per_cta, float* __restrict__ part,
                                                      float* __restrict__ part_exp) {
    normal_partial_body(SA, w, B, J, R, nrhs, rows_per_cta, part, part_exp, blockIdx.x, blockIdx.y);
}

// One CTA.  mode 0: X = M⁻¹ Z (R x nrhs) written as FP32 to X;
// mode 1: M⁻¹ (R x R) written as FP64 to Xd (sparse path).
// Work matrices: shared memory when gbuf == nullptr, else gbuf (global).
// split (mode 1 only): after a successful Cholesky, leave L in gL and a 1 in
// *gflag for normal_trsm (the R triangular solves for the columns of M⁻¹ then
// run on R SMs instead of one); otherwise *gflag = 0 and this CTA finishes.
__device__ __forceinline__ void normal_solve_body(const float* __restrict__ part, int nparts, int R, int nrhs,
                                                  int mode, int flags, float* __restrict__ X,
                                                  double* __restrict__ Xd, int* __restrict__ status,
                                                  double* __restrict__ gbuf, const float* __restrict__ part_exp,
                                                  const double* __restrict__ sums = nullptr,
                                                  double* __restrict__ gL = nullptr,
                                                  double* __restrict__ gflag = nullptr) {
    extern __shared__ __align__(16) double smd[];
    const int RR = R * R;
    const int T = tri_size(R);
    const int ncol = mode == 1 ? R : nrhs;
    const int nout = T + R * nrhs;
    double* red = smd;
    double* cs = red + 64;
    int* pr = (int*)(cs + 2 * (R / 2 + 1));
    double* M = gbuf ? gbuf : (double*)(pr + 2 * (R / 2 + 1) + 2);  // R x R
    double* Lm = M + RR;                                            // R x R
    double* Z = Lm + RR;                                            // R x ncol
    __shared__ int flag;
    __shared__ double pscale[1024];  // 2^(2 e_p) of the first 1024 partials
    if (threadIdx.x == 0) flag = 0;
    for (int p = threadIdx.x; p < nparts && p < 1024; p += blockDim.x)
        pscale[p] = part_exp ? ldexp(1.0, 2 * (int)part_exp[p]) : 1.0;
    __syncthreads();
    auto psc = [&](int p) -> double {
        return p < 1024 ? pscale[p] : (part_exp ? ldexp(1.0, 2 * (int)part_exp[p]) : 1.0);
    };
    // FP64 reduction of the partials, fixed order (or their sums from normal_reduce)
    for (int id = threadIdx.x; id < T; id += blockDim.x) {
        double a = 0.0;
        if (sums)
            a = sums[id];
        else
            for (int p = 0; p < nparts; ++p) a += (double)part[(size_t)p * nout + id] * psc(p);
        int i = 0, rem = id;
        while (rem >= R - i) {
            rem -= R - i;
            ++i;
        }
        M[i * R + i + rem] = a;
        M[(i + rem) * R + i] = a;
    }
    for (int id = threadIdx.x; id < R * ncol; id += blockDim.x) {
        double a;
        if (mode == 1) {
            a = (id / ncol == id % ncol) ? 1.0 : 0.0;
        } else if (sums) {
            a = sums[T + id];
        } else {
            a = 0.0;
            for (int p = 0; p < nparts; ++p) a += (double)part[(size_t)p * nout + T + id] * psc(p);
        }
        Z[id] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < RR; e += blockDim.x) Lm[e] = M[e];
    __syncthreads();
    for (int c = 0; c < R; ++c) {
        if (threadIdx.x == 0) {
            const double d = Lm[c * R + c];
            if (!(d > 0.0)) flag = 1;
            Lm[c * R + c] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double dc = Lm[c * R + c];
        for (int i = c + 1 + threadIdx.x; i < R; i += blockDim.x) Lm[i * R + c] /= dc;
        __syncthreads();
        const int n = R - c - 1;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = c + 1 + e / n, j = c + 1 + e % n;
            if (j <= i) Lm[i * R + j] -= Lm[i * R + c] * Lm[j * R + c];
        }
        __syncthreads();
    }
    if (!flag && gL) {
        if (gL != Lm)
            for (int e = threadIdx.x; e < RR; e += blockDim.x) gL[e] = Lm[e];
        if (threadIdx.x == 0) *gflag = 1.0;
        return;
    }
    if (!flag) {
        // forward then backward substitution, one thread per right-hand side
        for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
            for (int i = 0; i < R; ++i) {
                double a = Z[i * ncol + col];
                for (int k = 0; k < i; ++k) a -= Lm[i * R + k] * Z[k * ncol + col];
                Z[i * ncol + col] = a / Lm[i * R + i];
            }
            for (int i = R - 1; i >= 0; --i) {
                double a = Z[i * ncol + col];
                for (int k = i + 1; k < R; ++k) a -= Lm[k * R + i] * Z[k * ncol + col];
                Z[i * ncol + col] = a / Lm[i * R + i];
            }
        }
        __syncthreads();
    } else if (flags & KRP_PINV_FALLBACK) {
        // M⁺ Z by the FP64 eigendecomposition of M (Lm becomes eigenvectors)
        __syncthreads();
        double* A = M;  // overwritten by Jacobi; diagonal = eigenvalues
        jacobi_eig<double>(A, Lm, R, cs, pr, red, 30, 1e-14);
        __shared__ double lam_max;
        if (threadIdx.x == 0) {
            double mx = 0.0;
            for (int i = 0; i < R; ++i) mx = fmax(mx, A[i * R + i]);
            lam_max = mx;
        }
        __syncthreads();
        const double cut = R * 2.220446049250313e-16 * lam_max;
        // Y = Vᵀ Z scaled by 1/λ, then X = V Y; one thread per column
        for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
            double y[128];
            for (int u = 0; u < R; ++u) {
                double a = 0.0;
                const double l = A[u * R + u];
                if (l > cut)
                    for (int i = 0; i < R; ++i) a += Lm[i * R + u] * Z[i * ncol + col];
                y[u] = l > cut ? a / l : 0.0;
            }
            for (int i = 0; i < R; ++i) {
                double a = 0.0;
                for (int u = 0; u < R; ++u) a += Lm[i * R + u] * y[u];
                Z[i * ncol + col] = a;
            }
        }
        __syncthreads();
    } else {
        for (int e = threadIdx.x; e < R * ncol; e += blockDim.x) Z[e] = 0.0;
        if (threadIdx.x == 0) set_status(status, KRP_ESINGULAR);
        __syncthreads();
    }
    for (int e = threadIdx.x; e < R * ncol; e += blockDim.x) {
        if (mode == 1)
            Xd[e] = Z[e];
        else
            X[e] = (float)Z[e];
    }
    if (gflag && threadIdx.x == 0) *gflag = 0.0;   // done here: normal_trsm has nothing to do
}

__global__ void __launch_bounds__(256) normal_solve(const float* __restrict__ part, int nparts, int R, int nrhs,
                                                    int mode, int flags, float* __restrict__ X,
                                                    double* __restrict__ Xd, int* __restrict__ status,
                                                    double* __restrict__ gbuf, const float* __restrict__ part_exp) {
    normal_solve_body(part, nparts, R, nrhs, mode, flags, X, Xd, status, gbuf, part_exp);
}

// The FP64 reduction of normal_solve spread over CTAs: at R = 100 and 304
// partials it is 1.5 M FP64 adds, too many for the one SM the solve runs on.
// A CTA takes 32 output entries (one per lane); warp w sums partials w, w + 8,
// ... in order, then the 8 warps' sums are added in warp order.
__global__ void __launch_bounds__(256) normal_reduce(const float* __restrict__ part,
                                                     const float* __restrict__ part_exp, int nparts, int nout,
                                                     double* __restrict__ sums) {
    __shared__ double ws[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int id = blockIdx.x * 32 + lane;
    double a = 0.0;
    if (id < nout)
        for (int p = warp; p < nparts; p += 8) a += (double)part[(size_t)p * nout + id] * ldexp(1.0, 2 * (int)part_exp[p]);
    ws[warp][lane] = a;
    __syncthreads();
    if (warp == 0 && id < nout) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += ws[w][lane];
        sums[id] = t;
    }
}

__global__ void __launch_bounds__(256) normal_solve_sums(const double* __restrict__ sums, int R, int nrhs, int mode,
                                                         int flags, float* __restrict__ X, double* __restrict__ Xd,
                                                         int* __restrict__ status, double* __restrict__ gbuf,
                                                         double* __restrict__ gL, double* __restrict__ gflag) {
    normal_solve_body(nullptr, 0, R, nrhs, mode, flags, X, Xd, status, gbuf, nullptr, sums, gL, gflag);
}

// Column c of M⁻¹ = L⁻ᵀ L⁻¹ e_c by forward and backward substitution, one
// warp per column (CTA c), each inner product summed over the lanes in a
// fixed order; nothing to do unless normal_solve_sums left *gflag = 1.
__global__ void __launch_bounds__(32) normal_trsm(const double* __restrict__ L, int R,
                                                  const double* __restrict__ gflag, double* __restrict__ Xd) {
    __shared__ double z[128];
    if (*gflag != 1.0) return;
    const int col = blockIdx.x, lane = threadIdx.x;
    for (int i = lane; i < R; i += 32) z[i] = 0.0;
    __syncwarp();
    for (int i = col; i < R; ++i) {   // L z = e_col (z_i = 0 for i < col)
        double a = 0.0;
        for (int k = col + lane; k < i; k += 32) a += L[(size_t)i * R + k] * z[k];
        a = warp_sum_d(a);
        if (lane == 0) z[i] = ((i == col ? 1.0 : 0.0) - a) / L[(size_t)i * R + i];
        __syncwarp();
    }
    for (int i = R - 1; i >= 0; --i) {   // Lᵀ x = z
        double a = 0.0;
        for (int k = i + 1 + lane; k < R; k += 32) a += L[(size_t)k * R + i] * z[k];
        a = warp_sum_d(a);
        if (lane == 0) z[i] = (z[i] - a) / L[(size_t)i * R + i];
        __syncwarp();
    }
    for (int i = lane; i < R; i += 32) Xd[(size_t)i * R + col] = z[i];
}

// Batched forms: blockIdx.z (partials) or blockIdx.x (solve) is the problem.
__global__ void __launch_bounds__(256) normal_partial_batch(const SolveItem* __restrict__ items, int64_t J,
                                                            const float* __restrict__ SA,
                                                            const float* __restrict__ w,
                                                            const float* __restrict__ B, int nrhs) {
    const SolveItem& it = items[blockIdx.z];
    const int nout = tri_size(it.R) + it.R * nrhs;
    if ((int)blockIdx.x >= it.nparts || (int)blockIdx.y * 8 * (int)blockDim.x >= nout) return;  // CTA-uniform
    const int64_t rows_per_cta = (J + it.nparts - 1) / it.nparts;
    normal_partial_body(SA + J * it.row_off, w + (int64_t)blockIdx.z * J,
                        B ? B + (int64_t)blockIdx.z * J * nrhs : nullptr, J, it.R, nrhs, rows_per_cta, it.part,
                        it.part + (size_t)it.nparts * nout, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(256) normal_solve_batch(const SolveItem* __restrict__ items, int nrhs, int flags,
                                                          float* __restrict__ X, int* __restrict__ status) {
    const SolveItem& it = items[blockIdx.x];
    const int nout = tri_size(it.R) + it.R * nrhs;
    normal_solve_body(it.part, it.nparts, it.R, nrhs, 0, flags, X + it.x_off * nrhs, nullptr, status, nullptr,
                      it.part + (size_t)it.nparts * nout);
}

cudaError_t launch_solve_batch(const SolveItem* items_dev, int P, int max_parts, int Rmax, int64_t J,
                               const float* SA, const float* weight, const float* B, int nrhs, int flags, float* X,
                               int* status, cudaStream_t st) {
    const int nout = tri_size(Rmax) + Rmax * nrhs;
    const dim3 grid1(max_parts, (nout + 256 * 8 - 1) / (256 * 8), P);
    const size_t smem1 = (size_t)SOLVE_ROWS * (Rmax + nrhs) * 4;
    normal_partial_batch<<<grid1, 256, smem1, st>>>(items_dev, J, SA, weight, B, nrhs); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t small = 64 * 8 + 2 * (Rmax / 2 + 1) * 8 + 2 * (Rmax / 2 + 1) * 4 + 16;
    const size_t smem2 = small + (size_t)(2 * Rmax * Rmax + Rmax * nrhs) * 8;
    if (smem2 > 48 * 1024) {
        e = cudaFuncSetAttribute(normal_solve_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        if (e != cudaSuccess) return e;
    }
    normal_solve_batch<<<P, 256, smem2, st>>>(items_dev, nrhs, flags, X, status); count_launch();
    return cudaGetLastError();
}

namespace {
krp_status normal_common(krp_sampler* s, int64_t J, const float* SA, const float* weight, const float* B,
                         int nrhs, int mode, int flags, float* X) {
    const int R = s->R;
    const int T = tri_size(R);
    const int nout = T + R * nrhs;
    int nparts = (int)std::min<int64_t>((J + 255) / 256, (int64_t)s->num_sms * 2);
    nparts = nparts < 1 ? 1 : nparts;
    const int64_t rows_per_cta = (J + nparts - 1) / nparts;
    const int ncol = mode == 1 ? R : nrhs;
    // partials, their exponents, then (8-byte aligned) the FP64 sums
    const size_t sums_off = ((size_t)nparts * nout + nparts + 1) & ~(size_t)1;
    const size_t need = sums_off + (size_t)2 * nout;
    const size_t need64 = (size_t)2 * R * R + (size_t)R * ncol + (size_t)R * R;
    if (need > s->solve_scratch_floats) {
        if (s->solve_scratch) cudaFree(s->solve_scratch);
        s->solve_scratch = nullptr;
        s->solve_scratch_floats = 0;
        if (cudaMalloc(&s->solve_scratch, need * sizeof(float)) != cudaSuccess)
            return fail(s, KRP_ENOMEM, "solve scratch allocation failed");
        s->solve_scratch_floats = need;
    }
    const size_t smem1 = (size_t)SOLVE_ROWS * (R + nrhs) * 4;
    const dim3 grid1(nparts, (nout + 256 * 8 - 1) / (256 * 8));
    float* part_exp = s->solve_scratch + (size_t)nparts * nout;
    normal_partial<<<grid1, 256, smem1, s->stream>>>(SA, weight, B, J, R, nrhs, rows_per_cta, s->solve_scratch,
                                                     part_exp); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "normal_partial launch");
    const size_t small = 64 * 8 + 2 * (R / 2 + 1) * 8 + 2 * (R / 2 + 1) * 4 + 16;
    const size_t mats = (size_t)(2 * R * R + R * ncol) * 8;
    const bool in_smem = small + mats <= 160 * 1024;
    const size_t smem2 = small + (in_smem ? mats : 0);
    if (smem2 > 48 * 1024)
        cudaFuncSetAttribute(normal_solve_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    double* sums = reinterpret_cast<double*>(s->solve_scratch + sums_off);
    normal_reduce<<<(nout + 31) / 32, 256, 0, s->stream>>>(s->solve_scratch, part_exp, nparts, nout, sums);
    count_launch();
    // M⁻¹ for the sparse solve at larger R: its R triangular solves over R CTAs
    const bool split = mode == 1 && R >= 48;
    double* Xd = s->solve64 + (size_t)(2 * R * R + R * 128);
    double* gL = split ? s->solve64 + (size_t)R * R : nullptr;
    double* gflag = split ? s->solve64 + (size_t)2 * R * R : nullptr;
    normal_solve_sums<<<1, 256, smem2, s->stream>>>(sums, R, nrhs, mode, flags, X, Xd, s->status,
                                                    in_smem ? nullptr : s->solve64, gL, gflag); count_launch();
    if (split) {
        normal_trsm<<<R, 32, 0, s->stream>>>(gL, R, gflag, Xd);
        count_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "normal_solve launch");
    (void)need64;
    return KRP_OK;
}
}  // namespace

krp_status dense_solve(krp_sampler* s, int64_t J, const float* SA, const float* weight, const float* B_rows,
                       int nrhs, float* X, int flags) {
    return normal_common(s, J, SA, weight, B_rows, nrhs, 0, flags, X);
}

krp_status normal_inverse(krp_sampler* s, int64_t J, const float* SA, int flags) {
    return normal_common(s, J, SA, nullptr, nullptr, 0, 1, flags, nullptr);
}

}  // namespace krp
