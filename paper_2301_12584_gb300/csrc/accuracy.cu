// Least-squares accuracy workload (Sec. 4.2): the distortion D(S, A) =
// kappa(SQ) - 1 of a leverage sketch without materialising A or a basis of its
// range, by the route of the appendix on computing sketch distortion:
// kappa(SQ) = kappa(SA V Σ⁻¹) where AᵀA = ⊛_k U_kᵀU_k = V Σ² Vᵀ, i.e. the
// square root of the ratio of the extreme eigenvalues of
// W = Σ⁻¹ Vᵀ (SAᵀSA) V Σ⁻¹ over the range of A; and black-box entries of a
// Kronecker right-hand side b = c_1 ⊗ ... ⊗ c_N at the sampled rows.
#include "common.cuh"
#include "internal.h"
#include "jacobi.cuh"

#include <math.h>

#include <algorithm>
#include <string>

namespace krp {

__global__ void __launch_bounds__(256) normal_partial(const float* __restrict__ SA, const float* __restrict__ w,
                                                      const float* __restrict__ B, int64_t J, int R, int nrhs,
                                                      int64_t rows_per_cta, float* __restrict__ part,
                                                      float* __restrict__ part_exp);

namespace {

struct KronParams {
    const float* c[16];
    int krow[16];
    int n;
};

__global__ void __launch_bounds__(256) kron_rows(const __grid_constant__ KronParams P, int64_t J,
                                                 const int32_t* __restrict__ idx, float* __restrict__ B) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < J; s += (int64_t)gridDim.x * blockDim.x) {
        float v = 1.f;
        for (int m = 0; m < P.n; ++m) v *= __ldg(P.c[m] + idx[(int64_t)P.krow[m] * J + s]);
        B[s] = v;
    }
}

// One CTA.  part: nparts partial sums of the packed SAᵀSA; G64: the factors'
// FP64 Grams (N x R x R); incl: the included factors.  work: 6 R² doubles.
__global__ void __launch_bounds__(256) distortion_finish(const float* __restrict__ part, int nparts, int R,
                                                         const double* __restrict__ G64, PrepParams P,
                                                         double* __restrict__ work, double* __restrict__ out) {
    __shared__ double cs[4 * 65];
    __shared__ int pr[2 * 65];
    __shared__ double red[16];
    __shared__ int keep[128];
    __shared__ int r_kept;
    const int RR = R * R, T = tri_size(R);
    double* M = work;        // SAᵀSA, full
    double* A = M + RR;      // ⊛ G_k, then its eigenvalues on the diagonal
    double* V = A + RR;      // eigenvectors of ⊛ G_k (columns)
    double* Z = V + RR;      // V Σ⁻¹ on the kept columns (R x r)
    double* W = Z + RR;      // Zᵀ M Z (r x r), then its eigenvalues
    double* Y = W + RR;      // M Z, then the eigenvectors of W
    for (int e = threadIdx.x; e < T; e += blockDim.x) {
        double a = 0.0;
        for (int p = 0; p < nparts; ++p)
            a += (double)part[(size_t)p * T + e] * ldexp(1.0, 2 * (int)part[(size_t)nparts * T + p]);
        int i = 0, rem = e;
        while (rem >= R - i) {
            rem -= R - i;
            ++i;
        }
        M[i * R + i + rem] = a;
        M[(i + rem) * R + i] = a;
    }
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
        double g = 1.0;
        for (int q = 0; q < P.n_incl; ++q) g *= G64[(size_t)P.incl[q] * RR + e];
        A[e] = g;
    }
    __syncthreads();
    jacobi_eig<double>(A, V, R, cs, pr, red, 40, 1e-15);
    __syncthreads();
    if (threadIdx.x == 0) {
        double lmax = 0.0;
        for (int u = 0; u < R; ++u) lmax = fmax(lmax, A[u * R + u]);
        int r = 0;
        for (int u = 0; u < R; ++u)
            if (A[u * R + u] > R * 2.220446049250313e-16 * lmax) keep[r++] = u;
        r_kept = r;
    }
    __syncthreads();
    const int r = r_kept;
    for (int e = threadIdx.x; e < R * r; e += blockDim.x) {
        const int i = e / r, u = keep[e % r];
        Z[e] = V[i * R + u] / sqrt(A[u * R + u]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * r; e += blockDim.x) {  // Y = M Z
        const int i = e / r, u = e % r;
        double a = 0.0;
        for (int k = 0; k < R; ++k) a += M[i * R + k] * Z[k * r + u];
        Y[e] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {  // W = Zᵀ Y
        const int u = e / r, v = e % r;
        double a = 0.0;
        for (int k = 0; k < R; ++k) a += Z[k * r + u] * Y[k * r + v];
        W[e] = a;
    }
    __syncthreads();
    if (r > 0) jacobi_eig<double>(W, Y, r, cs, pr, red, 40, 1e-15);
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0, mn = INFINITY;
        for (int u = 0; u < r; ++u) mx = fmax(mx, W[u * r + u]);
        for (int u = 0; u < r; ++u)
            if (W[u * r + u] > 0.0) mn = fmin(mn, W[u * r + u]);
        out[0] = (r > 0 && mx > 0.0 && mn < INFINITY) ? sqrt(mx / mn) - 1.0 : INFINITY;
        out[1] = (double)r;
    }
}

}  // namespace
}  // namespace krp

using namespace krp;

extern "C" krp_status krp_kron_rows(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx,
                                    const float* const* c_host, float* B_rows) {
    if (!s) return fail(nullptr, KRP_EINVAL, "krp_kron_rows: NULL sampler");
    if (J < 1 || !idx || !c_host || !B_rows || exclude_j < -1 || exclude_j >= s->N)
        return fail(s, KRP_EINVAL, "krp_kron_rows: bad arguments");
    KronParams P{};
    for (int k = 0; k < s->N; ++k) {
        if (k == exclude_j) continue;
        if (!c_host[k]) return fail(s, KRP_EINVAL, "krp_kron_rows: a vector of an included factor is NULL");
        P.c[P.n] = c_host[k];
        P.krow[P.n] = k;
        ++P.n;
    }
    const int64_t grid = std::min<int64_t>((J + 255) / 256, (int64_t)s->num_sms * 8);
    kron_rows<<<(unsigned)grid, 256, 0, s->stream>>>(P, J, idx, B_rows); count_launch();
    return cuda_check(s, cudaGetLastError(), "krp_kron_rows launch");
}

extern "C" krp_status krp_sketch_distortion(krp_sampler* s, int exclude_j, int64_t J, const float* SA,
                                            double* D_host, int* rank_host) {
    if (!s) return fail(nullptr, KRP_EINVAL, "krp_sketch_distortion: NULL sampler");
    if (J < 1 || J >= ((int64_t)1 << 31) || !SA || !D_host || exclude_j < -1 || exclude_j >= s->N)
        return fail(s, KRP_EINVAL, "krp_sketch_distortion: bad arguments");
    if (s->R > 128) return fail(s, KRP_EINVAL, "krp_sketch_distortion: R > 128");
    if (s->last_exclude == -2)
        return fail(s, KRP_ESTATE, "krp_sketch_distortion: sample (or prepare) since the last factor change first");
    const int R = s->R, T = tri_size(R);
    int nparts = (int)std::min<int64_t>((J + 255) / 256, (int64_t)s->num_sms * 2);
    nparts = nparts < 1 ? 1 : nparts;
    const size_t need = (size_t)nparts * T + nparts + 8 + (size_t)12 * R * R;  // partials, exponents, 6 R² doubles, out
    if (need > s->solve_scratch_floats) {
        if (s->solve_scratch) cudaFree(s->solve_scratch);
        s->solve_scratch = nullptr;
        s->solve_scratch_floats = 0;
        if (cudaMalloc(&s->solve_scratch, need * sizeof(float)) != cudaSuccess)
            return fail(s, KRP_ENOMEM, "krp_sketch_distortion: scratch allocation failed");
        s->solve_scratch_floats = need;
    }
    float* part = s->solve_scratch;
    size_t o = ((size_t)nparts * T + nparts + 1) & ~(size_t)1;  // 8-byte aligned double area
    double* work = reinterpret_cast<double*>(s->solve_scratch + o);
    double* out = work + (size_t)6 * R * R;
    const int64_t rows_per_cta = (J + nparts - 1) / nparts;
    const dim3 grid1(nparts, (T + 256 * 8 - 1) / (256 * 8));
    normal_partial<<<grid1, 256, (size_t)32 * R * 4, s->stream>>>(SA, nullptr, nullptr, J, R, 0, rows_per_cta, part,
                                                                  part + (size_t)nparts * T);
    count_launch();
    PrepParams P{};
    for (int k = 0; k < s->N; ++k)
        if (k != exclude_j) P.incl[P.n_incl++] = k;
    distortion_finish<<<1, 256, 0, s->stream>>>(part, nparts, R, s->G64, P, work, out); count_launch();
    cudaError_t e = cudaGetLastError();
    double h[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "krp_sketch_distortion");
    *D_host = h[0];
    if (rank_host) *rank_host = (int)h[1];
    return KRP_OK;
}
