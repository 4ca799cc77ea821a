// C ABI of libkrpls: argument checks, storage, and the order of kernel
// launches for each call (declarations and contracts in include/krpls.h).
#include "common.cuh"
#include "internal.h"

#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>

namespace krp {

thread_local std::string g_error = "no error";
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_counter() { return g_launches.load(std::memory_order_relaxed); }

krp_status fail(krp_sampler* s, krp_status code, const std::string& msg) {
    if (s)
        s->last_error = msg;
    else
        g_error = msg;
    return code;
}

krp_status cuda_check(krp_sampler* s, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return KRP_OK;
    return fail(s, e == cudaErrorMemoryAllocation ? KRP_ENOMEM : KRP_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

krp_status als_buffers(krp_sampler* s, int64_t J, int32_t** idx, float** w, float** SA, double** sumsq);

}  // namespace krp

using namespace krp;

namespace {

template <typename T>
bool dalloc(T** p, size_t n) {
    *p = nullptr;
    return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

int log2i(int64_t p) {
    int d = 0;
    while (((int64_t)1 << d) < p) ++d;
    return d;
}

}  // namespace

namespace krp {
krp_status als_buffers(krp_sampler* s, int64_t J, int32_t** idx, float** w, float** SA, double** sumsq) {
    if (!s->als_sumsq && !dalloc(&s->als_sumsq, 2 * 128 + 8)) return fail(s, KRP_ENOMEM, "ALS scratch allocation failed");
    // per-CTA partials: 2 CTAs per SM x 128 columns (Y M⁻¹), 8 CTAs per SM (fit)
    if (!s->als_part && !dalloc(&s->als_part, (size_t)s->num_sms * 2 * 128 + (size_t)s->num_sms * 8))
        return fail(s, KRP_ENOMEM, "ALS scratch allocation failed");
    if (J > s->als_J) {
        cudaFree(s->als_idx);
        cudaFree(s->als_w);
        cudaFree(s->als_SA);
        s->als_J = 0;
        if (!dalloc(&s->als_idx, (size_t)s->N * J) || !dalloc(&s->als_w, (size_t)J) ||
            !dalloc(&s->als_SA, (size_t)J * s->R))
            return fail(s, KRP_ENOMEM, "ALS sample buffers allocation failed");
        s->als_J = J;
    }
    *idx = s->als_idx;
    *w = s->als_w;
    *SA = s->als_SA;
    *sumsq = s->als_sumsq;
    return KRP_OK;
}
}  // namespace krp

extern "C" {

void krp_destroy(krp_sampler* s) {
    if (!s) return;
    if (s->capturing) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s->stream, &g);
        if (g) cudaGraphDestroy(g);
    }
    cudaStreamSynchronize(s->stream);
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    for (float* p : s->U) cudaFree(p);
    for (float* p : s->tree) cudaFree(p);
    for (float* p : s->tree_lo) cudaFree(p);
    for (float* p : s->dtop) cudaFree(p);
    for (double* p : s->root64) cudaFree(p);
    cudaFree(s->G64);
    cudaFree(s->Gplus64);
    cudaFree(s->lam64);
    cudaFree(s->V64);
    cudaFree(s->work64);
    cudaFree(s->Gplus32);
    cudaFree(s->etree);
    cudaFree(s->V32);
    cudaFree(s->V32lo);
    cudaFree(s->rank_dev);
    cudaFree(s->status);
    cudaFree(s->nexact);
    cudaFree(s->build_scratch);
    cudaFree(s->solve_scratch);
    cudaFree(s->solve64);
    cudaFree(s->als_idx);
    cudaFree(s->als_w);
    cudaFree(s->als_SA);
    cudaFree(s->als_sumsq);
    cudaFree(s->als_part);
    cudaFree(s->nm_ws);
    delete s;
}

krp_status krp_create(krp_sampler** out, int N, const int64_t* I_host, int R, int F, int precision,
                      void* stream) {
    if (!out) return fail(nullptr, KRP_EINVAL, "krp_create: out is NULL");
    *out = nullptr;
    if (N < 1 || N > 16) return fail(nullptr, KRP_EINVAL, "krp_create: need 1 <= N <= 16");
    if (R < 1 || R > 128) return fail(nullptr, KRP_EINVAL, "krp_create: need 1 <= R <= 128");
    if (F == 0) F = R;
    if (F < 1 || F > 4 * R) return fail(nullptr, KRP_EINVAL, "krp_create: need 1 <= F <= 4R");
    if (!I_host) return fail(nullptr, KRP_EINVAL, "krp_create: I_host is NULL");
    for (int k = 0; k < N; ++k)
        if (I_host[k] < 1 || I_host[k] >= ((int64_t)1 << 31))
            return fail(nullptr, KRP_EINVAL, "krp_create: need 1 <= I_k < 2^31");
    if (precision != KRP_PREC_FP32 && precision != KRP_PREC_BF16X3 && precision != KRP_PREC_EXACT &&
        precision != KRP_PREC_TF32X3)
        return fail(nullptr, KRP_EINVAL, "krp_create: unknown precision");
    if (precision == KRP_PREC_EXACT && R > 32)
        return fail(nullptr, KRP_EINVAL, "krp_create: the exact-decision mode needs R <= 32");
    krp_sampler* s = new krp_sampler();
    s->exact = precision == KRP_PREC_EXACT ? 1 : 0;
    s->N = N;
    s->R = R;
    s->F = F;
    s->prec = precision;
    s->stream = (cudaStream_t)stream;
    s->T = tri_size(R);
    // exact-decision samplers keep one more float per node after the packed
    // triangle (the node's trace; in delta slots a bound on the delta's entries)
    s->Tp = s->exact ? ((s->T + 1 + 7) & ~7) : tri_stride(R);
    s->Rp = (int)next_pow2(R);
    s->dE = log2i(s->Rp);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete s;
        return fail(nullptr, KRP_ECUDA, std::string("krp_create: no CUDA device: ") + cudaGetErrorString(e));
    }
    s->I.assign(I_host, I_host + N);
    s->L.resize(N);
    s->depth.resize(N);
    s->U.assign(N, nullptr);
    s->tree.assign(N, nullptr);
    s->root64.assign(N, nullptr);
    s->tree_lo.assign(N, nullptr);
    s->dtop.assign(N, nullptr);
    s->Ke.assign(N, 0);
    s->has_factor.assign(N, 0);
    bool ok = true;
    for (int k = 0; k < N && ok; ++k) {
        const int64_t nleaf = (s->I[k] + F - 1) / F;
        s->L[k] = next_pow2(nleaf);
        s->depth[k] = log2i(s->L[k]);
        ok = dalloc(&s->U[k], (size_t)s->I[k] * R) && dalloc(&s->tree[k], (size_t)s->L[k] * s->Tp) &&
             dalloc(&s->root64[k], (size_t)s->Tp);
        if (ok) ok = cudaMemsetAsync(s->tree[k], 0, (size_t)s->L[k] * s->Tp * 4, s->stream) == cudaSuccess;
        if (ok && s->exact) {
            s->Ke[k] = std::min(KRP_EXACT_TOP, s->depth[k]);
            const size_t nd = ((size_t)1 << s->Ke[k]) * s->Tp;
            ok = dalloc(&s->tree_lo[k], (size_t)s->L[k] * s->Tp) && dalloc(&s->dtop[k], nd);
            if (ok) ok = cudaMemsetAsync(s->tree_lo[k], 0, (size_t)s->L[k] * s->Tp * 4, s->stream) == cudaSuccess;
            if (ok) ok = cudaMemsetAsync(s->dtop[k], 0, nd * 4, s->stream) == cudaSuccess;
        }
    }
    const size_t RR = (size_t)R * R;
    ok = ok && dalloc(&s->G64, N * RR) && dalloc(&s->Gplus64, RR) && dalloc(&s->lam64, (size_t)N * R) &&
         dalloc(&s->V64, N * RR) && dalloc(&s->work64, (size_t)6 * RR * (N + 1) + 256) &&
         dalloc(&s->Gplus32, (size_t)s->Tp) && dalloc(&s->etree, (size_t)N * s->Rp * s->Tp) &&
         dalloc(&s->V32, N * RR) && dalloc(&s->V32lo, N * RR) && dalloc(&s->rank_dev, 2) && dalloc(&s->status, 1) &&
         dalloc(&s->solve64, 3 * RR + 128 * (size_t)R);
    if (ok) ok = cudaMemsetAsync(s->status, 0, sizeof(int), s->stream) == cudaSuccess;
    if (ok && s->exact) ok = dalloc(&s->nexact, 1) &&
                             cudaMemsetAsync(s->nexact, 0, sizeof(unsigned long long), s->stream) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(s->etree, 0, (size_t)N * s->Rp * s->Tp * 4, s->stream) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(s->stream) == cudaSuccess;
    if (!ok) {
        krp_destroy(s);
        return fail(nullptr, KRP_ENOMEM, "krp_create: device allocation failed");
    }
    *out = s;
    return KRP_OK;
}

krp_status krp_set_factor_prec(krp_sampler* s, int j, const float* U, int precision) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    if (j < 0 || j >= s->N || !U) return fail(s, KRP_EINVAL, "krp_set_factor: bad factor index or NULL U");
    if (precision != KRP_PREC_FP32 && precision != KRP_PREC_BF16X3 && precision != KRP_PREC_EXACT &&
        precision != KRP_PREC_TF32X3)
        return fail(s, KRP_EINVAL, "krp_set_factor: unknown precision");
    if (precision == KRP_PREC_EXACT && !s->exact)
        return fail(s, KRP_EINVAL, "krp_set_factor: KRP_PREC_EXACT needs a sampler created with it");
    // Device-resident rows are read once by the build, which also writes the
    // sampler's copy; host rows are copied first.
    cudaPointerAttributes attr{};
    const bool on_device = cudaPointerGetAttributes(&attr, U) == cudaSuccess &&
                           (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    krp_status st;
    if (on_device) {
        st = build_tree(s, j, precision, U);
    } else {
        cudaError_t e = cudaMemcpyAsync(s->U[j], U, (size_t)s->I[j] * s->R * sizeof(float), cudaMemcpyDefault,
                                        s->stream);
        if (e != cudaSuccess) return cuda_check(s, e, "krp_set_factor copy");
        st = build_tree(s, j, precision);
    }
    if (st != KRP_OK) return st;
    s->has_factor[j] = 1;
    s->last_exclude = -2;  // Grams changed: the next draw needs a fresh prepare
    return KRP_OK;
}

krp_status krp_set_factor(krp_sampler* s, int j, const float* U) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    return krp_set_factor_prec(s, j, U, s->prec);
}

krp_status krp_set_descent_form(krp_sampler* s, int form) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    if (form != KRP_DESCENT_AUTO && form != KRP_DESCENT_TEAM && form != KRP_DESCENT_NODE_MAJOR &&
        form != KRP_DESCENT_NODE_MAJOR_TC)
        return fail(s, KRP_EINVAL, "krp_set_descent_form: unknown form");
    s->descent_form = form;
    return KRP_OK;
}

static krp_status check_sample_args(krp_sampler* s, int exclude_j) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    if (exclude_j < -1 || exclude_j >= s->N) return fail(s, KRP_EINVAL, "exclude_j out of range");
    if (s->N == 1 && exclude_j == 0) return fail(s, KRP_EINVAL, "no factor left to sample");
    for (int k = 0; k < s->N; ++k)
        if (k != exclude_j && !s->has_factor[k]) return fail(s, KRP_ESTATE, "factor not set");
    return KRP_OK;
}

krp_status krp_sample_prepare(krp_sampler* s, int exclude_j) {
    krp_status st = check_sample_args(s, exclude_j);
    if (st != KRP_OK) return st;
    return sampler_prep(s, exclude_j);
}

krp_status krp_sample_draw(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                           float* weight, float* logq, float* SA) {
    krp_status st = check_sample_args(s, exclude_j);
    if (st != KRP_OK) return st;
    if (s->last_exclude != exclude_j)
        return fail(s, KRP_ESTATE, "krp_sample_draw: krp_sample_prepare was not called for this exclude_j");
    if (J < 1 || J >= ((int64_t)1 << 31)) return fail(s, KRP_EINVAL, "krp_sample: need 1 <= J < 2^31");
    if (!idx || !weight) return fail(s, KRP_EINVAL, "krp_sample: idx and weight are required");
    return launch_descent(s, exclude_j, J, seed, draw_id, idx, weight, logq, SA);
}

krp_status krp_sample(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                      float* weight, float* logq, float* SA) {
    krp_status st = check_sample_args(s, exclude_j);
    if (st != KRP_OK) return st;
    if (J < 1 || J >= ((int64_t)1 << 31)) return fail(s, KRP_EINVAL, "krp_sample: need 1 <= J < 2^31");
    if (!idx || !weight) return fail(s, KRP_EINVAL, "krp_sample: idx and weight are required");
    st = sampler_prep(s, exclude_j);
    if (st != KRP_OK) return st;
    return launch_descent(s, exclude_j, J, seed, draw_id, idx, weight, logq, SA);
}

krp_status krp_debug_trace(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id,
                           int32_t* idx, float* weight, float* trace, int64_t n_trace) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    if (exclude_j < -1 || exclude_j >= s->N) return fail(s, KRP_EINVAL, "krp_debug_trace: exclude_j out of range");
    if (J < 1 || J >= ((int64_t)1 << 31) || !idx || !weight || !trace || n_trace < 1 || n_trace > J)
        return fail(s, KRP_EINVAL, "krp_debug_trace: bad J, n_trace or NULL buffer");
    if (s->N == 1 && exclude_j == 0) return fail(s, KRP_EINVAL, "krp_debug_trace: no factor left to sample");
    for (int k = 0; k < s->N; ++k)
        if (k != exclude_j && !s->has_factor[k]) return fail(s, KRP_ESTATE, "krp_debug_trace: factor not set");
    krp_status st = sampler_prep(s, exclude_j);
    if (st != KRP_OK) return st;
    return launch_descent(s, exclude_j, J, seed, draw_id, idx, weight, nullptr, nullptr, trace, n_trace);
}

krp_status krp_gather(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx, const float* weight,
                      float* SA) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    if (exclude_j < -1 || exclude_j >= s->N) return fail(s, KRP_EINVAL, "krp_gather: exclude_j out of range");
    if (J < 1 || J >= ((int64_t)1 << 31) || !idx || !weight || !SA)
        return fail(s, KRP_EINVAL, "krp_gather: bad J or NULL buffer");
    for (int k = 0; k < s->N; ++k)
        if (k != exclude_j && !s->has_factor[k]) return fail(s, KRP_ESTATE, "krp_gather: factor not set");
    return launch_gather(s, exclude_j, J, idx, weight, SA);
}

krp_status krp_solve_dense(krp_sampler* s, int64_t J, const float* SA, const float* weight, const float* B_rows,
                           int nrhs, float* X, int flags) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    if (J < 1 || J >= ((int64_t)1 << 31) || nrhs < 1 || nrhs > 64 || !SA || !weight || !B_rows || !X)
        return fail(s, KRP_EINVAL, "krp_solve_dense: bad J/nrhs or NULL buffer");
    return dense_solve(s, J, SA, weight, B_rows, nrhs, X, flags);
}

krp_status krp_sync_status(krp_sampler* s) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "krp_sync_status");
    int code = 0;
    e = cudaMemcpy(&code, s->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(s, e, "krp_sync_status read");
    if (code != 0) {
        const int zero = 0;
        cudaMemcpy(s->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
        const char* what = code == KRP_EZERO       ? "zero probability mass on the device"
                           : code == KRP_ENUMERIC  ? "non-finite probability mass on the device"
                           : code == KRP_ESINGULAR ? "normal matrix is not positive definite"
                                                   : "device-side failure";
        s->last_error = what;
    }
    return (krp_status)code;
}

int64_t krp_launch_count(void) { return krp::launch_counter(); }

krp_status krp_exact_count(krp_sampler* s, int64_t* count_host) {
    if (!s || !count_host) return fail(s, KRP_EINVAL, "krp_exact_count: NULL sampler or output");
    *count_host = 0;
    if (!s->exact) return KRP_OK;
    unsigned long long n = 0;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&n, s->nexact, sizeof(n), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(s, e, "krp_exact_count");
    *count_host = (int64_t)n;
    return KRP_OK;
}

krp_status krp_capture_begin(krp_sampler* s) {
    if (!s) return fail(nullptr, KRP_EINVAL, "krp_capture_begin: NULL sampler");
    if (s->capturing) return fail(s, KRP_ESTATE, "krp_capture_begin: already capturing");
    if (!s->stream) return fail(s, KRP_ESTATE, "krp_capture_begin: the sampler was created on the legacy stream");
    const cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) s->capturing = true;
    return cuda_check(s, e, "krp_capture_begin");
}

krp_status krp_capture_end(krp_sampler* s, int64_t* nodes_host) {
    if (!s) return fail(nullptr, KRP_EINVAL, "krp_capture_end: NULL sampler");
    if (!s->capturing) return fail(s, KRP_ESTATE, "krp_capture_end: not capturing");
    s->capturing = false;
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->graph_exec = nullptr;
    s->graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->stream, &s->graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph_exec, s->graph, 0);
    if (e == cudaSuccess && nodes_host) {
        size_t n = 0;
        e = cudaGraphGetNodes(s->graph, nullptr, &n);
        *nodes_host = (int64_t)n;
    }
    return cuda_check(s, e, "krp_capture_end");
}

krp_status krp_replay(krp_sampler* s) {
    if (!s) return fail(nullptr, KRP_EINVAL, "krp_replay: NULL sampler");
    if (!s->graph_exec) return fail(s, KRP_ESTATE, "krp_replay: nothing captured");
    return cuda_check(s, cudaGraphLaunch(s->graph_exec, s->stream), "krp_replay");
}

krp_status krp_debug_wait_timeout(krp_sampler* s, int tries) {
    if (!s) return fail(nullptr, KRP_EINVAL, "null sampler");
    if (tries < 1 || tries > 1000) return fail(s, KRP_EINVAL, "krp_debug_wait_timeout: need 1 <= tries <= 1000");
    return cuda_check(s, launch_wait_timeout_probe(s, tries), "wait probe launch");
}

const char* krp_last_error(const krp_sampler* s) { return s ? s->last_error.c_str() : g_error.c_str(); }

krp_status krp_tree_info(const krp_sampler* s, int j, int64_t* L_host, int* depth_host, int* node_stride_host) {
    if (!s || j < 0 || j >= s->N) return KRP_EINVAL;
    if (L_host) *L_host = s->L[j];
    if (depth_host) *depth_host = s->depth[j];
    if (node_stride_host) *node_stride_host = s->Tp;
    return KRP_OK;
}

krp_status krp_get_tree(const krp_sampler* s, int j, float* out_host, int64_t n_floats) {
    if (!s || j < 0 || j >= s->N || !out_host) return KRP_EINVAL;
    const int64_t n = s->L[j] * s->Tp;
    if (n_floats < n) return KRP_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return KRP_ECUDA;
    return cudaMemcpy(out_host, s->tree[j], n * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? KRP_OK : KRP_ECUDA;
}

krp_status krp_get_tree_exact(const krp_sampler* s, int j, float* lo_host, int64_t n_lo, float* dtop_host,
                              int64_t n_dtop) {
    if (!s || j < 0 || j >= s->N || !s->exact) return KRP_EINVAL;
    const int64_t nl = s->L[j] * s->Tp, nd = ((int64_t)1 << s->Ke[j]) * s->Tp;
    if ((lo_host && n_lo < nl) || (dtop_host && n_dtop < nd)) return KRP_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return KRP_ECUDA;
    if (lo_host && cudaMemcpy(lo_host, s->tree_lo[j], nl * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return KRP_ECUDA;
    if (dtop_host && cudaMemcpy(dtop_host, s->dtop[j], nd * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return KRP_ECUDA;
    return KRP_OK;
}

krp_status krp_get_factor(const krp_sampler* s, int j, float* out_host, int64_t n_floats) {
    if (!s || j < 0 || j >= s->N || !out_host || !s->has_factor[j]) return KRP_EINVAL;
    const int64_t n = s->I[j] * s->R;
    if (n_floats < n) return KRP_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return KRP_ECUDA;
    return cudaMemcpy(out_host, s->U[j], n * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? KRP_OK : KRP_ECUDA;
}

krp_status krp_get_prep(const krp_sampler* s, int k, double* lam_host, double* V_host, double* Gplus_host,
                        int* rank_host) {
    if (!s || k < 0 || k >= s->N) return KRP_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return KRP_ECUDA;
    const size_t RR = (size_t)s->R * s->R;
    bool ok = true;
    if (lam_host)
        ok = ok && cudaMemcpy(lam_host, s->lam64 + (size_t)k * s->R, s->R * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (V_host) ok = ok && cudaMemcpy(V_host, s->V64 + k * RR, RR * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (Gplus_host) ok = ok && cudaMemcpy(Gplus_host, s->Gplus64, RR * 8, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (rank_host) ok = ok && cudaMemcpy(rank_host, s->rank_dev, 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    return ok ? KRP_OK : KRP_ECUDA;
}

}  // extern "C"
