// Many independent KRP least-squares problems (config of many small samplers):
// each phase of the path runs as one launch over all problems — the
// segment-tree builds (Alg. 3), the preparation and descent of Alg. 2/4, and
// the normal-equation solve (Thm 2.1) — with the per-problem parameter blocks
// kept in device memory, so the whole sequence can be captured once as a CUDA
// graph and replayed.  Also the planted right-hand side used to pose such
// problems (B = A X + sigma xi evaluated at the sampled rows), which has no
// counterpart in the paper.
#include "common.cuh"
#include "internal.h"

#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

struct krp_batch {
    int P = 0, N = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::vector<krp_sampler*> s;
    int Rmax = 0, Fmax = 0, Tpmax = 0;
    std::vector<int64_t> row_off;  // prefix sums of R_p (P + 1)
    int64_t* row_off_dev = nullptr;
    krp::PrepItem* prep_dev = nullptr;
    krp::FastParams* fast_dev = nullptr;
    krp::PlantItem* plant_dev = nullptr;
    // build
    int LB = 8, Gmax = 1;
    bool vec = true;
    std::vector<krp::TreeDesc> trees;
    krp::TreeDesc* trees_dev = nullptr;
    int64_t* blk_prefix_dev = nullptr;
    int64_t nblocks = 0;
    std::vector<krp::UpDesc*> ups_dev;
    std::vector<int64_t*> up_prefix_dev;
    std::vector<int64_t> up_nctas;
    float* build_arena = nullptr;
    // solve
    int parts = 8, nrhs_max = 16;
    krp::SolveItem* solve_dev = nullptr;
    float* solve_arena = nullptr;
    int* status = nullptr;
    // descent
    int desc_ctas = 1;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool capturing = false;
    std::string last_error;
};

namespace krp {
namespace {

// ---------------------------------------------------------------- planted B --
// One warp per sampled row: a = ⊛_k U_k[i_k, :], B[s, c] = a · X[:, c] +
// sigma * xi(s, c).  xi is a standard normal by Box–Muller from Philox4x32-10
// with key (seed lo32, seed hi32) and counter (lin lo32, lin hi32, c,
// 0x9E3779B9), lin the C-order linear index of the tuple over the included
// factors (mod 2^64), so duplicated tuples get the same noise.
__device__ __forceinline__ void planted_row(const PlantItem& it, const int32_t* __restrict__ idx, int64_t J,
                                            const float* __restrict__ X, int nrhs, float sigma, uint2 key,
                                            float* __restrict__ B, int64_t s) {
    const int lane = threadIdx.x & 31;
    float a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = (lane + 32 * q < it.R) ? 1.f : 0.f;
    uint64_t lin = 0;
    for (int m = 0; m < it.N; ++m) {
        const int64_t i = idx[(int64_t)it.krow[m] * J + s];
        lin = lin * (uint64_t)it.I[m] + (uint64_t)i;
        const float* row = it.U[m] + i * it.R;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (lane + 32 * q < it.R) a[q] *= __ldg(row + lane + 32 * q);
    }
    for (int c = 0; c < nrhs; ++c) {
        float d = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (lane + 32 * q < it.R) d = fmaf(a[q], __ldg(X + (lane + 32 * q) * nrhs + c), d);
        d = warp_sum(d);
        if (lane == 0) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)lin, (uint32_t)(lin >> 32), (uint32_t)c, 0x9E3779B9u),
                                          key);
            const float u1 = u32_to_unit(r.x), u2 = u32_to_unit(r.y);
            const float xi = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
            B[s * nrhs + c] = d + sigma * xi;
        }
    }
}

__global__ void __launch_bounds__(256) planted_kernel(const PlantItem* __restrict__ items, int P, int64_t J,
                                                      const int32_t* __restrict__ idx, int N_idx,
                                                      const float* __restrict__ X, int nrhs, float sigma, uint2 key,
                                                      float* __restrict__ B) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < (int64_t)P * J; g += warps) {
        const int p = (int)(g / J);
        const int64_t s = g - (int64_t)p * J;
        const PlantItem& it = items[p];
        planted_row(it, idx + (int64_t)p * N_idx * J, J, X + it.row_off * nrhs, nrhs, sigma, key,
                    B + (int64_t)p * J * nrhs, s);
    }
}

__global__ void __launch_bounds__(256) planted_kernel_one(const __grid_constant__ PlantItem it, int64_t J,
                                                          const int32_t* __restrict__ idx,
                                                          const float* __restrict__ X, int nrhs, float sigma,
                                                          uint2 key, float* __restrict__ B) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < J; s += warps)
        planted_row(it, idx, J, X, nrhs, sigma, key, B, s);
}

template <typename T>
cudaError_t upload(T** dev, const std::vector<T>& host) {
    if (*dev) cudaFree(*dev);
    *dev = nullptr;
    if (host.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(dev, host.size() * sizeof(T));
    if (e == cudaSuccess) e = cudaMemcpy(*dev, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

krp_status bfail(krp_batch* b, krp_status code, const std::string& msg) {
    if (b) b->last_error = msg;
    return fail(nullptr, code, msg);
}

krp_status bcheck(krp_batch* b, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return KRP_OK;
    return bfail(b, KRP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

PlantItem plant_item_for(const krp_sampler* s, int exclude_j, int64_t row_off) {
    PlantItem it{};
    it.R = s->R;
    it.row_off = row_off;
    for (int k = 0; k < s->N; ++k) {
        if (k == exclude_j) continue;
        it.U[it.N] = s->U[k];
        it.I[it.N] = s->I[k];
        it.krow[it.N] = k;
        ++it.N;
    }
    return it;
}

// Point the tree descriptors at new sources (NULL: rebuild from the samplers'
// own copies) and refresh the device table in place, so a captured graph,
// which reads the table when it runs, picks the new sources up.
krp_status bind_sources(krp_batch* b, const float* const* U) {
    const int ntrees = b->P * b->N;
    for (int t = 0; t < ntrees; ++t) {
        TreeDesc& d = b->trees[t];
        krp_sampler* s = b->s[t / b->N];
        const int k = t % b->N;
        const float* src = U ? U[t] : nullptr;
        d.src = src ? src : s->U[k];
        d.copy_to = (src && src != s->U[k]) ? s->U[k] : nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!b->trees_dev) {
        std::vector<int64_t> prefix(ntrees + 1, 0);
        for (int t = 0; t < ntrees; ++t)
            prefix[t + 1] = prefix[t] + b->trees[t].L / ((int64_t)b->LB * b->trees[t].G);
        b->nblocks = prefix[ntrees];
        e = upload(&b->trees_dev, b->trees);
        if (e == cudaSuccess) e = upload(&b->blk_prefix_dev, prefix);
    } else {
        e = cudaMemcpy(b->trees_dev, b->trees.data(), b->trees.size() * sizeof(TreeDesc), cudaMemcpyHostToDevice);
    }
    return bcheck(b, e, "krp_batch: tree tables");
}

}  // namespace
}  // namespace krp

using namespace krp;

extern "C" {

krp_status krp_batch_create(krp_batch** out, krp_sampler* const* samplers, int P, void* stream) {
    if (!out) return fail(nullptr, KRP_EINVAL, "krp_batch_create: out is NULL");
    *out = nullptr;
    if (!samplers || P < 1) return fail(nullptr, KRP_EINVAL, "krp_batch_create: need P >= 1 samplers");
    krp_batch* b = new krp_batch();
    b->P = P;
    b->stream = static_cast<cudaStream_t>(stream);
    b->s.assign(samplers, samplers + P);
    b->N = samplers[0] ? samplers[0]->N : 0;
    for (int p = 0; p < P; ++p) {
        const krp_sampler* s = samplers[p];
        if (!s || s->N != b->N) {
            delete b;
            return fail(nullptr, KRP_EINVAL, "krp_batch_create: samplers must be non-NULL with equal N");
        }
        if (s->R > 32 || s->F > 32 || s->F < 1) {
            delete b;
            return fail(nullptr, KRP_EINVAL, "krp_batch_create: batched problems need R <= 32 and F <= 32");
        }
        if (s->exact) {
            delete b;
            return fail(nullptr, KRP_EINVAL, "krp_batch_create: exact-decision samplers are drawn one by one");
        }
        for (int k = 0; k < s->N; ++k)
            if (!s->has_factor[k]) {
                delete b;
                return fail(nullptr, KRP_ESTATE, "krp_batch_create: every factor of every sampler must be set");
            }
        b->Rmax = std::max(b->Rmax, s->R);
        b->Fmax = std::max(b->Fmax, s->F);
        b->Tpmax = std::max(b->Tpmax, s->Tp);
        if (s->R % 4) b->vec = false;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    // row offsets and the static parameter blocks
    b->row_off.assign(P + 1, 0);
    for (int p = 0; p < P; ++p) b->row_off[p + 1] = b->row_off[p] + samplers[p]->R;
    std::vector<PrepItem> prep(P);
    std::vector<FastParams> fast(P);
    std::vector<PlantItem> plant(P);
    for (int p = 0; p < P; ++p) {
        prep_item_for(samplers[p], -1, &prep[p]);
        fast_params_for(samplers[p], -1, &fast[p]);
        plant[p] = plant_item_for(samplers[p], -1, b->row_off[p]);
    }
    if (e == cudaSuccess) e = upload(&b->row_off_dev, b->row_off);
    if (e == cudaSuccess) e = upload(&b->prep_dev, prep);
    if (e == cudaSuccess) e = upload(&b->fast_dev, fast);
    if (e == cudaSuccess) e = upload(&b->plant_dev, plant);
    // tree build geometry: LB leaves per group (<= every tree's L), G <= 8 groups per block
    int64_t Lmin = INT64_MAX;
    for (int p = 0; p < P; ++p)
        for (int k = 0; k < b->N; ++k) Lmin = std::min(Lmin, samplers[p]->L[k]);
    b->LB = 1;
    while (b->LB < 8 && b->LB * 2 <= Lmin) b->LB *= 2;
    const int ntrees = P * b->N;
    b->trees.assign(ntrees, TreeDesc{});
    size_t arena = 0;
    std::vector<size_t> off(ntrees);
    for (int t = 0; t < ntrees; ++t) {
        krp_sampler* s = samplers[t / b->N];
        const int k = t % b->N;
        TreeDesc& d = b->trees[t];
        d.tree = s->tree[k];
        d.root64 = s->root64[k];
        d.I = s->I[k];
        d.L = s->L[k];
        d.R = s->R;
        d.F = s->F;
        d.Tp = s->Tp;
        d.G = 1;
        while (d.G < 8 && (int64_t)b->LB * d.G * 2 <= d.L) d.G *= 2;
        b->Gmax = std::max(b->Gmax, d.G);
        const int64_t tops = d.L / ((int64_t)b->LB * d.G);
        off[t] = arena;
        arena += (size_t)tops * 2 * d.Tp + 2 * (size_t)2 * (tops / 2 + 2) * d.Tp;  // pairs + two FP64 levels
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->build_arena, arena * sizeof(float));
    // level passes above the leaf kernel, per tree as build_tree does them:
    // lbb = min(16, n) nodes per CTA, ping-pong FP64 levels, the last pass
    // writing the FP64 root; trees with fewer passes sit out the later ones
    std::vector<std::vector<UpDesc>> passes;
    if (e == cudaSuccess) {
        for (int t = 0; t < ntrees; ++t) {
            TreeDesc& d = b->trees[t];
            float* base = b->build_arena + off[t];
            const int64_t tops = d.L / ((int64_t)b->LB * d.G);
            d.top = base;
            double* f64 = reinterpret_cast<double*>(base + (size_t)tops * 2 * d.Tp);
            d.up[0] = f64;
            d.up[1] = f64 + (size_t)(tops / 2 + 2) * d.Tp;
            int64_t n = tops;
            int q = 0;
            do {
                if ((int)passes.size() <= q) {
                    UpDesc idle{};
                    idle.lbb = 1;
                    passes.emplace_back(ntrees, idle);
                }
                UpDesc& u = passes[q][t];
                const int64_t lbb = std::min<int64_t>(16, n);
                u.Tp = d.Tp;
                u.tree = d.tree;
                u.n_in = n;
                u.lbb = (int)lbb;
                u.in_pairs = q == 0 ? d.top : nullptr;
                u.in64 = q == 0 ? nullptr : d.up[(q - 1) & 1];
                u.out = (n / lbb == 1) ? d.root64 : d.up[q & 1];
                n /= lbb;
                ++q;
            } while (n > 1);
        }
        for (auto& pass : passes) {
            std::vector<int64_t> prefix(ntrees + 1, 0);
            for (int t = 0; t < ntrees; ++t)
                prefix[t + 1] = prefix[t] + (pass[t].n_in > 0 ? pass[t].n_in / pass[t].lbb : 0);
            UpDesc* ud = nullptr;
            int64_t* pd = nullptr;
            e = upload(&ud, pass);
            if (e == cudaSuccess) e = upload(&pd, prefix);
            b->ups_dev.push_back(ud);
            b->up_prefix_dev.push_back(pd);
            b->up_nctas.push_back(prefix[ntrees]);
            if (e != cudaSuccess) break;
        }
    }
    if (e != cudaSuccess) {
        krp_batch_destroy(b);
        return fail(nullptr, KRP_ENOMEM, std::string("krp_batch_create: ") + cudaGetErrorString(e));
    }
    krp_status st = bind_sources(b, nullptr);
    // solve: `parts` partial sums per problem for nrhs <= nrhs_max
    std::vector<SolveItem> sol(P);
    size_t sarena = 0;
    for (int p = 0; p < P; ++p)
        sarena += (size_t)b->parts * (tri_size(samplers[p]->R) + samplers[p]->R * b->nrhs_max + 1);
    if (st == KRP_OK) e = cudaMalloc(&b->solve_arena, sarena * sizeof(float));
    if (st == KRP_OK && e == cudaSuccess) {
        size_t o = 0;
        for (int p = 0; p < P; ++p) {
            sol[p].R = samplers[p]->R;
            sol[p].nparts = b->parts;
            sol[p].row_off = b->row_off[p];
            sol[p].x_off = b->row_off[p];
            sol[p].part = b->solve_arena + o;
            o += (size_t)b->parts * (tri_size(samplers[p]->R) + samplers[p]->R * b->nrhs_max + 1);
        }
        e = upload(&b->solve_dev, sol);
    }
    if (st == KRP_OK && e == cudaSuccess) e = cudaMalloc(&b->status, sizeof(int));
    if (st == KRP_OK && e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
    if (st != KRP_OK || e != cudaSuccess) {
        krp_batch_destroy(b);
        return st != KRP_OK ? st : fail(nullptr, KRP_ENOMEM, std::string("krp_batch_create: ") + cudaGetErrorString(e));
    }
    *out = b;
    return KRP_OK;
}

void krp_batch_destroy(krp_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->row_off_dev);
    cudaFree(b->prep_dev);
    cudaFree(b->fast_dev);
    cudaFree(b->plant_dev);
    cudaFree(b->trees_dev);
    cudaFree(b->blk_prefix_dev);
    for (auto* p : b->ups_dev) cudaFree(p);
    for (auto* p : b->up_prefix_dev) cudaFree(p);
    cudaFree(b->build_arena);
    cudaFree(b->solve_dev);
    cudaFree(b->solve_arena);
    cudaFree(b->status);
    delete b;
}

krp_status krp_batch_set_sources(krp_batch* b, const float* const* U_host) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_set_sources: NULL batch");
    if (b->capturing) return bfail(b, KRP_ESTATE, "krp_batch_set_sources: not allowed while capturing");
    return bind_sources(b, U_host);
}

krp_status krp_batch_build(krp_batch* b) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_build: NULL batch");
    cudaError_t e = launch_leaves_batch(b->trees_dev, b->blk_prefix_dev, b->P * b->N, b->nblocks, b->LB, b->Rmax,
                                        b->Fmax, b->Tpmax, b->Gmax, b->vec, b->stream);
    for (size_t q = 0; q < b->ups_dev.size() && e == cudaSuccess; ++q)
        if (b->up_nctas[q] > 0)
            e = launch_up_batch(b->ups_dev[q], b->up_prefix_dev[q], b->P * b->N, b->up_nctas[q], b->Tpmax, q == 0,
                                b->stream);
    if (e == cudaSuccess)
        for (krp_sampler* s : b->s) s->last_exclude = -2;  // a factor changed: the next prep must rerun
    return bcheck(b, e, "krp_batch_build launch");
}

krp_status krp_batch_sample(krp_batch* b, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx, float* weight,
                            float* SA) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_sample: NULL batch");
    if (J < 1 || J >= ((int64_t)1 << 31) || !idx || !weight)
        return bfail(b, KRP_EINVAL, "krp_batch_sample: need 1 <= J < 2^31 and idx, weight");
    cudaError_t e = launch_prep_batch(b->prep_dev, b->P, b->N, b->Rmax, b->stream);
    if (e == cudaSuccess) {
        FastCall call{};
        call.key0 = (uint32_t)(seed & 0xffffffffu);
        call.key1 = (uint32_t)(seed >> 32);
        call.draw = (uint32_t)(draw_id & 0xffffffffu);
        call.N = b->N;
        call.J = J;
        call.idx = idx;
        call.weight = weight;
        call.SA = SA;
        call.row_off = b->row_off_dev;
        e = launch_descent_fast_batch(b->fast_dev, call, b->P, b->desc_ctas, b->stream);
    }
    if (e == cudaSuccess)
        for (krp_sampler* s : b->s) s->last_exclude = -1;
    return bcheck(b, e, "krp_batch_sample launch");
}

krp_status krp_batch_planted_rows(krp_batch* b, int64_t J, const int32_t* idx, const float* X_true, int nrhs,
                                  float sigma, uint64_t seed, float* B_rows) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_planted_rows: NULL batch");
    if (J < 1 || !idx || !X_true || !B_rows || nrhs < 1 || nrhs > 64)
        return bfail(b, KRP_EINVAL, "krp_batch_planted_rows: bad arguments");
    const int64_t warps = (int64_t)b->P * J;
    const int64_t grid = std::min<int64_t>((warps + 7) / 8, (int64_t)b->num_sms * 8);
    planted_kernel<<<(unsigned)grid, 256, 0, b->stream>>>(b->plant_dev, b->P, J, idx, b->N, X_true, nrhs, sigma,
                                                          make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), B_rows);
    count_launch();
    return bcheck(b, cudaGetLastError(), "krp_batch_planted_rows launch");
}

krp_status krp_batch_solve_dense(krp_batch* b, int64_t J, const float* SA, const float* weight, const float* B_rows,
                                 int nrhs, float* X, int flags) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_solve_dense: NULL batch");
    if (J < 1 || !SA || !weight || !B_rows || !X || nrhs < 1 || nrhs > b->nrhs_max)
        return bfail(b, KRP_EINVAL, "krp_batch_solve_dense: need J >= 1, buffers, 1 <= nrhs <= 16");
    const cudaError_t e = launch_solve_batch(b->solve_dev, b->P, b->parts, b->Rmax, J, SA, weight, B_rows, nrhs,
                                             flags, X, b->status, b->stream);
    return bcheck(b, e, "krp_batch_solve_dense launch");
}

krp_status krp_batch_sync_status(krp_batch* b) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_sync_status: NULL batch");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcheck(b, e, "krp_batch_sync_status");
    int st = 0, zero = 0;
    e = cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(b->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    for (krp_sampler* s : b->s) {  // the prep and descent report on each sampler's own word
        if (e != cudaSuccess || st != 0) break;
        e = cudaMemcpy(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && st != 0) e = cudaMemcpy(s->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return bcheck(b, e, "krp_batch_sync_status read");
    return (krp_status)st;
}

krp_status krp_batch_capture_begin(krp_batch* b) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_capture_begin: NULL batch");
    if (b->capturing) return bfail(b, KRP_ESTATE, "krp_batch_capture_begin: already capturing");
    if (!b->stream) return bfail(b, KRP_ESTATE, "krp_batch_capture_begin: the batch needs its own stream");
    const cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) b->capturing = true;
    return bcheck(b, e, "krp_batch_capture_begin");
}

krp_status krp_batch_capture_end(krp_batch* b, int64_t* nodes_host) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_capture_end: NULL batch");
    if (!b->capturing) return bfail(b, KRP_ESTATE, "krp_batch_capture_end: not capturing");
    b->capturing = false;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &b->graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess && nodes_host) {
        size_t n = 0;
        e = cudaGraphGetNodes(b->graph, nullptr, &n);
        *nodes_host = (int64_t)n;
    }
    return bcheck(b, e, "krp_batch_capture_end");
}

krp_status krp_batch_replay(krp_batch* b) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_replay: NULL batch");
    if (!b->exec) return bfail(b, KRP_ESTATE, "krp_batch_replay: nothing captured");
    return bcheck(b, cudaGraphLaunch(b->exec, b->stream), "krp_batch_replay");
}

krp_status krp_batch_set_tuning(krp_batch* b, int descent_ctas_per_problem) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_set_tuning: NULL batch");
    if (descent_ctas_per_problem < 1 || descent_ctas_per_problem > 64)
        return bfail(b, KRP_EINVAL, "krp_batch_set_tuning: descent CTAs per problem in 1..64");
    b->desc_ctas = descent_ctas_per_problem;
    return KRP_OK;
}

krp_status krp_batch_autotune(krp_batch* b, int64_t J, int* best_host) {
    if (!b) return fail(nullptr, KRP_EINVAL, "krp_batch_autotune: NULL batch");
    if (b->capturing) return bfail(b, KRP_ESTATE, "krp_batch_autotune: not allowed while capturing");
    if (J < 1 || J >= ((int64_t)1 << 31)) return bfail(b, KRP_EINVAL, "krp_batch_autotune: need 1 <= J < 2^31");
    int32_t* idx = nullptr;
    float* w = nullptr;
    cudaError_t e = cudaMalloc(&idx, (size_t)b->P * b->N * J * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&w, (size_t)b->P * J * sizeof(float));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    int best = b->desc_ctas;
    float best_ms = 1e30f;
    const int cands[] = {1, 2, 4, 8, 16};
    krp_status st = KRP_OK;
    if (e == cudaSuccess) st = krp_batch_sample(b, J, 0x5eedULL, 0, idx, w, nullptr);  // warm-up
    for (int c : cands) {
        if (e != cudaSuccess || st != KRP_OK) break;
        b->desc_ctas = c;
        cudaEventRecord(t0, b->stream);
        st = krp_batch_sample(b, J, 0x5eedULL, 1, idx, w, nullptr);
        cudaEventRecord(t1, b->stream);
        e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    b->desc_ctas = best;
    if (best_host) *best_host = best;
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(idx);
    cudaFree(w);
    if (st != KRP_OK) return st;
    return bcheck(b, e, "krp_batch_autotune");
}

const char* krp_batch_last_error(const krp_batch* b) { return b ? b->last_error.c_str() : krp_last_error(nullptr); }

// ------------------------------------------------------------ single planted --
krp_status krp_planted_rows(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx, const float* X_true,
                            int nrhs, float sigma, uint64_t seed, float* B_rows) {
    if (!s) return fail(nullptr, KRP_EINVAL, "krp_planted_rows: NULL sampler");
    if (J < 1 || !idx || !X_true || !B_rows || nrhs < 1 || nrhs > 64 || exclude_j < -1 || exclude_j >= s->N)
        return fail(s, KRP_EINVAL, "krp_planted_rows: bad arguments");
    if (s->R > 128) return fail(s, KRP_EINVAL, "krp_planted_rows: R > 128");
    for (int k = 0; k < s->N; ++k)
        if (k != exclude_j && !s->has_factor[k]) return fail(s, KRP_ESTATE, "krp_planted_rows: factor not set");
    const PlantItem it = plant_item_for(s, exclude_j, 0);
    const int64_t grid = std::min<int64_t>((J + 7) / 8, (int64_t)s->num_sms * 8);
    planted_kernel_one<<<(unsigned)grid, 256, 0, s->stream>>>(it, J, idx, X_true, nrhs, sigma,
                                                              make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)),
                                                              B_rows);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    return cuda_check(s, e, "krp_planted_rows");
}

}  // extern "C"
