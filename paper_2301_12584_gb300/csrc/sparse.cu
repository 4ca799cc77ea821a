// a7 + a8 (sparse) + a9: sampled-fiber lookup, scatter SpMM, Y M⁻¹, column
// normalisation, and the STS-CP sweep (Sec. 3.3; Alg. 6; App. A.9; fit of
// Sec. 4.3).
//
// Mode-j index (built once, host sort as in the paper's preprocessing): every
// nonzero gets the key packing its coordinates in the modes k != j (ascending
// k, ceil(log2 I_k) bits each); nonzeros are sorted by key, equal keys form a
// mode-j fiber (one row of mat(T, j)ᵀ restricted to its nonzeros).
// Lookup: a thread per sampled tuple binary-searches its key among the fiber
// keys.  Samples of the same fiber are then merged (their contributions
// differ only in the sketched row, so Σ_s w_s SA[s, :] per fiber is formed
// first, in a hash table keyed by the fiber, with H >= 2J slots); an
// exclusive scan of the merged fibers' lengths numbers the (fiber, nonzero)
// pairs, and warps take equal runs of those pairs, adding
// Y[i_j, :] += v · (Σ_s w_s SA[s, :])  (Y = SBᵀ SA, I_j x R) for each
// nonzero (i_j, v).  Repeated Zipf-hot fibers are so scattered once, and
// fibers of very different lengths spread over all warps.
// Then U_j = Y M⁻¹ with M = SAᵀ SA (FP64 Cholesky inverse, applied in FP32).
#include "common.cuh"
#include "internal.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

namespace krp {

struct LookupParams {
    const uint64_t* fkeys;
    const int64_t* fptr;
    const int32_t* fidx;
    const float* fval;
    int64_t nfib;
    int other[16];
    int kbits[16];
    int n_other;
    const int32_t* idx;  // N x J
    const float* weight;
    const float* SA;     // J x R
    int64_t J;
    int R;
    float* Y;            // I_j x RS, RS = R rounded up to 4 (columns >= R unused)
    int RS;
};

__global__ void __launch_bounds__(256) fiber_find(LookupParams P, int64_t* __restrict__ fiber) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < P.J; s += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
        for (int q = 0; q < P.n_other; ++q)
            key = (key << P.kbits[q]) | (uint64_t)(uint32_t)P.idx[(int64_t)P.other[q] * P.J + s];
        int64_t lo = 0, hi = P.nfib;  // lower_bound over the sorted fiber keys
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(P.fkeys + mid) < key)
                lo = mid + 1;
            else
                hi = mid;
        }
        fiber[s] = (lo < P.nfib && __ldg(P.fkeys + lo) == key) ? lo : -1;  // -1: the SB row is zero
    }
}

constexpr unsigned long long SLOT_EMPTY = ~0ull;

// A warp per sample: find (or claim) the fiber's slot by linear probing, then
// add w_s SA[s, :] to the slot's R-vector.
__global__ void __launch_bounds__(256) merge_samples(LookupParams P, const int64_t* __restrict__ fiber,
                                                     unsigned long long* __restrict__ keys, float* __restrict__ acc,
                                                     int log2H) {
    const int lane = threadIdx.x & 31;
    const int64_t H = (int64_t)1 << log2H;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < P.J; s += warps) {
        const int64_t f = fiber[s];
        if (f < 0) continue;
        int64_t slot = -1;
        if (lane == 0) {
            int64_t h = (int64_t)(((unsigned long long)f * 0x9E3779B97F4A7C15ull) >> (64 - log2H));
            for (int64_t probe = 0; probe < H; ++probe) {  // H >= 2J: a slot is always found
                const unsigned long long old = atomicCAS(keys + h, SLOT_EMPTY, (unsigned long long)f);
                if (old == SLOT_EMPTY || old == (unsigned long long)f) {
                    slot = h;
                    break;
                }
                h = (h + 1) & (H - 1);
            }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot < 0) continue;
        const float ws = __ldg(P.weight + s);
        for (int a = lane; a < P.R; a += 32) atomicAdd(acc + slot * P.R + a, ws * __ldg(P.SA + s * P.R + a));
    }
}

// Per slot: first nonzero and length of its fiber (0 for an empty slot).
__global__ void __launch_bounds__(256) slot_lengths(LookupParams P, const unsigned long long* __restrict__ keys,
                                                    int64_t H, int64_t* __restrict__ begin,
                                                    int64_t* __restrict__ len) {
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < H; h += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long f = keys[h];
        const bool used = f != SLOT_EMPTY;
        begin[h] = used ? __ldg(P.fptr + f) : 0;
        len[h] = used ? __ldg(P.fptr + f + 1) - __ldg(P.fptr + f) : 0;
    }
}

// Exclusive scan of len[0..n) into scan[0..n] (scan[n] = total), one CTA.
__global__ void __launch_bounds__(1024) scan_lengths(const int64_t* __restrict__ len, int64_t* __restrict__ scan,
                                                     int64_t n) {
    __shared__ int64_t part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t a = threadIdx.x * per, b = min(n, a + per);
    int64_t sum = 0;
    for (int64_t i = a; i < b; ++i) sum += len[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // inclusive Hillis-Steele scan
        const int64_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - sum;
    for (int64_t i = a; i < b; ++i) {
        scan[i] = run;
        run += len[i];
    }
    if (threadIdx.x == blockDim.x - 1) scan[n] = part[threadIdx.x];
}

// Warps take runs of SCATTER_RUN consecutive (slot, nonzero) pairs; lane l
// adds columns 4l .. 4l+3 of a nonzero's row with one vector atomic (Y rows
// are RS = R rounded up to 4 floats, 16-byte aligned; the padding columns
// receive zeros).
constexpr int SCATTER_RUN = 32;

__global__ void __launch_bounds__(256) fiber_scatter(LookupParams P, const int64_t* __restrict__ begin,
                                                     const int64_t* __restrict__ scan, int64_t H,
                                                     const float* __restrict__ acc) {
    const int lane = threadIdx.x & 31;
    const int64_t total = scan[H];
    const int64_t nrun = (total + SCATTER_RUN - 1) / SCATTER_RUN;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t run = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); run < nrun; run += warps) {
        const int64_t w0 = run * SCATTER_RUN, w1 = min(total, w0 + SCATTER_RUN);
        int64_t lo = 0, hi = H - 1;  // last slot with scan[h] <= w0
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(scan + mid) <= w0)
                lo = mid;
            else
                hi = mid - 1;
        }
        int64_t h = lo;
        for (int64_t w = w0; w < w1; ++w) {
            while (__ldg(scan + h + 1) <= w) ++h;
            const int64_t n = __ldg(begin + h) + (w - __ldg(scan + h));
            const int64_t ij = __ldg(P.fidx + n);
            const float v = __ldg(P.fval + n);
            const float* ah = acc + h * P.R;
            for (int a = 4 * lane; a < P.R; a += 128) {
                float4 d;
                d.x = v * __ldg(ah + a);
                d.y = a + 1 < P.R ? v * __ldg(ah + a + 1) : 0.f;
                d.z = a + 2 < P.R ? v * __ldg(ah + a + 2) : 0.f;
                d.w = a + 3 < P.R ? v * __ldg(ah + a + 3) : 0.f;
                atomicAdd(reinterpret_cast<float4*>(P.Y + ij * P.RS + a), d);
            }
        }
    }
}

// U[i, :] = Y[i, :] M⁻¹ (M⁻¹ FP64 -> FP32 in shared memory) and, when sumsq
// is non-null, σ²[c] += Σ_i U[i, c]² (double-float partials per thread, one
// FP64 atomic per column and CTA).  Persistent CTAs walk tiles of TM rows of
// Y, staged in shared memory with row stride R | 1 (the rows a warp reads
// fall in distinct banks); thread (ty, tx) accumulates RT rows x 8 columns,
// {4tx .. 4tx+3} and {RP/2 + 4tx ..}, against float4 rows of M⁻¹ (columns
// >= R zero).  RP = R padded to 32, 64 or 128.
constexpr int MINV_THREADS = 256;
template <int RP>
struct MinvCfg {
    static constexpr int TX = RP / 8, TY = MINV_THREADS / TX, RT = 4, TM = TY * RT;
    // M⁻¹, then the Y tile, which the final column reduction reuses for
    // 8 x MINV_THREADS doubles
    static size_t smem(int R) {
        return (size_t)RP * RP * 4 + std::max<size_t>((size_t)TM * (R | 1) * 4, (size_t)8 * MINV_THREADS * 8);
    }
};

template <int RP>
__global__ void __launch_bounds__(MINV_THREADS, 2) apply_minv(const float* __restrict__ Y, int RSY,
                                                              const double* __restrict__ Minv, int64_t I, int R,
                                                              float* __restrict__ U, double* __restrict__ sumsq) {
    using C = MinvCfg<RP>;
    constexpr int TX = C::TX, RT = C::RT, TM = C::TM;
    extern __shared__ __align__(16) float sm[];
    float* sM = sm;              // [R][RP]
    float* sY = sM + RP * RP;    // [TM][RS]
    const int RS = R | 1;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k < R; k += MINV_THREADS / 32)
        for (int c = lane; c < RP; c += 32) sM[k * RP + c] = c < R ? (float)Minv[k * R + c] : 0.f;
    df ss[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ss[q] = df{0.f, 0.f};
    const int64_t ntiles = (I + TM - 1) / TM;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * TM;
        const int nr = (int)min((int64_t)TM, I - r0);
        __syncthreads();   // the previous tile's reads of sY (and the writes of sM) are done
        const float* src = Y + r0 * RSY;
        for (int r = warp; r < nr; r += MINV_THREADS / 32)
            for (int k = lane; k < R; k += 32) sY[r * RS + k] = src[(int64_t)r * RSY + k];
        __syncthreads();
        float2 acc[RT][4];
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = make_float2(0.f, 0.f);
        const float* yrow = sY + ty * RT * RS;
        for (int k = 0; k < R; ++k) {
            const float4 m0 = *reinterpret_cast<const float4*>(sM + k * RP + 4 * tx);
            const float4 m1 = *reinterpret_cast<const float4*>(sM + k * RP + RP / 2 + 4 * tx);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float y = yrow[r * RS + k];
                const float2 yy = make_float2(y, y);
                acc[r][0] = ffma2(yy, make_float2(m0.x, m0.y), acc[r][0]);
                acc[r][1] = ffma2(yy, make_float2(m0.z, m0.w), acc[r][1]);
                acc[r][2] = ffma2(yy, make_float2(m1.x, m1.y), acc[r][2]);
                acc[r][3] = ffma2(yy, make_float2(m1.z, m1.w), acc[r][3]);
            }
        }
        // rows >= nr hold stale shared memory: neither written nor summed
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int row = ty * RT + r;
            if (row >= nr) continue;
            float* dst = U + (r0 + row) * R;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c0 = h * (RP / 2) + 4 * tx;
                const float v[4] = {acc[r][2 * h].x, acc[r][2 * h].y, acc[r][2 * h + 1].x, acc[r][2 * h + 1].y};
                if ((R & 3) == 0 && c0 + 3 < R) {
                    *reinterpret_cast<float4*>(dst + c0) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c0 + q < R) dst[c0 + q] = v[q];
                }
                if (sumsq) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) ss[4 * h + q] = df_add(ss[4 * h + q], df{v[q] * v[q], 0.f});
                }
            }
        }
    }
    if (!sumsq) return;
    // column totals: the TY threads of a column group in fixed order, then one
    // FP64 atomic per column
    __syncthreads();
    double* red = reinterpret_cast<double*>(sY);   // [TY][8 x TX] doubles <= TM * RS floats
#pragma unroll
    for (int q = 0; q < 8; ++q) red[ty * 8 * TX + q * TX + tx] = (double)ss[q].hi + (double)ss[q].lo;
    __syncthreads();
    for (int col = threadIdx.x; col < R; col += MINV_THREADS) {
        const int h = col / (RP / 2), rem = col % (RP / 2), t = rem / 4, q = 4 * h + rem % 4;
        double a = 0.0;
        for (int y = 0; y < C::TY; ++y) a += red[y * 8 * TX + q * TX + t];
        atomicAdd(sumsq + col, a);
    }
}

template <int RP>
cudaError_t launch_minv_t(const float* Y, int RSY, const double* Minv, int64_t I, int R, float* U, double* sumsq,
                          int num_sms, cudaStream_t st) {
    using C = MinvCfg<RP>;
    const size_t sm = C::smem(R);
    cudaError_t e = cudaFuncSetAttribute(apply_minv<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (I + C::TM - 1) / C::TM;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms * 2);
    apply_minv<RP><<<(unsigned)grid, MINV_THREADS, sm, st>>>(Y, RSY, Minv, I, R, U, sumsq);
    count_launch();
    return cudaGetLastError();
}

// Y: I x RSY (row stride RSY >= R)
cudaError_t launch_apply_minv(const float* Y, int RSY, const double* Minv, int64_t I, int R, float* U,
                              double* sumsq, int num_sms, cudaStream_t st) {
    if (R <= 32) return launch_minv_t<32>(Y, RSY, Minv, I, R, U, sumsq, num_sms, st);
    if (R <= 64) return launch_minv_t<64>(Y, RSY, Minv, I, R, U, sumsq, num_sms, st);
    return launch_minv_t<128>(Y, RSY, Minv, I, R, U, sumsq, num_sms, st);
}

// U[:, c] /= σ_c (a zero column stays zero), σ_c = sqrt(σ²_c) to sigma;
// a warp per row, lanes over columns.
__global__ void __launch_bounds__(256) col_scale(float* __restrict__ U, int64_t I, int R,
                                                 const double* __restrict__ sumsq, float* __restrict__ sigma) {
    __shared__ float inv[128];
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        const double sg = sqrt(sumsq[c]);
        inv[c] = sg > 0.0 ? (float)(1.0 / sg) : 1.f;
        if (blockIdx.x == 0) sigma[c] = (float)sg;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < I;
         i += (int64_t)gridDim.x * (blockDim.x >> 5))
        for (int c = lane; c < R; c += 32) U[i * R + c] *= inv[c];
}

// ⟨T, T̃⟩ = Σ_nnz v Σ_r σ_r Π_k U_k[i_k, r]  (FP64 accumulation).
struct FitParams {
    const float* U[16];
    const int32_t* coords;  // N x nnz
    const float* vals;
    const float* sigma;
    int64_t nnz;
    int N, R;
    double* out;
};

__global__ void __launch_bounds__(256) fit_inner(FitParams P) {
    __shared__ double red[8];
    double a = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P.nnz; e += (int64_t)gridDim.x * blockDim.x) {
        float m = 0.f;
        for (int r = 0; r < P.R; ++r) {
            float p = P.sigma[r];
            for (int k = 0; k < P.N; ++k) p *= __ldg(P.U[k] + (int64_t)P.coords[(int64_t)k * P.nnz + e] * P.R + r);
            m += p;
        }
        a += (double)P.vals[e] * (double)m;
    }
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(P.out, t);
    }
}

}  // namespace krp

using namespace krp;

namespace {

// Stable LSD radix sort of (key, perm) by key, 16-bit digits over `bits` bits.
void radix_sort(std::vector<uint64_t>& key, std::vector<uint32_t>& perm, int bits) {
    const size_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<uint32_t> p2(n);
    std::vector<size_t> cnt(65537);
    for (int shift = 0; shift < bits; shift += 16) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (size_t i = 0; i < n; ++i) ++cnt[((key[i] >> shift) & 0xffff) + 1];
        for (int d = 0; d < 65536; ++d) cnt[d + 1] += cnt[d];
        for (size_t i = 0; i < n; ++i) {
            const size_t dst = cnt[(key[i] >> shift) & 0xffff]++;
            k2[dst] = key[i];
            p2[dst] = perm[i];
        }
        key.swap(k2);
        perm.swap(p2);
    }
}

int bits_for(int64_t I) {
    int b = 1;
    while (b < 62 && ((int64_t)1 << b) < I) ++b;
    return b;
}

template <typename T>
bool dmalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

thread_local std::string g_tensor_error;

}  // namespace

extern "C" krp_status krp_sptensor_create(krp_sptensor** out, int N, const int64_t* I_host, int64_t nnz,
                                          const int32_t* const* coords_host, const float* vals_host,
                                          void* stream) {
    if (!out) return KRP_EINVAL;
    *out = nullptr;
    if (N < 2 || N > 16 || !I_host || !coords_host || !vals_host || nnz < 1 || nnz >= ((int64_t)1 << 32))
        return KRP_EINVAL;
    for (int k = 0; k < N; ++k)
        if (I_host[k] < 1 || I_host[k] >= ((int64_t)1 << 31) || !coords_host[k]) return KRP_EINVAL;
    for (int j = 0; j < N; ++j) {
        int b = 0;
        for (int k = 0; k < N; ++k)
            if (k != j) b += bits_for(I_host[k]);
        if (b > 63) return KRP_EINVAL;
    }
    for (int k = 0; k < N; ++k)
        for (int64_t e = 0; e < nnz; ++e)
            if (coords_host[k][e] < 0 || coords_host[k][e] >= I_host[k]) return KRP_EINVAL;
    krp_sptensor* t = new krp_sptensor();
    t->N = N;
    t->nnz = nnz;
    t->stream = (cudaStream_t)stream;
    t->I.assign(I_host, I_host + N);
    t->kbits.resize(N);
    for (int k = 0; k < N; ++k) t->kbits[k] = bits_for(I_host[k]);
    double n2 = 0.0;
    for (int64_t e = 0; e < nnz; ++e) n2 += (double)vals_host[e] * (double)vals_host[e];
    t->normT2 = n2;
    bool ok = dmalloc(&t->coords, (size_t)N * nnz) && dmalloc(&t->vals, (size_t)nnz);
    for (int k = 0; ok && k < N; ++k)
        ok = cudaMemcpy(t->coords + (size_t)k * nnz, coords_host[k], nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(t->vals, vals_host, nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    t->fkeys.assign(N, nullptr);
    t->fptr.assign(N, nullptr);
    t->fidx.assign(N, nullptr);
    t->fval.assign(N, nullptr);
    t->nfib.assign(N, 0);
    std::vector<uint64_t> key(nnz);
    std::vector<uint32_t> perm(nnz);
    for (int j = 0; ok && j < N; ++j) {
        int bits = 0;
        for (int64_t e = 0; e < nnz; ++e) {
            uint64_t kk = 0;
            for (int k = 0; k < N; ++k)
                if (k != j) kk = (kk << t->kbits[k]) | (uint64_t)(uint32_t)coords_host[k][e];
            key[e] = kk;
            perm[e] = (uint32_t)e;
        }
        for (int k = 0; k < N; ++k)
            if (k != j) bits += t->kbits[k];
        radix_sort(key, perm, bits);
        std::vector<uint64_t> fk;
        std::vector<int64_t> fp;
        std::vector<int32_t> fi(nnz);
        std::vector<float> fv(nnz);
        for (int64_t e = 0; e < nnz; ++e) {
            if (e == 0 || key[e] != key[e - 1]) {
                fk.push_back(key[e]);
                fp.push_back(e);
            }
            fi[e] = coords_host[j][perm[e]];
            fv[e] = vals_host[perm[e]];
        }
        fp.push_back(nnz);
        t->nfib[j] = (int64_t)fk.size();
        ok = dmalloc(&t->fkeys[j], fk.size()) && dmalloc(&t->fptr[j], fp.size()) && dmalloc(&t->fidx[j], (size_t)nnz) &&
             dmalloc(&t->fval[j], (size_t)nnz);
        ok = ok && cudaMemcpy(t->fkeys[j], fk.data(), fk.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t->fptr[j], fp.data(), fp.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t->fidx[j], fi.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t->fval[j], fv.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        krp_sptensor_destroy(t);
        return KRP_ENOMEM;
    }
    *out = t;
    return KRP_OK;
}

extern "C" void krp_sptensor_destroy(krp_sptensor* t) {
    if (!t) return;
    cudaStreamSynchronize(t->stream);
    cudaFree(t->coords);
    cudaFree(t->vals);
    for (int j = 0; j < (int)t->fkeys.size(); ++j) {
        cudaFree(t->fkeys[j]);
        cudaFree(t->fptr[j]);
        cudaFree(t->fidx[j]);
        cudaFree(t->fval[j]);
    }
    cudaFree(t->Y);
    cudaFree(t->lk_fiber);
    cudaFree(t->lk_keys);
    cudaFree(t->lk_begin);
    cudaFree(t->lk_len);
    cudaFree(t->lk_scan);
    cudaFree(t->lk_acc);
    delete t;
}

namespace krp {
// krp_solve_sparse, plus σ²[c] += Σ_i U_out[i, c]² when sumsq is non-null
krp_status solve_sparse_impl(krp_sampler* s, const krp_sptensor* tc, int j, int64_t J, const int32_t* idx,
                             const float* weight, const float* SA, float* U_out, int flags, double* sumsq) {
    if (!s || !tc || !idx || !weight || !SA || !U_out) return s ? fail(s, KRP_EINVAL, "null argument") : KRP_EINVAL;
    krp_sptensor* t = const_cast<krp_sptensor*>(tc);
    if (t->N != s->N || j < 0 || j >= s->N || J < 1 || J >= ((int64_t)1 << 31))
        return fail(s, KRP_EINVAL, "krp_solve_sparse: bad mode, J or tensor order");
    for (int k = 0; k < s->N; ++k)
        if (t->I[k] != s->I[k]) return fail(s, KRP_EINVAL, "krp_solve_sparse: tensor dims differ from the factors");
    const int R = s->R;
    const int RS = (R + 3) & ~3;   // Y's row stride: rows 16-byte aligned for the vector atomics
    const size_t ny = (size_t)s->I[j] * RS;
    if (ny > t->Y_floats) {
        cudaFree(t->Y);
        t->Y = nullptr;
        t->Y_floats = 0;
        if (!dmalloc(&t->Y, ny)) return fail(s, KRP_ENOMEM, "sparse Y scratch allocation failed");
        t->Y_floats = ny;
    }
    cudaError_t e = cudaMemsetAsync(t->Y, 0, ny * sizeof(float), s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "Y memset");
    LookupParams P{};
    P.fkeys = t->fkeys[j];
    P.fptr = t->fptr[j];
    P.fidx = t->fidx[j];
    P.fval = t->fval[j];
    P.nfib = t->nfib[j];
    for (int k = 0; k < s->N; ++k)
        if (k != j) {
            P.other[P.n_other] = k;
            P.kbits[P.n_other] = t->kbits[k];
            ++P.n_other;
        }
    P.idx = idx;
    P.weight = weight;
    P.SA = SA;
    P.J = J;
    P.R = R;
    P.Y = t->Y;
    P.RS = RS;
    int log2H = 1;
    while (((int64_t)1 << log2H) < 2 * J) ++log2H;
    const int64_t H = (int64_t)1 << log2H;
    if ((size_t)H + 1 > t->lk_n || (size_t)H * R > t->lk_acc_n) {
        cudaFree(t->lk_fiber);
        cudaFree(t->lk_keys);
        cudaFree(t->lk_begin);
        cudaFree(t->lk_len);
        cudaFree(t->lk_scan);
        cudaFree(t->lk_acc);
        t->lk_fiber = t->lk_begin = t->lk_len = t->lk_scan = nullptr;
        t->lk_keys = nullptr;
        t->lk_acc = nullptr;
        t->lk_n = t->lk_acc_n = 0;
        if (!dmalloc(&t->lk_fiber, H + 1) || !dmalloc(&t->lk_keys, H + 1) || !dmalloc(&t->lk_begin, H + 1) ||
            !dmalloc(&t->lk_len, H + 1) || !dmalloc(&t->lk_scan, H + 1) || !dmalloc(&t->lk_acc, (size_t)H * R))
            return fail(s, KRP_ENOMEM, "sparse lookup scratch allocation failed");
        t->lk_n = (size_t)H + 1;
        t->lk_acc_n = (size_t)H * R;
    }
    e = cudaMemsetAsync(t->lk_keys, 0xFF, (size_t)H * sizeof(unsigned long long), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->lk_acc, 0, (size_t)H * R * sizeof(float), s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "lookup table memset");
    const int64_t g0 = std::min<int64_t>((J + 255) / 256, (int64_t)s->num_sms * 8);
    fiber_find<<<(unsigned)g0, 256, 0, s->stream>>>(P, t->lk_fiber); count_launch();
    const int64_t g1 = std::min<int64_t>((J + 7) / 8, (int64_t)s->num_sms * 16);
    merge_samples<<<(unsigned)g1, 256, 0, s->stream>>>(P, t->lk_fiber, t->lk_keys, t->lk_acc, log2H); count_launch();
    const int64_t gs = std::min<int64_t>((H + 255) / 256, (int64_t)s->num_sms * 8);
    slot_lengths<<<(unsigned)gs, 256, 0, s->stream>>>(P, t->lk_keys, H, t->lk_begin, t->lk_len); count_launch();
    scan_lengths<<<1, 1024, 0, s->stream>>>(t->lk_len, t->lk_scan, H); count_launch();
    fiber_scatter<<<(unsigned)(s->num_sms * 16), 256, 0, s->stream>>>(P, t->lk_begin, t->lk_scan, H, t->lk_acc);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "fiber lookup launch");
    krp_status st = normal_inverse(s, J, SA, flags);
    if (st != KRP_OK) return st;
    const double* Minv = s->solve64 + (size_t)(2 * R * R + R * 128);
    e = launch_apply_minv(t->Y, RS, Minv, s->I[j], R, U_out, sumsq, s->num_sms, s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "apply_minv launch");
    return KRP_OK;
}
}  // namespace krp

extern "C" krp_status krp_solve_sparse(krp_sampler* s, const krp_sptensor* tc, int j, int64_t J,
                                       const int32_t* idx, const float* weight, const float* SA, float* U_out,
                                       int flags) {
    return solve_sparse_impl(s, tc, j, J, idx, weight, SA, U_out, flags, nullptr);
}

namespace krp {
krp_status als_buffers(krp_sampler* s, int64_t J, int32_t** idx, float** w, float** SA, double** sumsq);
}

extern "C" krp_status krp_cp_als_sweep(krp_sampler* s, const krp_sptensor* t, int64_t J, uint64_t seed,
                                       uint64_t draw_base, float* sigma) {
    if (!s || !t || !sigma) return s ? fail(s, KRP_EINVAL, "null argument") : KRP_EINVAL;
    int32_t* idx;
    float *w, *SA;
    double* sumsq;
    krp_status st = als_buffers(s, J, &idx, &w, &SA, &sumsq);
    if (st != KRP_OK) return st;
    const int R = s->R;
    for (int j = 0; j < s->N; ++j) {
        st = krp_sample(s, j, J, seed, draw_base + (uint64_t)j, idx, w, nullptr, SA);
        if (st != KRP_OK) return st;
        cudaError_t e = cudaMemsetAsync(sumsq, 0, R * sizeof(double), s->stream);
        if (e != cudaSuccess) return cuda_check(s, e, "sumsq memset");
        // U_j = Y M⁻¹ with its column sums of squares from the same pass
        st = solve_sparse_impl(s, t, j, J, idx, w, SA, s->U[j], KRP_PINV_FALLBACK, sumsq);
        if (st != KRP_OK) return st;
        const int64_t g2 = std::min<int64_t>((s->I[j] + 7) / 8, (int64_t)s->num_sms * 8);
        col_scale<<<(unsigned)g2, 256, 0, s->stream>>>(s->U[j], s->I[j], R, sumsq, sigma); count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_check(s, e, "normalise launch");
        st = build_tree(s, j, s->prec);
        if (st != KRP_OK) return st;
        s->has_factor[j] = 1;
    }
    return KRP_OK;
}

extern "C" krp_status krp_cp_fit(krp_sampler* s, const krp_sptensor* t, const float* sigma, double* fit_host) {
    if (!s || !t || !sigma || !fit_host) return s ? fail(s, KRP_EINVAL, "null argument") : KRP_EINVAL;
    if (t->N != s->N) return fail(s, KRP_EINVAL, "krp_cp_fit: tensor order differs");
    const int R = s->R, N = s->N;
    int32_t* idx;
    float *w, *SA;
    double* scratch;
    krp_status st = als_buffers(s, 1, &idx, &w, &SA, &scratch);
    if (st != KRP_OK) return st;
    double* inner = scratch + R;
    cudaMemsetAsync(inner, 0, sizeof(double), s->stream);
    FitParams P{};
    for (int k = 0; k < N; ++k) P.U[k] = s->U[k];
    P.coords = t->coords;
    P.vals = t->vals;
    P.sigma = sigma;
    P.nnz = t->nnz;
    P.N = N;
    P.R = R;
    P.out = inner;
    const int64_t g = std::min<int64_t>((t->nnz + 255) / 256, (int64_t)s->num_sms * 8);
    fit_inner<<<(unsigned)g, 256, 0, s->stream>>>(P); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "fit launch");
    std::vector<float> roots((size_t)N * s->Tp), sg(R);
    double in_h = 0.0;
    for (int k = 0; k < N; ++k)
        cudaMemcpyAsync(roots.data() + (size_t)k * s->Tp, s->tree[k], s->Tp * 4, cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(sg.data(), sigma, R * 4, cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(&in_h, inner, 8, cudaMemcpyDeviceToHost, s->stream);
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "fit sync");
    // ||T̃||² = σᵀ (⊛_k G_k) σ from the trees' roots
    double m2 = 0.0;
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b) {
            double g2 = (double)sg[a] * (double)sg[b];
            for (int k = 0; k < N; ++k)
                g2 *= (double)roots[(size_t)k * s->Tp + tri_index(std::min(a, b), std::max(a, b), R)];
            m2 += g2;
        }
    const double r2 = std::max(t->normT2 - 2.0 * in_h + m2, 0.0);
    *fit_host = 1.0 - sqrt(r2) / sqrt(t->normT2);
    return KRP_OK;
}
