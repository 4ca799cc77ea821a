// Node-major batched descent for 32 < R <= 128: the draws of the team kernel
// (the sampling loop of Alg. 2 with the loops exchanged as in App. A.6; Alg. 4
// on E_k and Z_k; Eqs. first_dist and second_conditional_dist) with the B
// samples of a CTA advanced through the trees level by level together.
//
// At each level the batch is grouped by the node its samples sit at (one warp
// sorts at most 32 (node, sample) keys); every distinct node is brought into
// shared memory once, by a bulk copy, and the masses of all its samples are
// formed from it.  The upper levels of Z_k and most of E_k (2R - 1 nodes in
// all) are shared by many samples and cost one fetch per CTA; deeper levels,
// one node per sample, stream through a D-stage ring of copies across the
// batch, so no sample waits alone on its own round trip.  One node is fetched
// per level (the left child's Gram; the right child's mass is the node's minus
// it), and leaves shared by several samples are fetched once as well.
//
// The whole CTA forms each mass: thread t owns float4 chunks t, t + 256, ...
// of the packed node and builds their weights w_p = h_i h_j (doubled off the
// diagonal) on the fly from the sample's vector in shared memory, so the batch
// is not limited by per-sample registers.  Decisions use FP32 unless tau lies
// within 1e-6 C of the cutoff, then the double-float CTA sum; tau, low and h
// are double-float; the leaf scan and the epilogue are the team kernel's.
// Every wait is bounded and agreed by the CTA before anyone acts on it.
#include "common.cuh"
#include "internal.h"

#include <math.h>

#include <algorithm>

namespace krp {
namespace {

constexpr int NM_THREADS = 256;
constexpr int NM_WARPS = NM_THREADS / 32;
constexpr int NM_BMAX = 32;   // samples per batch (one warp sorts them)
constexpr int NM_DMAX = 4;    // copies in flight
constexpr int NM_WAIT_TRIES = 1 << 16;

__device__ __forceinline__ uint32_t nm_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool nm_wait(uint64_t* m, uint32_t parity) {
    for (int it = 0; it < NM_WAIT_TRIES; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(nm_saddr(m)), "r"(parity), "r"(100000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Per-sample state of the batch (shared memory).
struct NmSample {
    int64_t c;                  // node of the current tree (heap index)
    float low_hi, low_lo;       // left edge of the current node's interval
    float tau_hi, tau_lo;       // target u * C
    float mnode;                // mass of the current node
    float cf, margin;           // stage total C and 1e-6 C
    float ue, ur;               // the factor's two uniforms
    int u;                      // eigencomponent drawn for the factor
    int ok;                     // still drawing (0: beyond J, or a zero / non-finite mass)
};

template <int RMAX>
struct NmCfg {
    static constexpr int TPMAX = ((RMAX * (RMAX + 1) / 2) + 7) & ~7;
    static constexpr int NCH = (TPMAX / 4 + NM_THREADS - 1) / NM_THREADS;   // float4 chunks per thread
    static constexpr int RPT = (4 * RMAX + NM_THREADS - 1) / NM_THREADS;    // leaf rows per thread (F <= 4R)
};

// Shared-memory layout, in bytes from the (128-aligned) base.
struct NmLayout {
    int B, D, RS, stage_floats;
    size_t stages, hh, hl, th, smp, red, perm, gstart, gnode, misc, mbar, total;
};

__host__ __device__ inline NmLayout nm_layout(int B, int D, int RS, int stage_floats) {
    NmLayout L;
    L.B = B;
    L.D = D;
    L.RS = RS;
    L.stage_floats = stage_floats;
    size_t o = 0;
    L.stages = o;
    o += (size_t)D * stage_floats * 4;
    L.hh = o;
    o += (size_t)B * RS * 4;
    L.hl = o;
    o += (size_t)B * RS * 4;
    L.th = o;
    o += (size_t)B * RS * 4;
    o = (o + 15) & ~(size_t)15;
    L.smp = o;
    o += (size_t)B * sizeof(NmSample);
    o = (o + 15) & ~(size_t)15;
    L.red = o;                   // 4 floats per warp
    o += (size_t)NM_WARPS * 4 * 4;
    L.perm = o;                  // B ints
    o += (size_t)NM_BMAX * 4;
    L.gstart = o;                // B + 1 ints
    o += (size_t)(NM_BMAX + 1) * 4;
    o = (o + 7) & ~(size_t)7;
    L.gnode = o;                 // B int64
    o += (size_t)NM_BMAX * 8;
    L.misc = o;                  // ngroups, pick[2]
    o += 16;
    o = (o + 7) & ~(size_t)7;
    L.mbar = o;
    o += (size_t)NM_DMAX * 8;
    L.total = (o + 127) & ~(size_t)127;
    return L;
}

template <int RMAX>
__global__ void __launch_bounds__(NM_THREADS, 2)
    krp_descent_nm(const __grid_constant__ FastParams P, int B, int D, int RS, int stage_floats) {
    using C = NmCfg<RMAX>;
    constexpr int NCH = C::NCH;
    extern __shared__ __align__(128) unsigned char smem[];
    const NmLayout Ly = nm_layout(B, D, RS, stage_floats);
    float* stages = reinterpret_cast<float*>(smem + Ly.stages);
    float* hh = reinterpret_cast<float*>(smem + Ly.hh);
    float* hl = reinterpret_cast<float*>(smem + Ly.hl);
    float* th = reinterpret_cast<float*>(smem + Ly.th);
    NmSample* smp = reinterpret_cast<NmSample*>(smem + Ly.smp);
    float* red = reinterpret_cast<float*>(smem + Ly.red);
    int* perm = reinterpret_cast<int*>(smem + Ly.perm);
    int* gstart = reinterpret_cast<int*>(smem + Ly.gstart);
    int64_t* gnode = reinterpret_cast<int64_t*>(smem + Ly.gnode);
    int* misc = reinterpret_cast<int*>(smem + Ly.misc);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + Ly.mbar);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = P.R, T = P.T, Tp = P.Tp;
    const int nc4 = Tp >> 2;

    // (i, j) of the first packed entry of each of this thread's chunks
    constexpr int NIJ = (NCH + 1) / 2;
    uint32_t ij[NIJ];
#pragma unroll
    for (int h = 0; h < NIJ; ++h) ij[h] = 0u;
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
        const int p = 4 * (tid + NM_THREADS * m);
        int i = 0, rem = p;
        if (p < T)
            while (rem >= R - i) {
                rem -= R - i;
                ++i;
            }
        const uint32_t code = p < T ? (uint32_t)(i | ((i + rem) << 8)) : 0u;
        ij[m >> 1] |= code << (16 * (m & 1));
    }
    if (tid == 0) {
        for (int d = 0; d < D; ++d)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(nm_saddr(&mbar[d])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ---------------------------------------------------------------- helpers
    // CTA sums, identical in every thread (fixed order over the warps)
    auto cta_sum = [&](float v) -> float {
        v = warp_sum(v);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < NM_WARPS; ++w) t += red[w];
        __syncthreads();
        return t;
    };
    auto cta_sum_df = [&](float part) -> df {
        const df v = warp_sum_df(df{part, 0.f});
        if (lane == 0) {
            red[2 * warp] = v.hi;
            red[2 * warp + 1] = v.lo;
        }
        __syncthreads();
        df t{0.f, 0.f};
#pragma unroll
        for (int w = 0; w < NM_WARPS; ++w) t = df_add(t, df{red[2 * w], red[2 * w + 1]});
        __syncthreads();
        return t;
    };
    // this thread's part of xᵀ G x for the packed node G (weights from x on the fly)
    auto partial = [&](const float* node, const float* x) -> float {
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c = tid + NM_THREADS * m;
            if (c < nc4) {
                const uint32_t code = (ij[m >> 1] >> (16 * (m & 1))) & 0xFFFFu;
                int i = code & 0xFF, j = code >> 8;
                const int p0 = 4 * c;
                float wv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float w = 0.f;
                    if (p0 + q < T) {
                        w = x[i] * x[j];
                        if (i != j) w += w;
                    }
                    wv[q] = w;
                    if (++j == R) j = ++i;
                }
                const float4 v = reinterpret_cast<const float4*>(node)[c];
                a0 = ffma2(make_float2(wv[0], wv[1]), make_float2(v.x, v.y), a0);
                a1 = ffma2(make_float2(wv[2], wv[3]), make_float2(v.z, v.w), a1);
            }
        }
        return (a0.x + a1.x) + (a0.y + a1.y);
    };

    // ring of copies: item n uses stage n % D with parity (n / D) & 1
    uint64_t consumed = 0;      // uniform
    uint64_t issued = 0;        // thread 0's count
    bool alive = true;
    auto issue = [&](uint64_t n, const float* src, uint32_t bytes) {
        uint64_t* b = &mbar[n % D];
        float* dst = stages + (size_t)(n % D) * stage_floats;
        if (bytes) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(nm_saddr(b)), "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    nm_saddr(dst)),
                "l"(src), "r"(bytes), "r"(nm_saddr(b))
                : "memory");
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(nm_saddr(b)) : "memory");
        }
        issued = n + 1;
    };
    // wait for item n (every thread; the CTA agrees on the outcome)
    auto take = [&](uint64_t n) -> bool {
        const bool ok = nm_wait(&mbar[n % D], (uint32_t)((n / D) & 1));
        if (!__syncthreads_and(ok)) {
            if (tid == 0) set_status(P.status, KRP_ETIMEOUT);
            alive = false;
            return false;
        }
        consumed = n + 1;
        return true;
    };

    // group the batch's live samples by key (node), ascending: perm[] holds the
    // samples in key order, groups g = [gstart[g], gstart[g+1]) with key gnode[g]
    auto group = [&](int nb) -> int {
        if (warp == 0) {
            const bool live = lane < nb && smp[lane].ok;
            uint64_t key = live ? (((uint64_t)smp[lane].c) << 6) | (uint64_t)lane : ~0ull;
            // bitonic sort of 32 keys across the warp
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)key, jj);
                    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(key >> 32), jj);
                    const uint64_t other = ((uint64_t)hi << 32) | lo;
                    const bool up = (lane & k) == 0;
                    const bool lower = (lane & jj) == 0;
                    const uint64_t mn = key < other ? key : other, mx = key < other ? other : key;
                    key = (lower == up) ? mn : mx;
                }
            }
            const bool valid = key != ~0ull;
            const int64_t node = (int64_t)(key >> 6);
            const int64_t prev_node = (int64_t)(((uint64_t)__shfl_up_sync(0xffffffffu, (uint32_t)(key >> 32), 1) << 32 |
                                                 __shfl_up_sync(0xffffffffu, (uint32_t)key, 1)) >> 6);
            const bool start = valid && (lane == 0 || prev_node != node);
            const uint32_t starts = __ballot_sync(0xffffffffu, start);
            const int nvalid = __popc(__ballot_sync(0xffffffffu, valid));
            if (valid) perm[lane] = (int)(key & 63u);
            if (start) {
                const int g = __popc(starts & ((1u << lane) - 1u));
                gstart[g] = lane;
                gnode[g] = node;
            }
            if (lane == 0) {
                const int ng = __popc(starts);
                gstart[ng] = nvalid;
                misc[0] = ng;
            }
        }
        __syncthreads();
        return misc[0];
    };

    // One stage of Alg. 4 for the batch on tree `tr` (depth levels below the
    // root, Lk leaves, nreal real rows in bins of F); use_row picks the
    // uniform; sg the trace slot.  On return smp[s].c is each live sample's
    // leaf (heap index) and low its left edge.
    auto descend = [&](const float* __restrict__ tr, int depth, int64_t Lk, int64_t nreal, int F, bool use_row,
                       int sg, int64_t b0, int pi, int nb) {
        for (int s = tid; s < nb; s += NM_THREADS) smp[s].c = 1;
        __syncthreads();
        for (int lvl = -1; lvl < depth && alive; ++lvl) {
            const int ng = group(nb);
            if (ng == 0) break;
            const uint64_t base = consumed;
            if (tid == 0)
                for (int g = 0; g < ng && g < D; ++g)
                    issue(base + g, tr + (lvl < 0 ? 0 : gnode[g]) * (int64_t)Tp, (uint32_t)Tp * 4u);
            for (int g = 0; g < ng; ++g) {
                if (!take(base + g)) return;
                const float* node = stages + (size_t)((base + g) % D) * stage_floats;
                for (int q = gstart[g]; q < gstart[g + 1]; ++q) {
                    const int s = perm[q];
                    NmSample& S = smp[s];
                    const float part = partial(node, th + (size_t)s * RS);
                    const int64_t sglob = b0 + s;
                    float* trc = (P.trace && sglob < P.n_trace && tid == 0)
                                     ? P.trace + ((sglob * P.n_incl + pi) * 2 + sg) * 66
                                     : nullptr;
                    if (lvl < 0) {          // the stage total C
                        const df Cm = cta_sum_df(part);
                        const float cf = Cm.hi + Cm.lo;
                        if (tid == 0) {
                            if (!(cf > 0.f) || !isfinite(cf)) {
                                set_status(P.status, isfinite(cf) ? KRP_EZERO : KRP_ENUMERIC);
                                S.ok = 0;
                            } else {
                                const df tau = df_mul_f(Cm, use_row ? S.ur : S.ue);
                                S.tau_hi = tau.hi;
                                S.tau_lo = tau.lo;
                                S.low_hi = S.low_lo = 0.f;
                                S.cf = cf;
                                S.margin = 1e-6f * cf;
                                S.mnode = cf;
                            }
                            if (trc) trc[0] = cf;
                        }
                    } else {
                        // the state is read before the CTA sum, whose barriers
                        // order these reads before thread 0's update below
                        const int64_t c = S.c;
                        const df tau{S.tau_hi, S.tau_lo}, low{S.low_hi, S.low_lo};
                        const float mnode = S.mnode, margin = S.margin;
                        const float mA = cta_sum(part);
                        const int64_t rfirst = ((2 * c + 1) << (depth - lvl - 1)) - Lk;
                        bool left = rfirst * F >= nreal;
                        df cut{0.f, 0.f};
                        if (!left) {
                            // tau, low and mA are CTA-uniform: so is the branch into the df sum
                            const float gapf = (tau.hi - low.hi) - mA;
                            if (fabsf(gapf) > margin) {
                                left = gapf < 0.f;
                                if (!left) cut = df_add(low, df{mA, 0.f});
                            } else {
                                cut = df_add(low, cta_sum_df(part));
                                left = df_le(tau, cut);
                            }
                        }
                        if (tid == 0) {
                            if (trc) {
                                trc[2 + 2 * lvl] = mA;
                                trc[3 + 2 * lvl] = mnode;
                            }
                            if (left) {
                                S.c = 2 * c;
                                S.mnode = mA;
                            } else {
                                S.c = 2 * c + 1;
                                S.low_hi = cut.hi;
                                S.low_lo = cut.lo;
                                S.mnode = mnode - mA;
                            }
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();   // the stage and every sample's state are settled
                if (tid == 0 && g + D < ng)
                    issue(base + g + D, tr + (lvl < 0 ? 0 : gnode[g + D]) * (int64_t)Tp, (uint32_t)Tp * 4u);
            }
        }
    };

    // leaf blocks by bulk copy when every block starts on a 16-byte boundary
    const bool leaf_tma = ((int64_t)P.F * R) % 4 == 0 && (int64_t)P.F * R <= stage_floats;
    const int64_t batches = (P.J + B - 1) / B;
    for (int64_t bt = blockIdx.x; bt < batches && alive; bt += gridDim.x) {
        const int64_t b0 = bt * B;
        const int nb = (int)min((int64_t)B, P.J - b0);
        for (int e = tid; e < B * RS; e += NM_THREADS) {
            const int s = e / RS, a = e - s * RS;
            hh[e] = (s < nb && a < R) ? 1.f : 0.f;
            hl[e] = 0.f;
        }
        for (int s = tid; s < B; s += NM_THREADS) smp[s].ok = s < nb ? 1 : 0;
        __syncthreads();
        for (int pi = 0; pi < P.n_incl && alive; ++pi) {
            const int k = P.incl[pi];
            for (int s = tid; s < nb; s += NM_THREADS) {
                const uint4 rnd = philox4x32_10(make_uint4((uint32_t)(b0 + s), P.draw, (uint32_t)pi, 0u),
                                                make_uint2(P.key0, P.key1));
                smp[s].ue = u32_to_unit(rnd.x);
                smp[s].ur = u32_to_unit(rnd.y);
            }
            // ---------------------------------------------- u-stage on E_k
            for (int e = tid; e < nb * RS; e += NM_THREADS) th[e] = hh[e] + hl[e];
            __syncthreads();
            descend(P.etree[k], P.dE, P.Rp, R, 1, false, 0, b0, pi, nb);
            if (!alive) break;
            for (int s = tid; s < nb; s += NM_THREADS) smp[s].u = (int)(smp[s].c - P.Rp);
            __syncthreads();
            // ---------------------------------------------- t-stage on Z_k
            for (int e = tid; e < nb * RS; e += NM_THREADS) {
                const int s = e / RS, a = e - s * RS;
                float v = 0.f;
                if (a < R && smp[s].ok) {
                    const int u = smp[s].u;
                    const float vh = __ldg(P.Vhi[k] + (size_t)u * R + a), vl = __ldg(P.Vlo[k] + (size_t)u * R + a);
                    const df t = df_add(df_mul_f(df{hh[e], hl[e]}, vh), df_mul_f(df{hh[e], hl[e]}, vl));
                    v = t.hi + t.lo;   // h̃ = h ∘ V[:,u], rounded once
                }
                th[e] = v;
            }
            __syncthreads();
            const int64_t Lk = P.L[k], Ik = P.I[k];
            const int F = P.F;
            descend(P.tree[k], P.depth[k], Lk, Ik, F, true, 1, b0, pi, nb);
            if (!alive) break;
            // ---------------------------------------------- leaf scans, grouped by leaf
            const float* Uk = P.U[k];
            const int ng = group(nb);
            const uint64_t base = consumed;
            auto leaf_issue = [&](int g) {
                const int64_t row0 = (gnode[g] - Lk) * F;
                const int nrows = (int)min((int64_t)F, Ik - row0);
                const uint32_t bytes = leaf_tma ? ((uint32_t)nrows * (uint32_t)R * 4u) & ~15u : 0u;
                issue(base + g, Uk + row0 * R, bytes);
            };
            if (tid == 0)
                for (int g = 0; g < ng && g < D; ++g) leaf_issue(g);
            for (int g = 0; g < ng && alive; ++g) {
                if (!take(base + g)) break;
                float* blk = stages + (size_t)((base + g) % D) * stage_floats;
                const int64_t row0 = (gnode[g] - Lk) * F;
                const int nrows = (int)min((int64_t)F, Ik - row0);
                const int nval = nrows * R;
                const int from = leaf_tma ? nval & ~3 : 0;   // what the copy did not bring
                for (int e = from + tid; e < nval; e += NM_THREADS) blk[e] = Uk[row0 * R + e];
                if (from < nval) __syncthreads();
                const int rpt = (F + NM_THREADS - 1) / NM_THREADS;
                for (int q = gstart[g]; q < gstart[g + 1]; ++q) {
                    const int s = perm[q];
                    NmSample& S = smp[s];
                    const float* x = th + (size_t)s * RS;
                    float qv[C::RPT];
                    float run = 0.f;
#pragma unroll
                    for (int r = 0; r < C::RPT; ++r) {
                        const int t = tid * rpt + r;
                        float d = 0.f;
                        if (r < rpt && t < nrows) {
                            const float* row = blk + (size_t)t * R;
                            // rows start on rotated columns: thread t reads bank (t (R + 1) + n) mod 32
                            int a = t % R, n = 0;
                            float d0 = 0.f, d1 = 0.f;
                            for (; n + 1 < R; n += 2) {
                                d0 = fmaf(row[a], x[a], d0);
                                a = a + 1 == R ? 0 : a + 1;
                                d1 = fmaf(row[a], x[a], d1);
                                a = a + 1 == R ? 0 : a + 1;
                            }
                            if (n < R) d0 = fmaf(row[a], x[a], d0);
                            d = d0 + d1;
                        }
                        qv[r] = (r < rpt && t < nrows) ? d * d : 0.f;
                        run += qv[r];
                    }
                    // exclusive scan of the per-thread totals over the CTA (FP32)
                    float inc = run;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const float v = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += v;
                    }
                    float cum = __shfl_up_sync(0xffffffffu, inc, 1);
                    if (lane == 0) cum = 0.f;
                    if (lane == 31) red[warp] = inc;
                    __syncthreads();
                    float off = 0.f;
                    for (int w = 0; w < warp; ++w) off += red[w];
                    cum += off;
                    __syncthreads();
                    const df tau{S.tau_hi, S.tau_lo}, low{S.low_hi, S.low_lo};
                    const df rel = df_add(tau, df_neg(low));
                    const float target = rel.hi + rel.lo, margin = S.margin;
                    int first = 0x7fffffff, lastpos = -1;
                    bool near = false;
#pragma unroll
                    for (int r = 0; r < C::RPT; ++r) {
                        const int t = tid * rpt + r;
                        if (r < rpt && t < nrows) {
                            cum += qv[r];
                            if (first == 0x7fffffff && target <= cum) first = t;
                            if (fabsf(cum - target) <= margin) near = true;
                            if (qv[r] > 0.f) lastpos = t;
                        }
                    }
                    if (__syncthreads_or(near)) {
                        // redo the scan in double-float: edges low + cumulative weights
                        df acc{0.f, 0.f};
#pragma unroll
                        for (int r = 0; r < C::RPT; ++r) acc = df_add(acc, df{qv[r], 0.f});
                        df incd = acc;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const float vh = __shfl_up_sync(0xffffffffu, incd.hi, o);
                            const float vl = __shfl_up_sync(0xffffffffu, incd.lo, o);
                            if (lane >= o) incd = df_add(df{vh, vl}, incd);
                        }
                        df cd{__shfl_up_sync(0xffffffffu, incd.hi, 1), __shfl_up_sync(0xffffffffu, incd.lo, 1)};
                        if (lane == 0) cd = df{0.f, 0.f};
                        if (lane == 31) {
                            red[2 * warp] = incd.hi;
                            red[2 * warp + 1] = incd.lo;
                        }
                        __syncthreads();
                        df offd{0.f, 0.f};
                        for (int w = 0; w < warp; ++w) offd = df_add(offd, df{red[2 * w], red[2 * w + 1]});
                        cd = df_add(offd, cd);
                        __syncthreads();
                        cd = df_add(cd, low);
                        first = 0x7fffffff;
#pragma unroll
                        for (int r = 0; r < C::RPT; ++r) {
                            const int t = tid * rpt + r;
                            if (r < rpt && t < nrows) {
                                cd = df_add(cd, df{qv[r], 0.f});
                                if (first == 0x7fffffff && df_le(tau, cd)) first = t;
                            }
                        }
                    }
#pragma unroll
                    for (int m = 16; m > 0; m >>= 1) {
                        first = min(first, __shfl_xor_sync(0xffffffffu, first, m));
                        lastpos = max(lastpos, __shfl_xor_sync(0xffffffffu, lastpos, m));
                    }
                    if (lane == 0) {
                        red[2 * warp] = __int_as_float(first);
                        red[2 * warp + 1] = __int_as_float(lastpos);
                    }
                    __syncthreads();
                    first = 0x7fffffff;
                    lastpos = -1;
#pragma unroll
                    for (int w = 0; w < NM_WARPS; ++w) {
                        first = min(first, __float_as_int(red[2 * w]));
                        lastpos = max(lastpos, __float_as_int(red[2 * w + 1]));
                    }
                    int t_sel = first != 0x7fffffff ? first : lastpos;
                    if (t_sel < 0) {   // no positive weight in the leaf: only through rounding
                        if (tid == 0) set_status(P.status, KRP_ENUMERIC);
                        t_sel = 0;
                    }
                    float* hs = hh + (size_t)s * RS;
                    float* ls = hl + (size_t)s * RS;
                    for (int a = tid; a < R; a += NM_THREADS) {
                        const df nh = df_mul_f(df{hs[a], ls[a]}, blk[(size_t)t_sel * R + a]);
                        hs[a] = nh.hi;
                        ls[a] = nh.lo;
                    }
                    if (tid == 0) P.idx[(int64_t)k * P.J + b0 + s] = (int32_t)(row0 + t_sel);
                    __syncthreads();
                }
                // the tail's plain stores precede the next copy into this stage
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0 && g + D < ng) leaf_issue(g + D);
            }
        }
        if (!alive) break;
        // -------------------------------------------------- epilogue per sample
        for (int e = tid; e < nb * RS; e += NM_THREADS) th[e] = hh[e] + hl[e];
        __syncthreads();
        const int gexp = P.rank[1];
        const float rk = (float)P.rank[0];
        for (int s = 0; s < nb; ++s) {
            const float* x = th + (size_t)s * RS;
            float part = 0.f;
#pragma unroll
            for (int m = 0; m < NCH; ++m) {
                const int c = tid + NM_THREADS * m;
                if (c < nc4) {
                    const uint32_t code = (ij[m >> 1] >> (16 * (m & 1))) & 0xFFFFu;
                    int i = code & 0xFF, j = code >> 8;
                    const int p0 = 4 * c;
                    const float4 v = __ldg(reinterpret_cast<const float4*>(P.Gplus32) + c);
                    const float g4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (p0 + q < T) {
                            float w = x[i] * x[j];
                            if (i != j) w += w;
                            part = fmaf(w, g4[q], part);
                        }
                        if (++j == R) j = ++i;
                    }
                }
            }
            // q_s = ℓ_s / rank, ℓ_s = hᵀG⁺h = lv 2^gexp (G⁺ stored scaled by 2^-gexp)
            const df lev = cta_sum_df(part);
            const bool ok = smp[s].ok != 0;
            const float lv = (lev.hi + lev.lo) / rk;
            const float w = ok ? ldexpf(1.0f / sqrtf((float)P.J * lv * ((gexp & 1) ? 2.f : 1.f)), -(gexp >> 1)) : 0.f;
            const int64_t sg = b0 + s;
            if (tid == 0) {
                P.weight[sg] = w;
                if (P.logq) P.logq[sg] = ok ? logf(lv) + (float)gexp * 0.6931471805599453f : -INFINITY;
            }
            if (P.SA)
                for (int a = tid; a < R; a += NM_THREADS) P.SA[sg * R + a] = w * x[a];
        }
        __syncthreads();
    }
    if (!alive && tid == 0) {
        // let copies still in flight into this CTA's shared memory land (bounded)
        for (uint64_t n = consumed; n < issued; ++n) nm_wait(&mbar[n % D], (uint32_t)((n / D) & 1));
    }
}

template <int RMAX>
cudaError_t launch_nm_t(const FastParams& P, int B, int D, int RS, int stage_floats, size_t smem, int per_sm,
                        int num_sms, cudaStream_t st) {
    auto k = krp_descent_nm<RMAX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const int64_t batches = (P.J + B - 1) / B;
    const int64_t grid = std::min<int64_t>(batches, (int64_t)per_sm * num_sms);
    k<<<(unsigned)grid, NM_THREADS, smem, st>>>(P, B, D, RS, stage_floats);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

// The node-major form for 32 < R <= 128; false if R is outside it or its
// smallest batch does not fit the shared memory.  Batch size B and ring depth
// D: the largest (B, D) with two CTAs per SM, else with one.
bool launch_descent_nm(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                       float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err) {
    const int R = s->R;
    if (R <= 32 || R > 128) return false;
    const int RS = (R + 3) & ~3;
    // a stage holds a node or a whole leaf block (by copy or by plain loads)
    const int64_t stage = std::max<int64_t>(s->Tp, (int64_t)s->F * R);
    const int stage_floats = (int)((stage + 31) / 32 * 32);
    const size_t per_sm_bytes = 227 * 1024;   // shared memory a block may use
    int B = 0, D = 0, per_sm = 0;
    const int Bs[3] = {32, 24, 16};
    for (int want = 2; want >= 1 && !B; --want)
        for (int bi = 0; bi < 3 && !B; ++bi)
            for (int d = 3; d >= 2 && !B; --d) {
                const size_t need = nm_layout(Bs[bi], d, RS, stage_floats).total;
                if ((need + 1024) * want <= 228 * 1024 && need <= per_sm_bytes) {
                    B = Bs[bi];
                    D = d;
                    per_sm = want;
                }
            }
    if (!B) return false;
    FastParams P;
    fast_params_for(s, exclude_j, &P);
    P.key0 = (uint32_t)(seed & 0xffffffffu);
    P.key1 = (uint32_t)(seed >> 32);
    P.draw = (uint32_t)(draw_id & 0xffffffffu);
    P.J = J;
    P.idx = idx;
    P.weight = weight;
    P.logq = logq;
    P.SA = SA;
    P.trace = trace;
    P.n_trace = trace ? n_trace : 0;
    const size_t smem = nm_layout(B, D, RS, stage_floats).total;
    *err = R <= 64 ? launch_nm_t<64>(P, B, D, RS, stage_floats, smem, per_sm, s->num_sms, s->stream)
                   : launch_nm_t<128>(P, B, D, RS, stage_floats, smem, per_sm, s->num_sms, s->stream);
    return true;
}

}  // namespace krp
