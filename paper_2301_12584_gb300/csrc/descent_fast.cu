// a4 + a5 (+ a6 fused) for R <= 32: the batched conditional descent with one
// warp per sample (the sampling loop of Alg. 2, loops exchanged as in App. A.6; Alg. 4
// on E_k and Z_k; Eqs. first_dist and second_conditional_dist).
//
// Per level the mass m(v) = wᵀ g over the packed upper triangle g of the
// node's partial Gram, with w_p = h_i h_j (x2 off the diagonal) for the
// history vector h of the stage (h for E_k, h̃ = h ∘ V[:,u] for Z_k).  The
// warp keeps w in shared memory as float4 chunks; each lane owns chunks
// lane + 32 m.
//
// Two levels per memory round trip: at node c the masses of slot c (left
// child of c), slot 2c (left child of 2c) and slot 2c+1 (left child of 2c+1)
// are loaded together (slots 2c and 2c+1 are adjacent), which decides levels
// l and l+1 — the second with whichever of the two it needs.
//
// Precision: masses are summed per lane in FP32 and across the warp in
// double-float; the target tau = u * C, the running offset low and every
// cutoff low + m(L(c)) are double-float, and so are h and h̃ (products of
// FP32 rows and FP64 eigenvectors), so that a branch differs from an FP64
// evaluation only when tau lies within ~1e-7 C of a cutoff.
//
// Exact-decision mode (EXACT, KRP_PREC_EXACT): the row stage starts from the
// double-float root (C and tau to ~2^-44), takes the top levels from the
// delta-encoded slots D_c = G_{2c} - alpha_c G_c (m(L(c)) = alpha_c m(c) +
// wᵀD_c, whose FP32 error is that of the small deviation wᵀD_c), carries a
// running bound on the FP32 path's error, and re-takes any decision whose gap
// tau - low - m(L(c)) falls within that bound plus KRP_EXACT_BAND C from
// double-float masses of the (hi, lo) slots with double-float weights of h̃:
// the offset low is then recomputed from the path's right turns, and the
// stage stays in that form to its leaf, whose rows are rescored in
// double-float when the FP32 scan is near an edge.  The eigencomponent stage
// (R bins) keeps the FP32 form.
#include "common.cuh"
#include "internal.h"

#include <math.h>

// The exact-decision kernels are built in a translation unit of their own
// (descent_exact.cu sets KRP_DESCENT_EXACT_TU and includes this file), so
// that their code stays out of the FP32 kernels' unit.
#ifndef KRP_DESCENT_EXACT_TU
#define KRP_DESCENT_EXACT_TU 0
#endif

namespace krp {


constexpr int FAST_TRACE_STRIDE = 66;

// X: exact-decision samplers, whose node slots carry one more float (a bound
// for the node's masses) after the packed triangle.
template <int RMAX, bool X = false>
struct FastCfg {
    static constexpr int TPMAX = ((RMAX * (RMAX + 1) / 2) + (X ? 1 : 0) + 7) & ~7;
    static constexpr int NC4 = TPMAX / 4;           // float4 chunks per node
    static constexpr int NCH = (NC4 + 31) / 32;     // chunks per lane
    static constexpr int WARPS = X ? 4 : 8;   // exact-decision kernels: more, smaller CTAs
    static constexpr int RPT = (4 * RMAX + 31) / 32;  // leaf rows per lane (F <= 4R)
    // per-warp shared memory: 3 staged nodes (slots 0..1 on a stage's first
    // fetch, then slots c, 2c, 2c+1; also the leaf rows), h (hi, lo), h̃ (hi,
    // lo), mbarrier
    static constexpr int STAGE = 3 * TPMAX;
    static constexpr int WARP_BYTES = ((STAGE + 4 * RMAX) * 4 + 16 + 127) & ~127;
    static constexpr int SMEM = WARPS * WARP_BYTES + 2 * TPMAX;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* m) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}
// Bounded wait for the mbarrier phase `parity`; false if it did not complete.
// Each try_wait may suspend the warp for up to ~0.1 ms (the hint), so the
// loop spins little; 1<<16 tries bound the wait to a few seconds.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, int max_tries = 1 << 16) {
    for (int it = 0; it < max_tries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(m)), "r"(parity), "r"(100000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

#if KRP_DESCENT_EXACT_TU
// Exact-decision mode: mass h̃ᵀ G h̃ of a node from its double-float slot (ghi,
// glo: shared or global) with double-float weights of h̃ = (th, thl), ~2^-44
// relative; every lane of the warp calls it and gets the same value.  It
// serves the rare near-edge decisions, so its loops stay rolled: inlined in
// the descent it then adds little to the loop's instruction footprint.
template <int NCH>
__device__ __forceinline__ df exact_mass_fn(const float* ghi, const float* glo, const float* th, const float* thl,
                                         const uint8_t* s_i, const uint8_t* s_j, int T, int nc4) {
    const int lane = threadIdx.x & 31;
    df acc{0.f, 0.f};
#pragma unroll 1
    for (int m = 0; m < NCH; ++m) {
        const int c4 = lane + 32 * m;
        if (c4 < nc4) {
            const float4 h4 = reinterpret_cast<const float4*>(ghi)[c4];
            const float4 l4 = reinterpret_cast<const float4*>(glo)[c4];
            const float gh[4] = {h4.x, h4.y, h4.z, h4.w}, gl[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                const int p = 4 * c4 + q;
                if (p < T) {
                    const int i = s_i[p], j = s_j[p];
                    df w = two_prod(th[i], th[j]);
                    w.lo = fmaf(th[i], thl[j], fmaf(thl[i], th[j], w.lo));
                    if (i != j) {
                        w.hi += w.hi;
                        w.lo += w.lo;
                    }
                    df t = two_prod(w.hi, gh[q]);
                    t.lo = fmaf(w.hi, gl[q], fmaf(w.lo, gh[q], t.lo));
                    acc = df_add(acc, t);
                }
            }
        }
    }
    return warp_sum_df(acc);
}
// Exact-decision mode: a leaf scan re-taken in double-float, every lane
// calling with its rows t = lane rpt + r of the leaf (rows: nrows rows of R
// floats, shared or global): q_t = (U[t] · h̃)^2 with h̃ = (th, thl),
// cumulative right edges from low.  Returns this lane's first row of positive
// weight whose edge reaches tau (0x7fffffff if none) and its last row of
// positive weight (-1); near_low: some edge lies within mlow of tau.
template <int RPT>
__device__ __forceinline__ int2 exact_leaf_scan(const float* rows, int R, int rpt, int nrows, const float* th,
                                             const float* thl, df tau, df low, float mlow, bool& near_low) {
    const int lane = threadIdx.x & 31;
    df qd[RPT];
#pragma unroll 1
    for (int r = 0; r < RPT; ++r) {
        const int t = lane * rpt + r;
        df d{0.f, 0.f};
        if (r < rpt && t < nrows) {
            const float* row = rows + t * R;
            for (int a = 0; a < R; ++a) {
                const float x = row[a];
                df pr = two_prod(x, th[a]);
                pr.lo = fmaf(x, thl[a], pr.lo);
                d = df_add(d, pr);
            }
        }
        qd[r] = df_mul(d, d);
    }
    df acc{0.f, 0.f};
#pragma unroll 1
    for (int r = 0; r < RPT; ++r)
        if (r < rpt && lane * rpt + r < nrows) acc = df_add(acc, qd[r]);
    df incd = acc;
#pragma unroll 1
    for (int o = 1; o < 32; o <<= 1) {
        const float vh = __shfl_up_sync(0xffffffffu, incd.hi, o);
        const float vl = __shfl_up_sync(0xffffffffu, incd.lo, o);
        if (lane >= o) incd = df_add(df{vh, vl}, incd);
    }
    df cd{__shfl_up_sync(0xffffffffu, incd.hi, 1), __shfl_up_sync(0xffffffffu, incd.lo, 1)};
    if (lane == 0) cd = df{0.f, 0.f};
    cd = df_add(cd, low);
    int first = 0x7fffffff, lastpos = -1;
    bool nl = false;
#pragma unroll 1
    for (int r = 0; r < RPT; ++r) {
        const int t = lane * rpt + r;
        if (r < rpt && t < nrows) {
            cd = df_add(cd, qd[r]);
            if (first == 0x7fffffff && qd[r].hi > 0.f && df_le(tau, cd)) first = t;
            if (qd[r].hi > 0.f) lastpos = t;
            if (fabsf(df_add(cd, df_neg(tau)).hi) <= mlow) nl = true;
        }
    }
    near_low = __any_sync(0xffffffffu, nl);
    return make_int2(first, lastpos);
}

#endif  // KRP_DESCENT_EXACT_TU

// The descent for samples cta*8 + warp, stepping by ncta*8 (ncta CTAs share
// the J samples of one problem).  P may live in parameter or shared memory.
// TRACE (exact-decision kernels): the instantiation that records traces; the
// others carry no tracing code.
template <int RMAX, bool EXACT = false, bool TRACE = false>
__device__ __forceinline__ void descent_fast_body(const FastParams& P, int64_t cta, int64_t ncta) {
    using C = FastCfg<RMAX, EXACT>;
    constexpr int NCH = C::NCH;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wbase = smem + warp * C::WARP_BYTES;
    float* stage = reinterpret_cast<float*>(wbase);                 // 3 x Tp (or leaf rows)
    float* hh = stage + C::STAGE;
    float* hl = hh + RMAX;
    float* th = hl + RMAX;
    float* thl = th + RMAX;   // h̃'s low parts (exact-decision mode)
    uint64_t* mbar = reinterpret_cast<uint64_t*>(thl + RMAX);
    uint8_t* s_i = smem + C::WARPS * C::WARP_BYTES;
    uint8_t* s_j = s_i + C::TPMAX;

    const int R = P.R, T = P.T, Tp = P.Tp;
    const int nc4 = Tp >> 2;
    for (int p = threadIdx.x; p < C::TPMAX; p += blockDim.x) {
        int i = 0, rem = p;
        if (p < T)
            while (rem >= R - i) {
                rem -= R - i;
                ++i;
            }
        s_i[p] = (uint8_t)(p < T ? i : 0);
        s_j[p] = (uint8_t)(p < T ? i + rem : 0);
    }
    if (lane == 0) {
        mbar_init(mbar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    bool alive = true;

    // Stage up to two contiguous global ranges into `stage` (bytes multiple of
    // 16): issue, then wait (bounded).
    auto fetch_issue = [&](const float* a, uint32_t abytes, const float* b, uint32_t bbytes) {
        __syncwarp();
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(mbar, abytes + bbytes);
            tma_load_1d(stage, a, abytes, mbar);
            if (bbytes) tma_load_1d(stage + Tp, b, bbytes, mbar);
        }
    };
    auto fetch_wait = [&]() -> bool {
        const bool ok = mbar_wait(mbar, phase);
        phase ^= 1u;
        if (!ok) {
            if (lane == 0) set_status(P.status, KRP_ETIMEOUT);
            alive = false;
        }
        return ok;
    };
    auto fetch = [&](const float* a, uint32_t abytes, const float* b, uint32_t bbytes) -> bool {
        fetch_issue(a, abytes, b, bbytes);
        return fetch_wait();
    };

    float4 w4[NCH];
    // weights of the packed entries for history vector x (smem, FP32)
    auto make_weights = [&](const float* x) {
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c = lane + 32 * m;
            float wv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int p = 4 * c + q;
                float w = 0.f;
                if (p < T) {
                    const int i = s_i[p], j = s_j[p];
                    w = x[i] * x[j];
                    if (i != j) w += w;
                }
                wv[q] = w;
            }
            w4[m] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
    };
    // lane partial of the mass of the staged node at `node` (smem)
    auto partial = [&](const float* node) -> float {
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c = lane + 32 * m;
            if (c < nc4) {
                const float4 v = reinterpret_cast<const float4*>(node)[c];
                a0 = ffma2(make_float2(w4[m].x, w4[m].y), make_float2(v.x, v.y), a0);
                a1 = ffma2(make_float2(w4[m].z, w4[m].w), make_float2(v.z, v.w), a1);
            }
        }
        return (a0.x + a1.x) + (a0.y + a1.y);
    };
    auto refine = [&](float part) -> df { return warp_sum_df(df{part, 0.f}); };
#if KRP_DESCENT_EXACT_TU
    // Exact-decision mode: bound on the error of a row weight q = d^2, d = U[t]
    // · h̃ an FP32 dot product over R terms with ab = sum_a |U[t]_a h̃_a|:
    // |d - d_exact| <= (R + 1) 2^-24 ab = dd (h̃ rounded to FP32 included), so
    // |q - d_exact^2| <= (2 |d| + dd) dd + 2^-24 q.
    auto row_err = [&](float d, float ab) -> float {
        const float dd = (float)(R + 1) * 5.9604644775390625e-8f * ab;
        return fmaf(fmaf(2.f, fabsf(d), dd), dd, 5.9604644775390625e-8f * d * d);
    };
#endif
    // Decision "tau <= low + m" (Alg. 4): FP32 when tau is more than `margin`
    // away from the cutoff, else the double-float mass.  (tau.hi - low.hi) - m
    // is within a few ulp(C) + |tau.lo| + |low.lo| < 3e-7 C of tau - low - m;
    // all three are warp-uniform, so the branch into the warp sum is too.
    auto go_left = [&](df tau, df low, float m, float part, float margin, df& cut) -> bool {
        const float gapf = (tau.hi - low.hi) - m;
        if (fabsf(gapf) > margin) {
            if (gapf < 0.f) return true;
            cut = df_add(low, df{m, 0.f});
            return false;
        }
        cut = df_add(low, refine(part));
        return df_le(tau, cut);
    };
    // One descent of Alg. 4 whose first fetch (slots 0 and 1, already issued)
    // holds the root and level 0.  Returns the leaf heap index; low is its left
    // edge; Cm the root mass; tau = u * Cm.
    auto descend = [&](const float* __restrict__ tr, int depth, int64_t Lk, int64_t nreal_rows, int F, float uu,
                       df& Cm, df& tau, df& low, float* trc) -> int64_t {
        low = df{0.f, 0.f};
        if (!fetch_wait()) return 1;
        const int nfirst = depth >= 1 ? 2 : 1;
        float pr[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) pr[q] = q < nfirst ? partial(stage + q * Tp) : 0.f;
        Cm = refine(pr[0]);
        const float cf = Cm.hi + Cm.lo;
        if (!(cf > 0.f) || !isfinite(cf)) return -1;
        tau = df_mul_f(Cm, uu);
        const float margin = 1e-6f * cf;
        if (trc) trc[0] = cf;
        int64_t c = 1;
        int lvl = 0;
        float mnode = cf;
        // level 0 from the first fetch
        float mA = depth >= 1 ? warp_sum(pr[1]) : 0.f, pA = pr[1];
        bool have_next = false;
        while (lvl < depth && alive) {
            if (lvl > 0) {
                // fetch slots c (level lvl) and 2c, 2c+1 (level lvl + 1) when two remain
                have_next = lvl + 2 <= depth;
                if (!fetch(tr + c * Tp, Tp * 4, have_next ? tr + 2 * c * Tp : nullptr, have_next ? 2 * Tp * 4 : 0))
                    break;
                pA = partial(stage);
                mA = warp_sum(pA);
            }
            bool left;
            {
                const int64_t rfirst = ((2 * c + 1) << (depth - lvl - 1)) - Lk;
                df cut;
                if (trc) {
                    trc[2 + 2 * lvl] = mA;
                    trc[3 + 2 * lvl] = mnode;
                }
                left = rfirst * F >= nreal_rows || go_left(tau, low, mA, pA, margin, cut);
                if (left) {
                    c = 2 * c;
                    mnode = mA;
                } else {
                    c = 2 * c + 1;
                    low = cut;
                    mnode = mnode - mA;
                }
                ++lvl;
            }
            if (!have_next) continue;
            // only the chosen child's left child is needed at the next level
            pA = partial(stage + (left ? Tp : 2 * Tp));
            mA = warp_sum(pA);
            {
                const int64_t rfirst = ((2 * c + 1) << (depth - lvl - 1)) - Lk;
                df cut;
                if (trc) {
                    trc[2 + 2 * lvl] = mA;
                    trc[3 + 2 * lvl] = mnode;
                }
                if (rfirst * F >= nreal_rows || go_left(tau, low, mA, pA, margin, cut)) {
                    c = 2 * c;
                    mnode = mA;
                } else {
                    c = 2 * c + 1;
                    low = cut;
                    mnode = mnode - mA;
                }
                ++lvl;
            }
        }
        return c;
    };

#if KRP_DESCENT_EXACT_TU
    // ---------------------------------------------- exact-decision mode
    // Double-float masses of a row stage's tree (tr, tl: hi and low parts) for
    // node c at depth lvl, by one rolled loop with a single inlined mass, so
    // that the rare exact path adds little to the descent's instruction
    // footprint.  what: 1 = the root (C), 2 = low (the left siblings of the
    // path's right turns; the left sibling of a right child n sits at slot
    // n/2), 4 = m(L(c)) (slot c).
    auto exact_pass = [&](const float* tr, const float* tl, int64_t c, int lvl, int what, df& Cx, df& lowx,
                          df& chx) {
        lowx = df{0.f, 0.f};
#pragma unroll 1
        for (int t = -1; t <= lvl; ++t) {
            int64_t slot = -1;
            if (t < 0) {
                if (what & 1) slot = 0;
            } else if (t < lvl) {
                const int64_t n = c >> (lvl - 1 - t);   // path node at depth t + 1
                if ((what & 2) && (n & 1)) slot = n >> 1;
            } else if (what & 4) {
                slot = c;
            }
            if (slot < 0) continue;   // warp-uniform
            const df m = exact_mass_fn<NCH>(tr + slot * Tp, tl + slot * Tp, th, thl, s_i, s_j, T, nc4);
            if (t < 0)
                Cx = m;
            else if (t < lvl)
                lowx = df_add(lowx, m);
            else
                chx = m;
        }
        if ((what & 2) && P.nexact && lane == 0) atomicAdd(P.nexact, 1ull);
    };
    // lane part of sum_p |w_p x_p| over the staged node x (bounds the FP32
    // mass's rounding error)
    auto abs_partial = [&](const float* node) -> float {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c4 = lane + 32 * m;
            if (c4 < nc4) {
                const float4 v = reinterpret_cast<const float4*>(node)[c4];
                acc = fmaf(fabsf(w4[m].x), fabsf(v.x), acc);
                acc = fmaf(fabsf(w4[m].y), fabsf(v.y), acc);
                acc = fmaf(fabsf(w4[m].z), fabsf(v.z), acc);
                acc = fmaf(fabsf(w4[m].w), fabsf(v.w), acc);
            }
        }
        return acc;
    };
    // Alg. 4 in the exact-decision mode, for both stages of a factor (one
    // code path, so that the loop's instruction footprint stays that of one
    // descent): the row stage on Z_k (tl: its low parts; dt: its delta-encoded
    // top, Ke levels) and the eigencomponent stage on E_k (tl null, Ke = 0:
    // near-edge decisions from double-float sums of the FP32 lane partials,
    // as in the FP32 form, since E_k has R leaves).  The first fetch (slots 0
    // and 1 of dt) is in flight.
    //
    // Error terms of the row stage.  An FP32 mass sum_p w_p x_p (weights from
    // h̃ rounded to FP32, x the stored slot, FP32 sums over a lane's chunks and
    // the warp) is off by at most 17 2^-24 sum_p |w_p x_p|, and, its T terms'
    // roundings having independent signs, typically by ~2^-24 sum_p |w_p x_p|
    // / sqrt(T): the error term taken is 8 2^-24 / sqrt(T) times a bound on
    // sum_p |w_p x_p| = sum_ab |h̃_a h̃_b x_ab|.  (The worst case would pass to
    // every deeper level through low and send most descents to the exact
    // path.)  The bound comes from the float after the slot's packed
    // triangle: a tree slot (PSD Gram) holds its trace, and sum_ab |h̃_a h̃_b
    // G_ab| <= |h̃|^2 tr G; a delta slot holds kappa_c = max_ab |D_ab| /
    // sqrt(g_a g_b) (g the root's diagonal), and the sum is <= kappa_c S with
    // S = (sum_a |h̃_a| sqrt(g_a))^2.  Both scale with |h̃|^2 rather than with
    // the mass, so they hold when h̃ is nearly orthogonal to the rows (masses
    // far below |h̃|^2 tr G).  C comes from the FP32 root (error eC = 8 2^-24
    // / sqrt(R) sum_p |w_p G_p|, the sum dominated by the R diagonal terms);
    // the top levels' masses are chained from it, so C's error
    // reaches a gap only as eC times the node's share of the root (the
    // product of the alpha or 1 - alpha taken), frozen below the top.  When a
    // gap falls within that term, C is taken to double-float first and tau,
    // low (by its share position) and M (by its share) corrected.
    // Returns the leaf heap index, with low its left edge, tau = u C, Cm the
    // root mass, xs whether the stage switched to exact masses, elow a bound
    // on low's FP32-path error, eleaf the C-error term left at the leaf.
    auto descend_exact = [&](const float* tr, const float* tl, const float* dt, int depth, int Ke, int64_t Lk,
                             int64_t Ik, int F, float uu, float hn2, df& Cm, df& tau, df& low, bool& xs,
                             float& elow, float& eleaf, float* trc) -> int64_t {
        low = df{0.f, 0.f};
        xs = false;
        elow = 0.f;
        eleaf = 0.f;
        if (!fetch_wait()) return 1;
        Cm = refine(partial(stage));
        const float cf = Cm.hi + Cm.lo;
        if (!(cf > 0.f) || !isfinite(cf)) return -1;
        tau = df_mul_f(Cm, uu);
        const float band = KRP_EXACT_BAND * cf;
        const float coarse = 4e-7f * cf;   // error of the FP32 gap below: a few ulp(C)
        float S = 0.f, eC = 0.f;
        const float etop = 4.76837158203125e-7f * rsqrtf((float)T);   // 8 2^-24 / sqrt(T)
        if (tl) {
            float sp = 0.f;
            if (lane < R) sp = fabsf(th[lane]) * sqrtf(stage[lane * R - (lane * (lane - 1)) / 2]);
            const float sr = warp_sum(sp);
            S = sr * sr;
            eC = 4.76837158203125e-7f * rsqrtf((float)R) * warp_sum(abs_partial(stage));
        }
        bool xc = false;            // C taken to double-float
        float share = 1.f, spos = 0.f;  // share of the root: node c's, and low's position (top levels)
        // traced samples record the masses of the path's nodes (double-float of
        // the (hi, lo) slots when there are low parts) and each node's mass as
        // its parent's minus its left sibling's
        const bool tracing = TRACE && __any_sync(0xffffffffu, trc != nullptr);
        df Mx = Cm;
        if constexpr (TRACE) {
            if (tracing && tl) {
                df l0, c0;
                exact_pass(tr, tl, 1, 0, 1, Mx, l0, c0);
            }
            if (trc) trc[0] = Mx.hi;
        }
        constexpr float KAPPA = 9.5367431640625e-7f;   // 2^-20 |m|: the eigencomponent stage's error term
        int64_t c = 1;
        int lvl = 0;
        df M = Cm;         // mass of node c (top levels)
        float eM = 0.f;    // bound on its error (C's own error aside)
        const int64_t nfull = Ik / F;   // leaves holding F rows
        // One decision at node c (depth lvl) from its staged left-child slot:
        // chained (delta slot) above depth Ke, plain below.  The branch is
        // taken from an FP32 estimate of m(L(c)) unless the gap is within the
        // estimate's error; the double-float m(L(c)) that the offset and the
        // chain carry forward is formed beside it.
        auto step = [&](const float* node) {
            const float part = partial(node);
            const float m = warp_sum(part);
            const bool top = lvl < Ke;
            float a = 0.5f;   // alpha_c: 1/2 unless c holds the rows' ragged end
            if (top && (c - ((int64_t)1 << lvl) + 1) > (nfull >> (depth - lvl))) a = node_alpha(c, lvl, Lk, F, Ik);
            const float mf = top ? fmaf(a, M.hi, m) : m;
            float e;
            if (tl) {
                const float bnd = node[P.T];
                e = top ? fmaf(a, eM, etop * bnd * S) : etop * bnd * hn2;
            } else {
                e = KAPPA * fabsf(m);
            }
            auto chain = [&]() -> df {
                return top ? df_add_f(a == 0.5f ? df{0.5f * M.hi, 0.5f * M.lo} : df_mul_f(M, a), m) : df{m, 0.f};
            };
            df mL = chain();
            const int64_t rfirst = ((2 * c + 1) << (depth - lvl - 1)) - Lk;
            bool left = true;
            if (rfirst * F < Ik) {
                const float gapf = (tau.hi - low.hi) - mf;
                const float ed = (tl && !xc && !xs) ? 2.f * eC * share : 0.f;
                if (!xs && fabsf(gapf) > coarse + band + elow + e + ed) {
                    left = gapf < 0.f;
                } else {
                    if (!tl) mL = refine(part);
                    df gap = df_add(df_add(tau, df_neg(low)), df_neg(mL));
                    // row stage: within C's error term, C to double-float
                    // (tau, low and M corrected through their shares); within
                    // the FP32 path's error, the switch to exact masses (C, low
                    // from the path, m(L(c))); once switched, m(L(c)) exact
                    float edn = ed;
#pragma unroll 1
                    for (int pass = 0; tl && pass < 2; ++pass) {
                        int what = 0;
                        if (xs)
                            what = 4;
                        else if (edn > 0.f && fabsf(gap.hi) <= band + elow + e + edn)
                            what = 1;
                        else if (fabsf(gap.hi) <= band + elow + e)
                            what = xc ? 6 : 7;
                        if (!what) break;
                        df Cx, lx, chx;
                        exact_pass(tr, tl, c, lvl, what, Cx, lx, chx);
                        if (what & 1) {
                            const df dC = df_add(Cx, df_neg(Cm));
                            tau = df_mul_f(Cx, uu);
                            if (!(what & 2)) {
                                low = df_add(low, df_mul_f(dC, spos));
                                M = df_add(M, df_mul_f(dC, share));
                            }
                            Cm = Cx;
                            xc = true;
                            edn = 0.f;
                        }
                        if (what & 2) {
                            low = lx;
                            xs = true;
                            elow = e = 0.f;
                        }
                        mL = (what & 4) ? chx : chain();
                        gap = df_add(df_add(tau, df_neg(low)), df_neg(mL));
                        if (what & 4) break;
                    }
                    left = gap.hi < 0.f || (gap.hi == 0.f && gap.lo <= 0.f);
                }
            }
            if constexpr (TRACE) {
                if (tracing) {
                    df mx = refine(part), c0, l0;
                    if (tl) exact_pass(tr, tl, c, lvl, 4, c0, l0, mx);
                    if (trc) {
                        trc[2 + 2 * lvl] = mx.hi;
                        trc[3 + 2 * lvl] = Mx.hi;
                    }
                    Mx = left ? mx : df_add(Mx, df_neg(mx));
                }
            }
            if (left) {
                c = 2 * c;
                if (top) {
                    M = mL;
                    eM = e;
                    share *= a;
                }
            } else {
                c = 2 * c + 1;
                low = df_add(low, mL);
                if (top) {
                    M = df_add(M, df_neg(mL));
                    eM += e;
                    spos = fmaf(a, share, spos);
                    share *= 1.f - a;
                }
                elow += e;
            }
            ++lvl;
        };
        // level 0 from the first fetch, then two levels per fetch (slot c,
        // then the chosen one of slots 2c, 2c + 1); one call site for step
        const float* node = stage + Tp;
        bool staged = true;   // node holds this level's slot
        while (lvl < depth && alive) {
            bool have_next = false;
            if (!staged) {
                have_next = lvl + 2 <= depth;
                const float* a = (lvl < Ke ? dt : tr) + c * Tp;
                const float* b = have_next ? (lvl + 1 < Ke ? dt : tr) + 2 * c * Tp : nullptr;
                if (!fetch(a, Tp * 4, b, have_next ? 2 * Tp * 4 : 0)) break;
                node = stage;
            }
            const int64_t c0 = c;
            step(node);
            staged = have_next;
            if (have_next) node = stage + (c == 2 * c0 ? Tp : 2 * Tp);
        }
        if (tl && !xc && !xs) eleaf = 2.f * eC * share;
        return c;
    };
#endif  // KRP_DESCENT_EXACT_TU
    const bool leaf_tma = (R & 3) == 0 && P.F * R <= C::STAGE;
    const int64_t warps_total = ncta * C::WARPS;
    for (int64_t s = cta * C::WARPS + warp; s < P.J && alive; s += warps_total) {
        if (lane < RMAX) {
            hh[lane] = lane < R ? 1.f : 0.f;
            hl[lane] = 0.f;
        }
        __syncwarp();
        bool ok = true;
        for (int pi = 0; pi < P.n_incl; ++pi) {
            const int k = P.incl[pi];
            const uint4 rnd = philox4x32_10(make_uint4((uint32_t)s, P.draw, (uint32_t)pi, 0u),
                                            make_uint2(P.key0, P.key1));
            const float u_eig = u32_to_unit(rnd.x), u_row = u32_to_unit(rnd.y);
            float* trc = (P.trace && s < P.n_trace && lane == 0)
                             ? P.trace + ((s * P.n_incl + pi) * 2) * FAST_TRACE_STRIDE
                             : nullptr;
            // Two stages through one code path: stage 0 draws the eigencomponent
            // u from E_k (leaf size 1, Y = G_k, history h); stage 1 draws the row
            // from Z_k (leaf size F, Y = [1], history h̃ = h ∘ V[:,u]).
            const int64_t Lk = P.L[k], Ik = P.I[k];
            const int F = P.F;
            df tau{0.f, 0.f}, low{0.f, 0.f};
            float cf = 0.f, margin = 0.f;
            int64_t c = 1;
            int u = 0;
            bool xs = false;    // exact-decision mode: the row stage switched to exact masses
            float elow = 0.f;   // exact-decision mode: bound on the FP32 path's error in low
            float eleaf = 0.f;  // exact-decision mode: C's error term at the leaf
            float hn2 = 0.f;    // exact-decision mode: |h̃|^2 in FP32
            for (int sg = 0; sg < 2; ++sg) {
                const bool xrow = EXACT && sg == 1;
                const float* tr = sg ? P.tree[k] : P.etree[k];
                const int depth = sg ? P.depth[k] : P.dE;
                // issue the first fetch (root and levels 0-1; in the exact row
                // stage the root and D_1), then build the stage's weights while
                // it is in flight
                const int nfirst = depth >= 1 ? 2 : 1;
                fetch_issue(xrow ? P.dtop[k] : tr, (uint32_t)(nfirst * Tp * 4), nullptr, 0);
                if (sg == 0) {
                    if (lane < RMAX) th[lane] = hh[lane] + hl[lane];
                } else if (lane < RMAX) {
                    float vh = 0.f, vl = 0.f;
                    if (lane < R) {
                        vh = __ldg(P.Vhi[k] + (size_t)u * R + lane);
                        vl = __ldg(P.Vlo[k] + (size_t)u * R + lane);
                    }
                    const df t = df_add(df_mul_f(df{hh[lane], hl[lane]}, vh), df_mul_f(df{hh[lane], hl[lane]}, vl));
                    th[lane] = t.hi;   // h̃ = h ∘ V[:,u], rounded once (t is normalised)
                    thl[lane] = t.lo;
                }
                __syncwarp();
                make_weights(th);
                if constexpr (EXACT) hn2 = warp_sum(lane < R ? th[lane] * th[lane] : 0.f);
                if (trc && sg) trc += FAST_TRACE_STRIDE;
                df Cm;
                if constexpr (EXACT) {
#if KRP_DESCENT_EXACT_TU
                    c = descend_exact(tr, sg ? P.tlo[k] : nullptr, xrow ? P.dtop[k] : tr, depth, sg ? P.Ke[k] : 0,
                                      sg ? Lk : P.Rp, sg ? Ik : R, sg ? F : 1, sg ? u_row : u_eig, hn2, Cm, tau,
                                      low, xs, elow, eleaf, trc);
#endif
                } else {
                    c = descend(tr, depth, sg ? Lk : P.Rp, sg ? Ik : R, sg ? F : 1, sg ? u_row : u_eig, Cm,
                                tau, low, trc);
                }
                if (!alive) break;
                if (c < 0) {
                    const float cv = Cm.hi + Cm.lo;
                    if (lane == 0) set_status(P.status, isfinite(cv) ? KRP_EZERO : KRP_ENUMERIC);
                    ok = false;
                    break;
                }
                cf = Cm.hi + Cm.lo;
                margin = 1e-6f * cf;
                if (sg == 0) u = (int)(c - P.Rp);
            }
            if (!alive || !ok) break;
            // ------------------------------------------------ leaf scan
            const int64_t row0 = (c - Lk) * F;
            const int nrows = (int)min((int64_t)F, Ik - row0);
            const int rpt = (F + 31) >> 5;
            const float* Uk = P.U[k];
            if (leaf_tma && !fetch(Uk + row0 * R, (uint32_t)(nrows * R * 4), nullptr, 0)) break;
            float q[C::RPT];
            float run = 0.f;
            float erow = 0.f;   // exact-decision mode: bound on this lane's row weights' errors
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = lane * rpt + r;
                float d = 0.f;
                if (r < rpt && t < nrows) {
                    if (leaf_tma) {
                        const float4* row = reinterpret_cast<const float4*>(stage + t * R);
                        const float4* hv = reinterpret_cast<const float4*>(th);
                        const int nq = R >> 2;
                        float2 acc = make_float2(0.f, 0.f);
                        float ab = 0.f;
                        for (int a = 0; a < nq; ++a) {
                            const int j = (a + t) % nq;   // rotate chunks: conflict-free banks
                            const float4 x = row[j], y = hv[j];
                            acc = ffma2(make_float2(x.x, x.y), make_float2(y.x, y.y), acc);
                            acc = ffma2(make_float2(x.z, x.w), make_float2(y.z, y.w), acc);
                            if constexpr (EXACT) {
                                ab = fmaf(fabsf(x.x), fabsf(y.x), ab);
                                ab = fmaf(fabsf(x.y), fabsf(y.y), ab);
                                ab = fmaf(fabsf(x.z), fabsf(y.z), ab);
                                ab = fmaf(fabsf(x.w), fabsf(y.w), ab);
                            }
                        }
                        d = acc.x + acc.y;
#if KRP_DESCENT_EXACT_TU
                        if constexpr (EXACT) erow += row_err(d, ab);
#endif
                    } else {
                        const float* row = Uk + (row0 + t) * R;
                        float ab = 0.f;
                        for (int a = 0; a < R; ++a) {
                            const float x = __ldg(row + a);
                            d = fmaf(x, th[a], d);
                            if constexpr (EXACT) ab = fmaf(fabsf(x), fabsf(th[a]), ab);
                        }
#if KRP_DESCENT_EXACT_TU
                        if constexpr (EXACT) erow += row_err(d, ab);
#endif
                    }
                }
                q[r] = d * d;
                run += q[r];
            }
            const df rel = df_add(tau, df_neg(low));
            const float target = rel.hi + rel.lo;
            float inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            float cum = __shfl_up_sync(0xffffffffu, inc, 1);
            if (lane == 0) cum = 0.f;
            int first = 0x7fffffff, lastpos = -1;
            bool near = false;
            float mlow = 0.f;   // exact-decision mode: the offset's part of the margin
            if constexpr (EXACT) {
                // low's FP32-path error and C's, then the FP32 scan's own: the
                // rows' weights (row_err) and ~10 roundings of the running sums
                mlow = KRP_EXACT_BAND * cf + elow + eleaf;
                margin = mlow + warp_sum(erow) + 9.5367431640625e-7f * __shfl_sync(0xffffffffu, inc, 31);
            }
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = lane * rpt + r;
                if (r < rpt && t < nrows) {
                    cum += q[r];
                    // exact-decision mode: a row of zero weight is never drawn
                    // (after a switch to exact masses tau could sit at the
                    // leaf's left edge; the FP32 path's own offsets keep tau
                    // above it)
                    if (first == 0x7fffffff && target <= cum && (!EXACT || q[r] > 0.f)) first = t;
                    if (fabsf(cum - target) <= margin) near = true;
                    if (q[r] > 0.f) lastpos = t;
                }
            }
            const bool any_near = __any_sync(0xffffffffu, near);
            if constexpr (EXACT) {
#if KRP_DESCENT_EXACT_TU
              if (any_near) {
                // re-take the leaf scan with rows rescored in double-float: q =
                // (U[t] · h̃)^2 with h̃ = (th, thl); if an edge is then still
                // within the offset's error of tau, once more from the exact
                // offset
                int2 fl;
                for (int pass = 0; pass < 2; ++pass) {
                    bool nl;
                    fl = exact_leaf_scan<C::RPT>(leaf_tma ? stage : Uk + row0 * R, R, rpt, nrows, th, thl, tau, low,
                                                 xs ? 0.f : mlow, nl);
                    if (xs || !nl) break;
                    df Cx, chx;
                    exact_pass(P.tree[k], P.tlo[k], c, P.depth[k], 3, Cx, low, chx);
                    tau = df_mul_f(Cx, u_row);
                    xs = true;
                }
                first = fl.x;
                lastpos = fl.y;
              }
#endif
            } else if (any_near) {
                // redo the scan in double-float: edges low + cumulative weights
                df acc{0.f, 0.f};
#pragma unroll
                for (int r = 0; r < C::RPT; ++r)
                    if (r < rpt && lane * rpt + r < nrows) acc = df_add(acc, df{q[r], 0.f});
                df incd = acc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float vh = __shfl_up_sync(0xffffffffu, incd.hi, o);
                    const float vl = __shfl_up_sync(0xffffffffu, incd.lo, o);
                    if (lane >= o) incd = df_add(df{vh, vl}, incd);
                }
                df cd{__shfl_up_sync(0xffffffffu, incd.hi, 1), __shfl_up_sync(0xffffffffu, incd.lo, 1)};
                if (lane == 0) cd = df{0.f, 0.f};
                cd = df_add(cd, low);
                first = 0x7fffffff;
#pragma unroll
                for (int r = 0; r < C::RPT; ++r) {
                    const int t = lane * rpt + r;
                    if (r < rpt && t < nrows) {
                        cd = df_add(cd, df{q[r], 0.f});
                        if (first == 0x7fffffff && df_le(tau, cd)) first = t;
                    }
                }
            }
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) {
                first = min(first, __shfl_xor_sync(0xffffffffu, first, m));
                lastpos = max(lastpos, __shfl_xor_sync(0xffffffffu, lastpos, m));
            }
            int t_sel = first != 0x7fffffff ? first : lastpos;
            if (t_sel < 0) {  // no positive weight in the leaf: only through rounding
                if (lane == 0) set_status(P.status, KRP_ENUMERIC);
                t_sel = 0;
            }
            const int64_t trow = row0 + t_sel;
            if (lane < R) {
                const float x = leaf_tma ? stage[t_sel * R + lane] : __ldg(Uk + trow * R + lane);
                const df nh = df_mul_f(df{hh[lane], hl[lane]}, x);
                hh[lane] = nh.hi;
                hl[lane] = nh.lo;
            }
            if (lane == 0) P.idx[(int64_t)k * P.J + s] = (int32_t)trow;
            __syncwarp();
        }
        if (!alive) break;
        // ------------------------------------------------ epilogue
        if (lane < RMAX) th[lane] = hh[lane] + hl[lane];
        __syncwarp();
        make_weights(th);
        float part = 0.f;
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c4 = lane + 32 * m;
            if (c4 < nc4) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(P.Gplus32) + c4);
                part = fmaf(w4[m].x, v.x, part);
                part = fmaf(w4[m].y, v.y, part);
                part = fmaf(w4[m].z, v.z, part);
                part = fmaf(w4[m].w, v.w, part);
            }
        }
        // q_s = ℓ_s / rank with ℓ_s = hᵀG⁺h = lv 2^gexp (G⁺ is stored scaled by 2^-gexp);
        // w_s = 1/sqrt(J q_s) formed without q_s itself, which can underflow FP32
        const df lev = refine(part);
        const float lv = (lev.hi + lev.lo) / (float)P.rank[0];
        const int gexp = P.rank[1];
        const float w = ok ? ldexpf(1.0f / sqrtf((float)P.J * lv * ((gexp & 1) ? 2.f : 1.f)), -(gexp >> 1)) : 0.f;
        if (lane == 0) {
            P.weight[s] = w;
            if (P.logq) P.logq[s] = ok ? logf(lv) + (float)gexp * 0.6931471805599453f : -INFINITY;
        }
        if (P.SA && lane < R) P.SA[s * R + lane] = w * th[lane];
        __syncwarp();
    }
    if (!alive) {
        // a staged copy never completed: wait once more (bounded) so that no
        // copy into this CTA's shared memory is left in flight, then return
        mbar_wait(mbar, phase ^ 1u);
    }
}

// Four CTAs (32 samples) per SM where the registers allow it without spills
// (RMAX <= 16: 63 registers); at RMAX = 32 a 64-register cap spills and the
// draw slows from 1.24 to 1.34 ms, so three.  The exact-decision kernels keep
// their double-float state in registers at two CTAs per SM (at three they
// spill, and run slower).
template <int RMAX, bool EXACT, bool TRACE = false>
__global__ void __launch_bounds__(EXACT ? 128 : 256, EXACT ? 5 : (RMAX <= 16 ? 4 : 3))
    krp_descent_fast(const __grid_constant__ FastParams P) {
    descent_fast_body<RMAX, EXACT, TRACE>(P, blockIdx.x, gridDim.x);
}

namespace {
template <int RMAX, bool EXACT, bool TRACE = false>
cudaError_t launch_fast_t(const FastParams& P, int num_sms, cudaStream_t st) {
    using C = FastCfg<RMAX, EXACT>;
    auto k = krp_descent_fast<RMAX, EXACT, TRACE>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::WARPS * 32, C::SMEM);
    per_sm = per_sm > 0 ? per_sm : 1;
    const int64_t need = (P.J + C::WARPS - 1) / C::WARPS;
    const int64_t grid = need < (int64_t)num_sms * per_sm ? need : (int64_t)num_sms * per_sm;
    k<<<(unsigned)grid, C::WARPS * 32, C::SMEM, st>>>(P); count_launch();
    return cudaGetLastError();
}
}  // namespace

#if KRP_DESCENT_EXACT_TU
// Exact-decision descent for R <= rmax (8, 16 or 32).
cudaError_t launch_fast_exact(const FastParams& P, int rmax, int num_sms, cudaStream_t st) {
    if (P.trace) {
        if (rmax <= 8) return launch_fast_t<8, true, true>(P, num_sms, st);
        if (rmax <= 16) return launch_fast_t<16, true, true>(P, num_sms, st);
        return launch_fast_t<32, true, true>(P, num_sms, st);
    }
    if (rmax <= 8) return launch_fast_t<8, true>(P, num_sms, st);
    if (rmax <= 16) return launch_fast_t<16, true>(P, num_sms, st);
    return launch_fast_t<32, true>(P, num_sms, st);
}
#else
cudaError_t launch_fast_exact(const FastParams& P, int rmax, int num_sms, cudaStream_t st);

// Test hook for the bounded wait: one warp waits on an mbarrier that nothing
// completes, with `tries` suspending tries, and must report KRP_ETIMEOUT.
__global__ void wait_timeout_probe(int tries, int* status) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        mbar_init(&mbar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool done = mbar_wait(&mbar, 0u, tries);
    if (!__all_sync(0xffffffffu, done) && threadIdx.x == 0) set_status(status, KRP_ETIMEOUT);
}

cudaError_t launch_wait_timeout_probe(krp_sampler* s, int tries) {
    wait_timeout_probe<<<1, 32, 0, s->stream>>>(tries, s->status); count_launch();
    return cudaGetLastError();
}

// Static part of a problem's parameter block (factors, trees, eigenvectors,
// G⁺, status); the per-call fields are left zero.
void fast_params_for(const krp_sampler* s, int exclude_j, FastParams* out) {
    FastParams& P = *out;
    P = FastParams{};
    for (int k = 0; k < s->N; ++k) {
        P.U[k] = s->U[k];
        P.tree[k] = s->tree[k];
        if (s->exact) {
            P.tlo[k] = s->tree_lo[k];
            P.dtop[k] = s->dtop[k];
            P.Ke[k] = s->Ke[k];
        }
        P.etree[k] = s->etree + (size_t)k * s->Rp * s->Tp;
        P.Vhi[k] = s->V32 + (size_t)k * s->R * s->R;
        P.Vlo[k] = s->V32lo + (size_t)k * s->R * s->R;
        P.I[k] = s->I[k];
        P.L[k] = s->L[k];
        P.depth[k] = s->depth[k];
        if (k != exclude_j) P.incl[P.n_incl++] = k;
    }
    P.R = s->R;
    P.F = s->F;
    P.T = s->T;
    P.Tp = s->Tp;
    P.Rp = s->Rp;
    P.dE = s->dE;
    P.Gplus32 = s->Gplus32;
    P.rank = s->rank_dev;
    P.status = s->status;
}

bool launch_descent_fast(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err) {
    if (s->R > 32) return false;
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
    P.nexact = s->exact ? s->nexact : nullptr;
    if (s->exact)
        *err = launch_fast_exact(P, s->R, s->num_sms, s->stream);
    else if (s->R <= 8)
        *err = launch_fast_t<8, false>(P, s->num_sms, s->stream);
    else if (s->R <= 16)
        *err = launch_fast_t<16, false>(P, s->num_sms, s->stream);
    else
        *err = launch_fast_t<32, false>(P, s->num_sms, s->stream);
    return true;
}

// Batched descent: CTA b serves problem p = b / ctas_per_problem, taking the
// static block table[p] into shared memory and the per-call fields from `call`
// (outputs of problem p at idx + p N J, weight + p J, SA + J row_off[p]).
// RMAX = 32 serves every R <= 32.
__global__ void __launch_bounds__(256, 3) krp_descent_fast_batch(const FastParams* __restrict__ table,
                                                                 const __grid_constant__ FastCall call,
                                                                 int ctas_per_problem) {
    __shared__ __align__(16) FastParams sP;
    const int p = blockIdx.x / ctas_per_problem;
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(table + p);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sP);
        for (int w = threadIdx.x; w < (int)(sizeof(FastParams) / 4); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sP.key0 = call.key0;
        sP.key1 = call.key1;
        sP.draw = call.draw;
        sP.J = call.J;
        sP.idx = call.idx + (int64_t)p * call.N * call.J;
        sP.weight = call.weight + (int64_t)p * call.J;
        sP.SA = call.SA ? call.SA + call.J * call.row_off[p] : nullptr;
        sP.logq = nullptr;
        sP.trace = nullptr;
        sP.n_trace = 0;
    }
    __syncthreads();
    descent_fast_body<32>(sP, blockIdx.x % ctas_per_problem, ctas_per_problem);
}

cudaError_t launch_descent_fast_batch(const FastParams* table_dev, const FastCall& call, int P, int ctas_per_problem,
                                      cudaStream_t st) {
    using C = FastCfg<32>;
    cudaFuncSetAttribute(krp_descent_fast_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    cudaFuncSetAttribute(krp_descent_fast_batch, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    krp_descent_fast_batch<<<(unsigned)(P * ctas_per_problem), 256, C::SMEM, st>>>(table_dev, call, ctas_per_problem);
    count_launch();
    return cudaGetLastError();
}

#endif  // KRP_DESCENT_EXACT_TU

}  // namespace krp
