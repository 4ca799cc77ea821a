// a4 + a5 (+ a6 fused) for 32 < R <= 128: the batched conditional descent of
// the R <= 32 kernel (the sampling loop of Alg. 2 with the loops exchanged as
// in App. A.6; Alg. 4 on E_k and Z_k; Eqs. first_dist and
// second_conditional_dist) with a team of TEAM warps per sample, because a
// node of the tree (R(R+1)/2 floats: 8.3 KB at R = 64, 33 KB at R = 128) is
// too much quadratic form for one warp.
//
// Per team: one mbarrier and a 3-node shared stage filled by TMA bulk copies —
// the first fetch of a stage brings the root and level 0, later ones bring
// node c and both candidates of the next level (slots 2c, 2c+1), so two
// levels cost one memory round trip; after each decision only the chosen
// child's next-level mass is formed.  The team's threads own fixed float4
// chunks of a node (weights w_p = h_i h_j, doubled off the diagonal, in
// registers, the (i, j) of each chunk's first entry kept as an 8+8-bit code);
// masses are team sums; decisions use FP32 unless tau is within 1e-6 C of the
// cutoff, then the double-float team sum, with tau, low and h in double-float.  Every wait is bounded and
// its outcome agreed by the whole team (bar.red) before anyone acts on it.
#include "common.cuh"
#include "internal.h"

#include <math.h>

#include <algorithm>

namespace krp {
namespace {

__device__ __forceinline__ uint32_t tsm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool tmb_wait(uint64_t* m, uint32_t parity, int max_tries = 1 << 16) {
    for (int it = 0; it < max_tries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(tsm_u32(m)), "r"(parity), "r"(100000u)
            : "memory");
        if (done) return true;
    }
    return false;
}


template <int RMAX, int TEAM, int CTA_THREADS = 256, int MINB = 2>
struct TeamCfg {
    static constexpr int NT = 32 * TEAM;                        // threads per sample
    static constexpr int THREADS = CTA_THREADS;
    static constexpr int BLOCKS = MINB;                         // CTAs per SM the registers are sized for
    static constexpr int TEAMS = CTA_THREADS / NT;              // samples per CTA
    static constexpr int TPMAX = ((RMAX * (RMAX + 1) / 2) + 7) & ~7;
    static constexpr int NC4 = TPMAX / 4;
    static constexpr int NCH = (NC4 + NT - 1) / NT;             // float4 chunks per thread
    static constexpr int RPT = (4 * RMAX + NT - 1) / NT;        // leaf rows per thread (F <= 4R)
    static constexpr int STAGE = 3 * TPMAX;                     // floats
    // stage, hh, hl, th, 4 x TEAM floats of reductions, pick/flag ints, mbarrier
    static constexpr int TEAM_BYTES = ((STAGE + 3 * RMAX + 4 * TEAM) * 4 + 4 * 4 + 16 + 127) & ~127;
    static constexpr int SMEM = TEAMS * TEAM_BYTES;
    // one team's bytes for the actual node stride: a three-node stage of 3 Tp floats
    static int team_bytes(int Tp) { return ((3 * Tp + 3 * RMAX + 4 * TEAM) * 4 + 4 * 4 + 16 + 127) & ~127; }
};

template <int RMAX, int TEAM, int CTA_THREADS, int MINB>
__global__ void __launch_bounds__(CTA_THREADS, MINB)
    krp_descent_team(const __grid_constant__ FastParams P) {
    using C = TeamCfg<RMAX, TEAM, CTA_THREADS, MINB>;
    constexpr int NT = C::NT, NCH = C::NCH;
    extern __shared__ __align__(128) unsigned char smem[];
    const int team = threadIdx.x / NT, tt = threadIdx.x % NT, lane = tt & 31, wib = tt >> 5;
    // a CTA of one team lays its stage out for the actual node stride (3 Tp
    // floats); CTAs of several teams use the fixed stride of RMAX
    constexpr bool ONE = C::TEAMS == 1;
    const int stage_f = ONE ? 3 * P.Tp : C::STAGE;
    unsigned char* base = smem + (ONE ? 0 : (size_t)team * C::TEAM_BYTES);
    float* stage = reinterpret_cast<float*>(base);
    float* hh = stage + stage_f;
    float* hl = hh + RMAX;
    float* th = hl + RMAX;
    float* red = th + RMAX;                    // TEAM floats (sums), then 2 TEAM (double-float sums)
    float* red2 = red + TEAM;
    float* scn = red2 + 2 * TEAM;              // TEAM floats (scan totals)
    int* pick = reinterpret_cast<int*>(scn + TEAM);   // [0] first, [1] last
    uint64_t* mbar = reinterpret_cast<uint64_t*>(base + ((stage_f + 3 * RMAX + 4 * TEAM) * 4 + 16 + 7) / 8 * 8);

    const int R = P.R, T = P.T, Tp = P.Tp;
    const int nc4 = Tp >> 2;

    auto team_sync = [&]() {
        if (TEAM == 1)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(NT) : "memory");
    };
    auto team_and = [&](bool v) -> bool {
        if (TEAM == 1) return __all_sync(0xffffffffu, v);
        uint32_t r;
        asm volatile(
            "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(r)
            : "r"((uint32_t)v), "r"(1 + team), "r"(NT)
            : "memory");
        return r != 0;
    };
    auto team_or = [&](bool v) -> bool {
        if (TEAM == 1) return __any_sync(0xffffffffu, v);
        uint32_t r;
        asm volatile(
            "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(r)
            : "r"((uint32_t)v), "r"(1 + team), "r"(NT)
            : "memory");
        return r != 0;
    };
    // sums identical in every thread of the team (fixed order across warps)
    auto team_sum = [&](float v) -> float {
        v = warp_sum(v);
        if (TEAM == 1) return v;
        if (lane == 0) red[wib] = v;
        team_sync();
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < TEAM; ++w) t += red[w];
        team_sync();
        return t;
    };
    auto team_sum_df = [&](float part) -> df {
        df v = warp_sum_df(df{part, 0.f});
        if (TEAM == 1) return v;
        if (lane == 0) {
            red2[2 * wib] = v.hi;
            red2[2 * wib + 1] = v.lo;
        }
        team_sync();
        df t{0.f, 0.f};
#pragma unroll
        for (int w = 0; w < TEAM; ++w) t = df_add(t, df{red2[2 * w], red2[2 * w + 1]});
        team_sync();
        return t;
    };

    // (i, j) of the first packed entry p = 4 (tt + NT m) of each of this
    // thread's chunks, 8 bits each, two chunks per word; the chunk's other
    // entries follow along the row (j + 1, wrapping to (i + 1, i + 1)).
    constexpr int NIJ = (NCH + 1) / 2;
    uint32_t ij[NIJ];
#pragma unroll
    for (int h = 0; h < NIJ; ++h) ij[h] = 0u;
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
        const int p = 4 * (tt + NT * m);
        int i = 0, rem = p;
        if (p < T)
            while (rem >= R - i) {
                rem -= R - i;
                ++i;
            }
        const uint32_t code = p < T ? (uint32_t)(i | ((i + rem) << 8)) : 0u;
        ij[m >> 1] |= code << (16 * (m & 1));
    }
    if (tt == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tsm_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    bool alive = true;

    auto fetch_issue = [&](const float* a, uint32_t abytes, const float* b, uint32_t bbytes) {
        team_sync();  // everyone is done with the stage
        if (tt == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tsm_u32(mbar)),
                         "r"(abytes + bbytes)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             tsm_u32(stage)),
                         "l"(a), "r"(abytes), "r"(tsm_u32(mbar))
                         : "memory");
            if (bbytes)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        tsm_u32(stage + Tp)),
                    "l"(b), "r"(bbytes), "r"(tsm_u32(mbar))
                    : "memory");
        }
    };
    auto fetch_wait = [&]() -> bool {
        const bool ok = team_and(tmb_wait(mbar, phase));
        phase ^= 1u;
        if (!ok) {
            if (tt == 0) set_status(P.status, KRP_ETIMEOUT);
            alive = false;
        }
        return ok;
    };
    auto fetch = [&](const float* a, uint32_t abytes, const float* b, uint32_t bbytes) -> bool {
        fetch_issue(a, abytes, b, bbytes);
        return fetch_wait();
    };

    float4 w4[NCH];
    auto make_weights = [&](const float* x) {
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const uint32_t code = (ij[m >> 1] >> (16 * (m & 1))) & 0xFFFFu;
            int i = code & 0xFF, j = code >> 8;
            const int p0 = 4 * (tt + NT * m);
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
            w4[m] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
    };
    auto partial = [&](const float* node) -> float {
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c = tt + NT * m;
            if (c < nc4) {
                const float4 v = reinterpret_cast<const float4*>(node)[c];
                a0 = ffma2(make_float2(w4[m].x, w4[m].y), make_float2(v.x, v.y), a0);
                a1 = ffma2(make_float2(w4[m].z, w4[m].w), make_float2(v.z, v.w), a1);
            }
        }
        return (a0.x + a1.x) + (a0.y + a1.y);
    };
    // tau, low and m are the same in every thread of the team, so the branch
    // into the double-float sum is team-uniform.  (tau.hi - low.hi) - m is
    // within a few ulp(C) + |tau.lo| + |low.lo| < 3e-7 C of tau - low - m.
    auto go_left = [&](df tau, df low, float m, float part, float margin, df& cut) -> bool {
        const float gapf = (tau.hi - low.hi) - m;
        if (fabsf(gapf) > margin) {
            if (gapf < 0.f) return true;
            cut = df_add(low, df{m, 0.f});
            return false;
        }
        cut = df_add(low, team_sum_df(part));
        return df_le(tau, cut);
    };
    // One descent of Alg. 4 whose first fetch (slots 0 and 1, already issued)
    // holds the root and level 0.  Returns the leaf heap index (-1: zero or
    // non-finite root mass); low is the leaf's left edge, Cm the root mass.
    auto descend = [&](const float* __restrict__ tr, int depth, int64_t Lk, int64_t nreal_rows, int F, float uu,
                       df& Cm, df& tau, df& low, float* trc) -> int64_t {
        low = df{0.f, 0.f};
        if (!fetch_wait()) return 1;
        const int nfirst = depth >= 1 ? 2 : 1;
        float pr[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) pr[q] = q < nfirst ? partial(stage + q * Tp) : 0.f;
        Cm = team_sum_df(pr[0]);
        const float cf = Cm.hi + Cm.lo;
        if (!(cf > 0.f) || !isfinite(cf)) return -1;
        tau = df_mul_f(Cm, uu);
        const float margin = 1e-6f * cf;
        if (trc) trc[0] = cf;
        int64_t c = 1;
        int lvl = 0;
        float mnode = cf;
        float mA = depth >= 1 ? team_sum(pr[1]) : 0.f, pA = pr[1];
        bool have_next = false;
        while (lvl < depth && alive) {
            if (lvl > 0) {
                have_next = lvl + 2 <= depth;
                if (!fetch(tr + c * Tp, Tp * 4, have_next ? tr + 2 * c * Tp : nullptr, have_next ? 2 * Tp * 4 : 0))
                    break;
                pA = partial(stage);
                mA = team_sum(pA);
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
            pA = partial(stage + (left ? Tp : 2 * Tp));
            mA = team_sum(pA);
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

    const bool leaf_tma = (R & 3) == 0 && P.F * R <= stage_f;
    const int64_t teams_total = (int64_t)gridDim.x * C::TEAMS;
    for (int64_t s = (int64_t)blockIdx.x * C::TEAMS + team; s < P.J && alive; s += teams_total) {
        for (int a = tt; a < RMAX; a += NT) {
            hh[a] = a < R ? 1.f : 0.f;
            hl[a] = 0.f;
        }
        team_sync();
        bool ok = true;
        for (int pi = 0; pi < P.n_incl; ++pi) {
            const int k = P.incl[pi];
            const uint4 rnd = philox4x32_10(make_uint4((uint32_t)s, P.draw, (uint32_t)pi, 0u),
                                            make_uint2(P.key0, P.key1));
            const float u_eig = u32_to_unit(rnd.x), u_row = u32_to_unit(rnd.y);
            float* trc = (P.trace && s < P.n_trace && tt == 0)
                             ? P.trace + ((s * P.n_incl + pi) * 2) * 66
                             : nullptr;
            const int64_t Lk = P.L[k], Ik = P.I[k];
            const int F = P.F;
            df tau{0.f, 0.f}, low{0.f, 0.f};
            float cf = 0.f, margin = 0.f;
            int64_t c = 1;
            int u = 0;
            for (int sg = 0; sg < 2; ++sg) {
                const float* tr = sg ? P.tree[k] : P.etree[k];
                const int depth = sg ? P.depth[k] : P.dE;
                const int nfirst = depth >= 1 ? 2 : 1;
                fetch_issue(tr, (uint32_t)(nfirst * Tp * 4), nullptr, 0);
                for (int a = tt; a < RMAX; a += NT) {
                    if (sg == 0) {
                        th[a] = hh[a] + hl[a];
                    } else {
                        float vh = 0.f, vl = 0.f;
                        if (a < R) {
                            vh = __ldg(P.Vhi[k] + (size_t)u * R + a);
                            vl = __ldg(P.Vlo[k] + (size_t)u * R + a);
                        }
                        const df t = df_add(df_mul_f(df{hh[a], hl[a]}, vh), df_mul_f(df{hh[a], hl[a]}, vl));
                        th[a] = t.hi + t.lo;   // h̃ = h ∘ V[:,u], rounded once
                    }
                }
                team_sync();
                make_weights(th);
                if (trc && sg) trc += 66;
                df Cm;
                c = descend(tr, depth, sg ? Lk : P.Rp, sg ? Ik : R, sg ? F : 1, sg ? u_row : u_eig, Cm, tau, low,
                            trc);
                if (!alive) break;
                if (c < 0) {
                    const float cv = Cm.hi + Cm.lo;
                    if (tt == 0) set_status(P.status, isfinite(cv) ? KRP_EZERO : KRP_ENUMERIC);
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
            const int rpt = (F + NT - 1) / NT;
            const float* Uk = P.U[k];
            if (leaf_tma && !fetch(Uk + row0 * R, (uint32_t)(nrows * R * 4), nullptr, 0)) break;
            float q[C::RPT];
            float run = 0.f;
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = tt * rpt + r;
                float d = 0.f;
                if (r < rpt && t < nrows) {
                    if (leaf_tma) {
                        const float4* row = reinterpret_cast<const float4*>(stage + t * R);
                        const float4* hv = reinterpret_cast<const float4*>(th);
                        const int nq = R >> 2;
                        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
                        int j = t % nq;   // rows start on rotated columns (no bank conflicts)
                        for (int a = 0; a < nq; ++a) {
                            const float4 x = row[j], y = hv[j];
                            a0 = ffma2(make_float2(x.x, x.y), make_float2(y.x, y.y), a0);
                            a1 = ffma2(make_float2(x.z, x.w), make_float2(y.z, y.w), a1);
                            j = j + 1 == nq ? 0 : j + 1;
                        }
                        d = (a0.x + a1.x) + (a0.y + a1.y);
                    } else {
                        const float* row = Uk + (row0 + t) * R;
                        for (int a = 0; a < R; ++a) d = fmaf(__ldg(row + a), th[a], d);
                    }
                }
                q[r] = (r < rpt && t < nrows) ? d * d : 0.f;
                run += q[r];
            }
            // exclusive scan of the per-thread totals over the team (FP32)
            float inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            float cum = __shfl_up_sync(0xffffffffu, inc, 1);
            if (lane == 0) cum = 0.f;
            if (TEAM > 1) {
                if (lane == 31) scn[wib] = inc;
                team_sync();
                float off = 0.f;
                for (int w = 0; w < wib; ++w) off += scn[w];
                cum += off;
                team_sync();
            }
            const df rel = df_add(tau, df_neg(low));
            const float target = rel.hi + rel.lo;
            int first = 0x7fffffff, lastpos = -1;
            bool near = false;
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = tt * rpt + r;
                if (r < rpt && t < nrows) {
                    cum += q[r];
                    if (first == 0x7fffffff && target <= cum) first = t;
                    if (fabsf(cum - target) <= margin) near = true;
                    if (q[r] > 0.f) lastpos = t;
                }
            }
            if (team_or(near)) {
                // redo the scan in double-float: edges low + cumulative weights
                df acc{0.f, 0.f};
#pragma unroll
                for (int r = 0; r < C::RPT; ++r) acc = df_add(acc, df{q[r], 0.f});
                df incd = acc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float vh = __shfl_up_sync(0xffffffffu, incd.hi, o);
                    const float vl = __shfl_up_sync(0xffffffffu, incd.lo, o);
                    if (lane >= o) incd = df_add(df{vh, vl}, incd);
                }
                df cd{__shfl_up_sync(0xffffffffu, incd.hi, 1), __shfl_up_sync(0xffffffffu, incd.lo, 1)};
                if (lane == 0) cd = df{0.f, 0.f};
                if (TEAM > 1) {
                    if (lane == 31) {
                        red2[2 * wib] = incd.hi;
                        red2[2 * wib + 1] = incd.lo;
                    }
                    team_sync();
                    df off{0.f, 0.f};
                    for (int w = 0; w < wib; ++w) off = df_add(off, df{red2[2 * w], red2[2 * w + 1]});
                    cd = df_add(off, cd);
                    team_sync();
                }
                cd = df_add(cd, low);
                first = 0x7fffffff;
#pragma unroll
                for (int r = 0; r < C::RPT; ++r) {
                    const int t = tt * rpt + r;
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
            if (TEAM > 1) {
                if (tt == 0) {
                    pick[0] = 0x7fffffff;
                    pick[1] = -1;
                }
                team_sync();
                if (lane == 0) {
                    atomicMin(&pick[0], first);
                    atomicMax(&pick[1], lastpos);
                }
                team_sync();
                first = pick[0];
                lastpos = pick[1];
                team_sync();
            }
            int t_sel = first != 0x7fffffff ? first : lastpos;
            if (t_sel < 0) {  // no positive weight in the leaf: only through rounding
                if (tt == 0) set_status(P.status, KRP_ENUMERIC);
                t_sel = 0;
            }
            const int64_t trow = row0 + t_sel;
            for (int a = tt; a < R; a += NT) {
                const float x = leaf_tma ? stage[t_sel * R + a] : __ldg(Uk + trow * R + a);
                const df nh = df_mul_f(df{hh[a], hl[a]}, x);
                hh[a] = nh.hi;
                hl[a] = nh.lo;
            }
            if (tt == 0) P.idx[(int64_t)k * P.J + s] = (int32_t)trow;
            team_sync();
        }
        if (!alive) break;
        // ------------------------------------------------ epilogue
        for (int a = tt; a < RMAX; a += NT) th[a] = hh[a] + hl[a];
        team_sync();
        make_weights(th);
        float part = 0.f;
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c4 = tt + NT * m;
            if (c4 < nc4) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(P.Gplus32) + c4);
                part = fmaf(w4[m].x, v.x, part);
                part = fmaf(w4[m].y, v.y, part);
                part = fmaf(w4[m].z, v.z, part);
                part = fmaf(w4[m].w, v.w, part);
            }
        }
        // q_s = ℓ_s / rank, ℓ_s = hᵀG⁺h = lv 2^gexp (G⁺ stored scaled by 2^-gexp)
        const df lev = team_sum_df(part);
        const float lv = (lev.hi + lev.lo) / (float)P.rank[0];
        const int gexp = P.rank[1];
        const float w = ok ? ldexpf(1.0f / sqrtf((float)P.J * lv * ((gexp & 1) ? 2.f : 1.f)), -(gexp >> 1)) : 0.f;
        if (tt == 0) {
            P.weight[s] = w;
            if (P.logq) P.logq[s] = ok ? logf(lv) + (float)gexp * 0.6931471805599453f : -INFINITY;
        }
        if (P.SA)
            for (int a = tt; a < R; a += NT) P.SA[s * R + a] = w * th[a];
        team_sync();
    }
    if (!alive && tt == 0) {
        // a staged copy never completed: wait once more (bounded) so that no
        // copy into this CTA's shared memory is left in flight, then return
        tmb_wait(mbar, phase ^ 1u);
    }
}

template <int RMAX, int TEAM, int CTA_THREADS = 256, int MINB = 2>
cudaError_t launch_team_t(const FastParams& P, int num_sms, cudaStream_t st) {
    using C = TeamCfg<RMAX, TEAM, CTA_THREADS, MINB>;
    auto k = krp_descent_team<RMAX, TEAM, CTA_THREADS, MINB>;
    const int smem = C::TEAMS == 1 ? C::team_bytes(P.Tp) : C::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    // CTAs per SM: what the shared memory holds, up to the register design (MINB)
    const int per_sm = std::max(1, std::min(MINB, (228 * 1024) / (smem + 1024)));
    const int64_t need = (P.J + C::TEAMS - 1) / C::TEAMS;
    const int64_t grid = need < (int64_t)num_sms * per_sm ? need : (int64_t)num_sms * per_sm;
    k<<<(unsigned)grid, CTA_THREADS, smem, st>>>(P); count_launch();
    return cudaGetLastError();
}

}  // namespace

// 32 < R <= 128 path of the descent; false if R is outside it.
bool launch_descent_team(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err) {
    if (s->R <= 32 || s->R > 128) return false;
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
    // 64 < R <= 104: one team of 4 warps per 128-thread CTA, three CTAs per SM
    // (a stage of 3 Tp floats <= 65 KB); larger R: teams of 8 warps, two per SM
    if (s->R <= 64)
        *err = launch_team_t<64, 2>(P, s->num_sms, s->stream);
    else if (s->R <= 104)
        *err = launch_team_t<104, 4, 128, 3>(P, s->num_sms, s->stream);
    else
        *err = launch_team_t<128, 8>(P, s->num_sms, s->stream);
    return true;
}

}  // namespace krp
