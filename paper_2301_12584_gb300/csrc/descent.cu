// a4 + a5 (+ a6 fused): batched conditional descent (the sampling loop of Alg. 2, with
// the loops exchanged as in App. A.6 so all J samples are in flight; Alg. 4
// RowSample on E_k and Z_k; Eqs. first_dist and second_conditional_dist).
//
// A "team" of TEAM warps owns one sample at a time and walks every included
// factor k in ascending order:
//   u-stage: descend E_k (depth log2 Rp, leaf size 1) with node masses
//            m(v) = hᵀ P^v h, P^v = G^v ∘ G_k, target tau = u_eig * m(root);
//   t-stage: h̃ = h ∘ V_k[:, u], descend Z_k (depth d_k) with masses
//            m(v) = h̃ᵀ G^v h̃ (Y = [1]), then scan the leaf's <= F rows with
//            weights (U_k[t] · h̃)² (Lemma 3.2 point 3) and pick the first row
//            whose cumulative edge reaches tau;
//   update:  h ∘= U_k[t, :].
// Branch rule (Alg. 4): go left iff tau <= low + m(left child); a right child
// with no real rows (padding) is never entered.  Every thread of the team owns
// E packed-triangle entries p = tid + 32*TEAM*e; for a fixed history vector it
// precomputes w_p = h_i h_j (x2 off the diagonal), so each level is E
// coalesced loads, E FMAs and one team reduction — the node quadratic form of
// Alg. 4 with the symmetric triangle read once.
// Epilogue: ℓ_s = hᵀ G⁺ h, q_s = ℓ_s / rank, w_s = 1/sqrt(J q_s) (Sec. 2.1),
// and optionally SA[s,:] = w_s h (the gather, fused).
// Precision: the history h and h̃ are carried as double-float (FP32 pairs); the
// target tau and the running left edge `low` are double-float; each branch is
// decided on the FP32 mass unless tau lies within 1e-6 of the stage's root mass
// of the cutoff, and then on the team's double-float sum of the per-thread
// partials.  The leaf scan is redone in double-float in the same case.
#include "common.cuh"
#include "internal.h"

#include <math.h>

namespace krp {

struct DescentParams {
    const float* U[16];      // factor rows
    const float* tree[16];   // Z_k
    const float* etree[16];  // E_k
    const float* V32[16];    // eigenvectors of G_{>k}, row u
    const float* V32lo[16];  // their FP32 residuals (double-float eigenvectors)
    int64_t I[16];
    int64_t L[16];
    int depth[16];
    int incl[16];
    int n_incl;
    int R, F, T, Tp, Rp, dE;
    const float* Gplus32;
    const int* rank;
    int* status;
    uint32_t key0, key1, draw;
    int64_t J;
    int32_t* idx;
    float* weight;
    float* logq;
    float* SA;
    float* trace;   // optional: per traced sample, factor, stage: [root mass, (m_left, m_node) per level]
    int64_t n_trace;
};

constexpr int TRACE_STRIDE = 66;  // 1 root mass + 1 pad + 32 levels x (m_left, m_node)

template <int RMAX, int TEAM>
struct DescentCfg {
    static constexpr int THREADS = 32 * TEAM;
    static constexpr int TMAX = ((RMAX * (RMAX + 1) / 2) + 7) & ~7;
    static constexpr int E = (TMAX + THREADS - 1) / THREADS;
    static constexpr int TEAMS_PER_CTA = 256 / THREADS;
    static constexpr int RPT = (4 * RMAX + THREADS - 1) / THREADS;  // leaf rows per thread (F <= 4R)
};

template <int TEAM>
struct TeamSync {
    __device__ static void sync(int team) {
        if (TEAM == 1)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(TEAM * 32) : "memory");
    }
};

template <int RMAX, int TEAM>
__global__ void __launch_bounds__(256) krp_descent(DescentParams P) {
    using C = DescentCfg<RMAX, TEAM>;
    constexpr int E = C::E;
    constexpr int NT = C::THREADS;
    __shared__ uint8_t s_i[C::TMAX], s_j[C::TMAX];
    __shared__ __align__(16) float s_h[C::TEAMS_PER_CTA][RMAX];
    __shared__ __align__(16) float s_hl[C::TEAMS_PER_CTA][RMAX];
    __shared__ __align__(16) float s_ht[C::TEAMS_PER_CTA][RMAX];
    __shared__ float s_red[C::TEAMS_PER_CTA][TEAM];
    __shared__ float s_red2[C::TEAMS_PER_CTA][TEAM][2];
    __shared__ float s_scan[C::TEAMS_PER_CTA][TEAM];
    __shared__ int s_pick[C::TEAMS_PER_CTA][2];

    const int R = P.R, T = P.T, Tp = P.Tp;
    for (int p = threadIdx.x; p < C::TMAX; p += blockDim.x) {
        int i = 0, rem = p;
        if (p < T) {
            while (rem >= R - i) {
                rem -= R - i;
                ++i;
            }
        }
        s_i[p] = (uint8_t)(p < T ? i : 0);
        s_j[p] = (uint8_t)(p < T ? i + rem : 0);
    }
    __syncthreads();

    const int team = threadIdx.x / NT;
    const int tid = threadIdx.x % NT;
    const int lane = threadIdx.x & 31;
    const int wib = tid >> 5;  // warp in team
    float* h = s_h[team];
    float* hl = s_hl[team];
    float* ht = s_ht[team];

    auto team_sum = [&](float v) -> float {
        v = warp_sum(v);
        if (TEAM == 1) return v;
        if (lane == 0) s_red[team][wib] = v;
        TeamSync<TEAM>::sync(team);
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < TEAM; ++w) t += s_red[team][w];
        TeamSync<TEAM>::sync(team);
        return t;
    };

    float wgt[E];
    auto make_weights = [&](const float* hv) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int p = tid + NT * e;
            float w = 0.f;
            if (p < T) {
                const int i = s_i[p], j = s_j[p];
                w = hv[i] * hv[j];
                if (i != j) w += w;
            }
            wgt[e] = w;
        }
    };
    // Team double-float sum of per-thread FP32 partials (identical in every thread).
    auto team_sum_df = [&](float part) -> df {
        df v = warp_sum_df(df{part, 0.f});
        if (TEAM == 1) return v;
        if (lane == 0) {
            s_red2[team][wib][0] = v.hi;
            s_red2[team][wib][1] = v.lo;
        }
        TeamSync<TEAM>::sync(team);
        df t{0.f, 0.f};
#pragma unroll
        for (int w = 0; w < TEAM; ++w) t = df_add(t, df{s_red2[team][w][0], s_red2[team][w][1]});
        TeamSync<TEAM>::sync(team);
        return t;
    };
    auto node_part = [&](const float* __restrict__ node) -> float {
        float acc = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int p = tid + NT * e;
            if (p < Tp) acc = fmaf(wgt[e], __ldg(node + p), acc);
        }
        return acc;
    };
    // "tau <= low + m" (Alg. 4): FP32 mass unless tau is within `margin` of the
    // cutoff, then the double-float mass.  Every operand is team-uniform.
    auto go_left = [&](df tau, df low, float m, float part, float margin, df& cut) -> bool {
        cut = df_add(low, df{m, 0.f});
        const df gap = df_add(tau, df_neg(cut));
        if (fabsf(gap.hi) > margin) return gap.hi < 0.f;
        cut = df_add(low, team_sum_df(part));
        return df_le(tau, cut);
    };

    const int64_t total_teams = (int64_t)gridDim.x * C::TEAMS_PER_CTA;
    for (int64_t s = (int64_t)blockIdx.x * C::TEAMS_PER_CTA + team; s < P.J; s += total_teams) {
        for (int a = tid; a < RMAX; a += NT) {
            h[a] = (a < R) ? 1.f : 0.f;
            hl[a] = 0.f;
        }
        TeamSync<TEAM>::sync(team);
        bool ok = true;
        for (int pi = 0; pi < P.n_incl; ++pi) {
            const int k = P.incl[pi];
            const uint4 rnd = philox4x32_10(make_uint4((uint32_t)s, P.draw, (uint32_t)pi, 0u),
                                            make_uint2(P.key0, P.key1));
            const float u_eig = u32_to_unit(rnd.x), u_row = u32_to_unit(rnd.y);
            // ---------------- eigencomponent stage (E_k, leaf size 1)
            make_weights(h);
            const float* et = P.etree[k];
            df Cd = team_sum_df(node_part(et));
            float Cm = Cd.hi + Cd.lo;
            if (!(Cm > 0.f) || !isfinite(Cm)) {
                if (tid == 0) set_status(P.status, isfinite(Cm) ? KRP_EZERO : KRP_ENUMERIC);
                ok = false;
                break;
            }
            df tau = df_mul_f(Cd, u_eig), low{0.f, 0.f}, cut;
            float margin = 1e-6f * Cm;
            int64_t c = 1;
            float* trc = (P.trace && s < P.n_trace && tid == 0)
                             ? P.trace + ((s * P.n_incl + pi) * 2 + 0) * TRACE_STRIDE
                             : nullptr;
            float mnode = Cm;
            if (trc) trc[0] = Cm;
            for (int lvl = 0; lvl < P.dE; ++lvl) {
                const float part = node_part(et + c * Tp);
                const float mL = team_sum(part);
                if (trc) {
                    trc[2 + 2 * lvl] = mL;
                    trc[3 + 2 * lvl] = mnode;
                }
                const int64_t rfirst = ((2 * c + 1) << (P.dE - lvl - 1)) - P.Rp;  // first leaf of right child
                if (rfirst >= R || go_left(tau, low, mL, part, margin, cut)) {
                    c = 2 * c;
                    mnode = mL;
                } else {
                    c = 2 * c + 1;
                    low = cut;
                    mnode = mnode - mL;
                }
            }
            const int u = (int)(c - P.Rp);
            // ---------------- row stage (Z_k, leaf size F, Y = [1])
            const float* Vu = P.V32[k] + (size_t)u * R;
            const float* Vul = P.V32lo[k] + (size_t)u * R;
            for (int a = tid; a < RMAX; a += NT) {
                float v = 0.f;
                if (a < R) {  // h̃ = h ∘ V[:,u] from double-float factors, rounded once
                    const df hd{h[a], hl[a]};
                    const df t = df_add(df_mul_f(hd, __ldg(Vu + a)), df_mul_f(hd, __ldg(Vul + a)));
                    v = t.hi + t.lo;
                }
                ht[a] = v;
            }
            TeamSync<TEAM>::sync(team);
            make_weights(ht);
            const float* tr = P.tree[k];
            Cd = team_sum_df(node_part(tr));
            Cm = Cd.hi + Cd.lo;
            if (!(Cm > 0.f) || !isfinite(Cm)) {
                if (tid == 0) set_status(P.status, isfinite(Cm) ? KRP_EZERO : KRP_ENUMERIC);
                ok = false;
                break;
            }
            tau = df_mul_f(Cd, u_row);
            low = df{0.f, 0.f};
            margin = 1e-6f * Cm;
            c = 1;
            const int64_t Lk = P.L[k], Ik = P.I[k];
            const int dk = P.depth[k];
            const int F = P.F;
            if (trc) trc += TRACE_STRIDE;
            mnode = Cm;
            if (trc) trc[0] = Cm;
            for (int lvl = 0; lvl < dk; ++lvl) {
                const float part = node_part(tr + c * Tp);
                const float mL = team_sum(part);
                const int64_t rfirst = ((2 * c + 1) << (dk - lvl - 1)) - Lk;
                if (trc) {
                    trc[2 + 2 * lvl] = mL;
                    trc[3 + 2 * lvl] = mnode;
                }
                if (rfirst * F >= Ik || go_left(tau, low, mL, part, margin, cut)) {
                    c = 2 * c;
                    mnode = mL;
                } else {
                    c = 2 * c + 1;
                    low = cut;
                    mnode = mnode - mL;
                }
            }
            // leaf scan: rows [row0, row0 + nrows)
            const int64_t row0 = (c - Lk) * F;
            const int nrows = (int)min((int64_t)F, Ik - row0);
            const float* Uk = P.U[k];
            const int rpt = (F + NT - 1) / NT;  // rows per thread, <= C::RPT since F <= 4R
            float q[C::RPT];
            float run = 0.f;
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = tid * rpt + r;
                float d = 0.f;
                if (r < rpt && t < nrows) {
                    const float* row = Uk + (row0 + t) * R;
                    if ((R & 3) == 0) {
                        for (int a = 0; a < R; a += 4) {
                            const float4 x = __ldg(reinterpret_cast<const float4*>(row + a));
                            const float4 y = *reinterpret_cast<const float4*>(ht + a);
                            d = fmaf(x.x, y.x, d);
                            d = fmaf(x.y, y.y, d);
                            d = fmaf(x.z, y.z, d);
                            d = fmaf(x.w, y.w, d);
                        }
                    } else {
                        for (int a = 0; a < R; ++a) d = fmaf(__ldg(row + a), ht[a], d);
                    }
                }
                q[r] = (r < rpt && t < nrows) ? d * d : 0.f;
                run += q[r];
            }
            // team exclusive scan of the per-thread totals (FP32)
            float incl_scan = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float v = __shfl_up_sync(0xffffffffu, incl_scan, o);
                if (lane >= o) incl_scan += v;
            }
            float base = __shfl_up_sync(0xffffffffu, incl_scan, 1);
            if (lane == 0) base = 0.f;
            if (TEAM > 1) {
                if (lane == 31) s_scan[team][wib] = incl_scan;
                TeamSync<TEAM>::sync(team);
                float off = 0.f;
                for (int w = 0; w < wib; ++w) off += s_scan[team][w];
                base += off;
                TeamSync<TEAM>::sync(team);
            }
            // first row whose right edge low + cum reaches tau; else the last row with weight > 0
            const df rel = df_add(tau, df_neg(low));
            const float target = rel.hi + rel.lo;
            int first = 0x7fffffff, lastpos = -1;
            bool near = false;
            float cum = base;
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = tid * rpt + r;
                if (r < rpt && t < nrows) {
                    cum += q[r];
                    if (first == 0x7fffffff && target <= cum) first = t;
                    if (fabsf(cum - target) <= margin) near = true;
                    if (q[r] > 0.f) lastpos = t;
                }
            }
            int any_near = __any_sync(0xffffffffu, near) ? 1 : 0;
            if (TEAM > 1) {
                if (tid == 0) s_pick[team][0] = 0;
                TeamSync<TEAM>::sync(team);
                if (lane == 0 && any_near) atomicOr(&s_pick[team][0], 1);
                TeamSync<TEAM>::sync(team);
                any_near = s_pick[team][0];
                TeamSync<TEAM>::sync(team);
            }
            if (any_near) {
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
                        s_red2[team][wib][0] = incd.hi;
                        s_red2[team][wib][1] = incd.lo;
                    }
                    TeamSync<TEAM>::sync(team);
                    df off{0.f, 0.f};
                    for (int w = 0; w < wib; ++w) off = df_add(off, df{s_red2[team][w][0], s_red2[team][w][1]});
                    cd = df_add(off, cd);
                    TeamSync<TEAM>::sync(team);
                }
                cd = df_add(cd, low);
                first = 0x7fffffff;
#pragma unroll
                for (int r = 0; r < C::RPT; ++r) {
                    const int t = tid * rpt + r;
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
                if (tid == 0) {
                    s_pick[team][0] = 0x7fffffff;
                    s_pick[team][1] = -1;
                }
                TeamSync<TEAM>::sync(team);
                if (lane == 0) {
                    atomicMin(&s_pick[team][0], first);
                    atomicMax(&s_pick[team][1], lastpos);
                }
                TeamSync<TEAM>::sync(team);
                first = s_pick[team][0];
                lastpos = s_pick[team][1];
                TeamSync<TEAM>::sync(team);
            }
            int t_sel = first != 0x7fffffff ? first : lastpos;
            if (t_sel < 0) {  // leaf with no positive weight: reached only through rounding
                if (tid == 0) set_status(P.status, KRP_ENUMERIC);
                t_sel = 0;
            }
            const int64_t trow = row0 + t_sel;
            for (int a = tid; a < R; a += NT) {
                const df nh = df_mul_f(df{h[a], hl[a]}, __ldg(Uk + trow * R + a));
                h[a] = nh.hi;
                hl[a] = nh.lo;
            }
            if (tid == 0) P.idx[(int64_t)k * P.J + s] = (int32_t)trow;
            TeamSync<TEAM>::sync(team);
        }
        // ---------------- epilogue: probability, weight, fused gather
        make_weights(h);
        // q_s = ℓ_s / rank, ℓ_s = hᵀG⁺h = lv 2^gexp (G⁺ stored scaled by 2^-gexp)
        const df levd = team_sum_df(node_part(P.Gplus32));
        const float lv = (levd.hi + levd.lo) / (float)P.rank[0];
        const int gexp = P.rank[1];
        const float w = ok ? ldexpf(1.0f / sqrtf((float)P.J * lv * ((gexp & 1) ? 2.f : 1.f)), -(gexp >> 1)) : 0.f;
        if (tid == 0) {
            P.weight[s] = w;
            if (P.logq) P.logq[s] = ok ? logf(lv) + (float)gexp * 0.6931471805599453f : -INFINITY;
        }
        if (P.SA)
            for (int a = tid; a < R; a += NT) P.SA[s * R + a] = w * h[a];
        TeamSync<TEAM>::sync(team);
    }
}

namespace {
template <int RMAX, int TEAM>
cudaError_t launch_descent_t(const DescentParams& P, int num_sms, cudaStream_t st) {
    using C = DescentCfg<RMAX, TEAM>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, krp_descent<RMAX, TEAM>, 256, 0);
    per_sm = per_sm > 0 ? per_sm : 1;
    const int64_t need = (P.J + C::TEAMS_PER_CTA - 1) / C::TEAMS_PER_CTA;
    const int64_t grid = need < (int64_t)num_sms * per_sm ? need : (int64_t)num_sms * per_sm;
    krp_descent<RMAX, TEAM><<<(unsigned)grid, 256, 0, st>>>(P); count_launch();
    return cudaGetLastError();
}
}  // namespace

krp_status launch_descent(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id,
                          int32_t* idx, float* weight, float* logq, float* SA, float* trace, int64_t n_trace) {
    cudaError_t fe = cudaSuccess;
    if (launch_descent_fast(s, exclude_j, J, seed, draw_id, idx, weight, logq, SA, trace, n_trace, &fe))
        return fe == cudaSuccess ? KRP_OK : cuda_check(s, fe, "descent launch");
    DescentParams P{};
    P.n_incl = 0;
    for (int k = 0; k < s->N; ++k) {
        P.U[k] = s->U[k];
        P.tree[k] = s->tree[k];
        P.etree[k] = s->etree + (size_t)k * s->Rp * s->Tp;
        P.V32[k] = s->V32 + (size_t)k * s->R * s->R;
        P.V32lo[k] = s->V32lo + (size_t)k * s->R * s->R;
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
    cudaError_t e;
    const int R = s->R;
    if (R <= 8)
        e = launch_descent_t<8, 1>(P, s->num_sms, s->stream);
    else if (R <= 16)
        e = launch_descent_t<16, 1>(P, s->num_sms, s->stream);
    else if (R <= 32)
        e = launch_descent_t<32, 1>(P, s->num_sms, s->stream);
    else if (R <= 64)
        e = launch_descent_t<64, 2>(P, s->num_sms, s->stream);
    else
        e = launch_descent_t<128, 8>(P, s->num_sms, s->stream);
    if (e != cudaSuccess) return cuda_check(s, e, "descent launch");
    return KRP_OK;
}

// ---------------------------------------------------------------------------
// a6: sampled-row gather SA[s,:] = w_s * prod_k U_k[idx[k][s], :]
// (warp per sample, lanes over columns).
// ---------------------------------------------------------------------------
struct GatherParams {
    const float* U[16];
    int incl[16];
    int n_incl;
    int R;
    int64_t J;
    const int32_t* idx;
    const float* weight;
    float* SA;
};

__global__ void __launch_bounds__(256) krp_gather_kernel(GatherParams P) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < P.J; s += warps) {
        const float w = P.weight[s];
        for (int a = lane; a < P.R; a += 32) {
            float v = w;
            for (int pi = 0; pi < P.n_incl; ++pi) {
                const int k = P.incl[pi];
                const int64_t row = P.idx[(int64_t)k * P.J + s];
                v *= __ldg(P.U[k] + row * P.R + a);
            }
            P.SA[s * P.R + a] = v;
        }
    }
}

krp_status launch_gather(krp_sampler* s, int exclude_j, int64_t J, const int32_t* idx, const float* weight,
                         float* SA) {
    GatherParams P{};
    for (int k = 0; k < s->N; ++k) {
        P.U[k] = s->U[k];
        if (k != exclude_j) P.incl[P.n_incl++] = k;
    }
    P.R = s->R;
    P.J = J;
    P.idx = idx;
    P.weight = weight;
    P.SA = SA;
    const int64_t need = (J + 7) / 8;
    const int64_t grid = need < (int64_t)s->num_sms * 8 ? need : (int64_t)s->num_sms * 8;
    krp_gather_kernel<<<(unsigned)grid, 256, 0, s->stream>>>(P); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "gather launch");
    return KRP_OK;
}

}  // namespace krp
