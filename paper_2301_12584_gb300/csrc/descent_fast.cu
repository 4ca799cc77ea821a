// a4 + a5 (+ a6 fused) for R <= 32: the batched conditional descent with one
// warp per sample (Alg. 2 lines 6-12, loops exchanged as in App. A.6; Alg. 4
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
#include "common.cuh"
#include "internal.h"

#include <math.h>

namespace krp {

struct FastParams {
    const float* U[16];
    const float* tree[16];
    const float* etree[16];
    const float* Vhi[16];
    const float* Vlo[16];
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
    float* trace;
    int64_t n_trace;
};

constexpr int FAST_TRACE_STRIDE = 66;

template <int RMAX>
struct FastCfg {
    static constexpr int TPMAX = ((RMAX * (RMAX + 1) / 2) + 7) & ~7;
    static constexpr int NC4 = TPMAX / 4;           // float4 chunks per node
    static constexpr int NCH = (NC4 + 31) / 32;     // chunks per lane
    static constexpr int WARPS = 8;
    static constexpr int RPT = (4 * RMAX + 31) / 32;  // leaf rows per lane (F <= 4R)
};

template <int RMAX>
__global__ void __launch_bounds__(256, 2) krp_descent_fast(FastParams P) {
    using C = FastCfg<RMAX>;
    constexpr int NCH = C::NCH;
    __shared__ __align__(16) float4 s_w[C::WARPS][NCH * 32];
    __shared__ __align__(16) float s_hh[C::WARPS][RMAX];   // h, high parts
    __shared__ __align__(16) float s_hl[C::WARPS][RMAX];   // h, low parts
    __shared__ __align__(16) float s_th[C::WARPS][RMAX];   // FP32 h̃ for the leaf scan
    __shared__ uint8_t s_i[C::TPMAX], s_j[C::TPMAX];

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
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* sw = s_w[warp];
    float* hh = s_hh[warp];
    float* hl = s_hl[warp];
    float* th = s_th[warp];

    // weights of the packed entries for history vector x (FP32 values in smem)
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
            sw[c] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        }
        __syncwarp();
    };
    // masses of up to three nodes loaded together (each a double-float)
    auto mass3 = [&](const float* __restrict__ a, const float* __restrict__ b, const float* __restrict__ d, int nn,
                     df& ma, df& mb, df& md) {
        float4 va[NCH], vb[NCH], vd[NCH];
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const int c = lane + 32 * m;
            const bool ok = c < nc4;
            va[m] = ok ? __ldg(reinterpret_cast<const float4*>(a) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (nn > 1) {
                vb[m] = ok ? __ldg(reinterpret_cast<const float4*>(b) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                vd[m] = ok ? __ldg(reinterpret_cast<const float4*>(d) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float sa = 0.f, sb = 0.f, sd = 0.f;
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
            const float4 w = sw[lane + 32 * m];
            sa = fmaf(w.x, va[m].x, sa);
            sa = fmaf(w.y, va[m].y, sa);
            sa = fmaf(w.z, va[m].z, sa);
            sa = fmaf(w.w, va[m].w, sa);
            if (nn > 1) {
                sb = fmaf(w.x, vb[m].x, sb);
                sb = fmaf(w.y, vb[m].y, sb);
                sb = fmaf(w.z, vb[m].z, sb);
                sb = fmaf(w.w, vb[m].w, sb);
                sd = fmaf(w.x, vd[m].x, sd);
                sd = fmaf(w.y, vd[m].y, sd);
                sd = fmaf(w.z, vd[m].z, sd);
                sd = fmaf(w.w, vd[m].w, sd);
            }
        }
        ma = warp_sum_df(df{sa, 0.f});
        if (nn > 1) {
            mb = warp_sum_df(df{sb, 0.f});
            md = warp_sum_df(df{sd, 0.f});
        }
    };

    // One descent of Alg. 4 (row stage adds the leaf scan): returns the leaf
    // heap index; low is the double-float left edge of that leaf.
    auto descend = [&](const float* __restrict__ tr, int depth, int64_t Lk, int64_t nreal_rows, int F,
                       df tau, df& low, float* trc, float croot) -> int64_t {
        int64_t c = 1;
        int lvl = 0;
        float mnode = croot;
        while (lvl < depth) {
            const bool two = lvl + 2 <= depth;
            df mA, mB, mD;
            mass3(tr + c * Tp, tr + 2 * c * Tp, tr + (2 * c + 1) * Tp, two ? 3 : 1, mA, mB, mD);
            // level lvl at node c
            {
                const int64_t rfirst = ((2 * c + 1) << (depth - lvl - 1)) - Lk;
                const df cut = df_add(low, mA);
                if (trc) {
                    trc[2 + 2 * lvl] = mA.hi + mA.lo;
                    trc[3 + 2 * lvl] = mnode;
                }
                if (df_le(tau, cut) || rfirst * F >= nreal_rows) {
                    c = 2 * c;
                    mnode = mA.hi + mA.lo;
                    mA = mB;
                } else {
                    c = 2 * c + 1;
                    low = cut;
                    mnode = mnode - (mA.hi + mA.lo);
                    mA = mD;
                }
                ++lvl;
            }
            if (!two) break;
            // level lvl at the chosen child, its left-child mass already loaded
            {
                const int64_t rfirst = ((2 * c + 1) << (depth - lvl - 1)) - Lk;
                const df cut = df_add(low, mA);
                if (trc) {
                    trc[2 + 2 * lvl] = mA.hi + mA.lo;
                    trc[3 + 2 * lvl] = mnode;
                }
                if (df_le(tau, cut) || rfirst * F >= nreal_rows) {
                    c = 2 * c;
                    mnode = mA.hi + mA.lo;
                } else {
                    c = 2 * c + 1;
                    low = cut;
                    mnode = mnode - (mA.hi + mA.lo);
                }
                ++lvl;
            }
        }
        return c;
    };

    const int64_t warps_total = (int64_t)gridDim.x * C::WARPS;
    for (int64_t s = (int64_t)blockIdx.x * C::WARPS + warp; s < P.J; s += warps_total) {
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
            // ------------------------------------------------ eigencomponent stage
            if (lane < RMAX) th[lane] = hh[lane] + hl[lane];
            __syncwarp();
            make_weights(th);
            const float* et = P.etree[k];
            df Cm, dummy1, dummy2;
            mass3(et, nullptr, nullptr, 1, Cm, dummy1, dummy2);
            float cf = Cm.hi + Cm.lo;
            if (!(cf > 0.f) || !isfinite(cf)) {
                if (lane == 0) set_status(P.status, isfinite(cf) ? KRP_EZERO : KRP_ENUMERIC);
                ok = false;
                break;
            }
            if (trc) trc[0] = cf;
            df low{0.f, 0.f};
            int64_t c = descend(et, P.dE, P.Rp, R, 1, df_mul_f(Cm, u_eig), low, trc, cf);
            const int u = (int)(c - P.Rp);
            // ------------------------------------------------ row stage
            if (lane < RMAX) {
                float vh = 0.f, vl = 0.f;
                if (lane < R) {
                    vh = __ldg(P.Vhi[k] + (size_t)u * R + lane);
                    vl = __ldg(P.Vlo[k] + (size_t)u * R + lane);
                }
                // h̃ = h ∘ V[:,u] in double-float, rounded once to FP32
                const df t = df_add(df_mul_f(df{hh[lane], hl[lane]}, vh), df_mul_f(df{hh[lane], hl[lane]}, vl));
                th[lane] = t.hi + t.lo;
            }
            __syncwarp();
            make_weights(th);
            const float* tr = P.tree[k];
            mass3(tr, nullptr, nullptr, 1, Cm, dummy1, dummy2);
            cf = Cm.hi + Cm.lo;
            if (!(cf > 0.f) || !isfinite(cf)) {
                if (lane == 0) set_status(P.status, isfinite(cf) ? KRP_EZERO : KRP_ENUMERIC);
                ok = false;
                break;
            }
            if (trc) {
                trc += FAST_TRACE_STRIDE;
                trc[0] = cf;
            }
            const df tau = df_mul_f(Cm, u_row);
            low = df{0.f, 0.f};
            const int64_t Lk = P.L[k], Ik = P.I[k];
            const int F = P.F;
            c = descend(tr, P.depth[k], Lk, Ik, F, tau, low, trc, cf);
            // ------------------------------------------------ leaf scan
            const int64_t row0 = (c - Lk) * F;
            const int nrows = (int)min((int64_t)F, Ik - row0);
            const int rpt = (F + 31) >> 5;
            const float* Uk = P.U[k];
            float q[C::RPT];
            df run{0.f, 0.f};
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = lane * rpt + r;
                float d = 0.f;
                if (r < rpt && t < nrows) {
                    const float* row = Uk + (row0 + t) * R;
                    if ((R & 3) == 0) {
#pragma unroll 8
                        for (int a = 0; a < R; a += 4) {
                            const float4 x = __ldg(reinterpret_cast<const float4*>(row + a));
                            const float4 y = *reinterpret_cast<const float4*>(th + a);
                            d = fmaf(x.x, y.x, d);
                            d = fmaf(x.y, y.y, d);
                            d = fmaf(x.z, y.z, d);
                            d = fmaf(x.w, y.w, d);
                        }
                    } else {
                        for (int a = 0; a < R; ++a) d = fmaf(__ldg(row + a), th[a], d);
                    }
                }
                q[r] = d * d;
                run = df_add(run, df{q[r], 0.f});
            }
            // inclusive warp scan of the per-lane totals in double-float
            df inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float vh = __shfl_up_sync(0xffffffffu, inc.hi, o);
                const float vl = __shfl_up_sync(0xffffffffu, inc.lo, o);
                if (lane >= o) inc = df_add(df{vh, vl}, inc);
            }
            df cum{__shfl_up_sync(0xffffffffu, inc.hi, 1), __shfl_up_sync(0xffffffffu, inc.lo, 1)};
            if (lane == 0) cum = df{0.f, 0.f};
            cum = df_add(cum, low);
            // first row whose right edge low + cum reaches tau; else last row with weight
            int first = 0x7fffffff, lastpos = -1;
#pragma unroll
            for (int r = 0; r < C::RPT; ++r) {
                const int t = lane * rpt + r;
                if (r < rpt && t < nrows) {
                    cum = df_add(cum, df{q[r], 0.f});
                    if (first == 0x7fffffff && df_le(tau, cum)) first = t;
                    if (q[r] > 0.f) lastpos = t;
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
                const df nh = df_mul_f(df{hh[lane], hl[lane]}, __ldg(Uk + trow * R + lane));
                hh[lane] = nh.hi;
                hl[lane] = nh.lo;
            }
            if (lane == 0) P.idx[(int64_t)k * P.J + s] = (int32_t)trow;
            __syncwarp();
        }
        // ------------------------------------------------ epilogue
        if (lane < RMAX) th[lane] = hh[lane] + hl[lane];
        __syncwarp();
        make_weights(th);
        df lev, d1, d2;
        mass3(P.Gplus32, nullptr, nullptr, 1, lev, d1, d2);
        const float qs = (lev.hi + lev.lo) / (float)(*P.rank);
        const float w = ok ? 1.0f / sqrtf((float)P.J * qs) : 0.f;
        if (lane == 0) {
            P.weight[s] = w;
            if (P.logq) P.logq[s] = ok ? logf(qs) : -INFINITY;
        }
        if (P.SA && lane < R) P.SA[s * R + lane] = w * th[lane];
        __syncwarp();
    }
}

namespace {
template <int RMAX>
cudaError_t launch_fast_t(const FastParams& P, int num_sms, cudaStream_t st) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, krp_descent_fast<RMAX>, 256, 0);
    per_sm = per_sm > 0 ? per_sm : 1;
    const int64_t need = (P.J + 7) / 8;
    const int64_t grid = need < (int64_t)num_sms * per_sm ? need : (int64_t)num_sms * per_sm;
    krp_descent_fast<RMAX><<<(unsigned)grid, 256, 0, st>>>(P); count_launch();
    return cudaGetLastError();
}
}  // namespace

bool launch_descent_fast(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err) {
    if (s->R > 32) return false;
    FastParams P{};
    for (int k = 0; k < s->N; ++k) {
        P.U[k] = s->U[k];
        P.tree[k] = s->tree[k];
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
    if (s->R <= 8)
        *err = launch_fast_t<8>(P, s->num_sms, s->stream);
    else if (s->R <= 16)
        *err = launch_fast_t<16>(P, s->num_sms, s->stream);
    else
        *err = launch_fast_t<32>(P, s->num_sms, s->stream);
    return true;
}

}  // namespace krp
