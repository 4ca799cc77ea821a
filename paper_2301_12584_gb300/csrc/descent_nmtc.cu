// f2 on the tensor cores: the node-major descent with every node's masses
// formed as a dense contraction H_v G_v on tcgen05 (the batched,
// level-synchronous sampling of App. A.10; the sampling loop of Alg. 2 with the
// loops exchanged as in App. A.6; Alg. 4 on E_k and Z_k; Eqs. first_dist and
// second_conditional_dist), for 32 < R <= 128 and leaves of F <= 128 rows.
//
// All J samples of a draw move through a tree one level at a time.  The
// samples that sit at the same node v form a group, kept contiguous in a
// permutation of the samples and cut into tiles of at most 128.  For a tile,
// the mass of v's left child 2v under sample s is x_sᵀ G_{2v} x_s (x_s = h for
// the eigencomponent tree E_k, h ∘ v_u for the factor's tree Z_k): with H the
// tile's 128 x R block of vectors, D = H G_{2v} (M = 128, N = R, K = R) runs on
// the tensor cores into tensor memory and m_s = Σ_j D[s, j] x_s[j] is read
// back.  At a leaf the same product with the leaf's rows, D = H U_leafᵀ, gives
// the rank-1 row weights (U[t] · x_s)² of Eq. second_conditional_dist, and each
// sample scans its row of D; after the last factor the leverage hᵀG⁺h of every
// sample (Sec. 2.1's q_s) is the same contraction with G⁺.
//
// Precision: split TF32 (TF32x3).  Every operand x = hi + lo (hi = tf32(x),
// lo = tf32(x - hi)); a product is hi hi' + hi lo' + lo hi', accumulated in
// FP32 in tensor memory (~2^-21 |x||y| per product).  A decision is taken in
// FP32 unless tau lies within 1e-6 C of the cutoff (the team kernel's band);
// then the left child's mass is formed again from the packed node (one warp
// per such sample: FP32 partials per lane, summed in double-float) and the
// cutoff compared in double-float.  The leaf scan re-runs its
// cumulative sum in double-float near an edge, as the team kernel does.
//
// After each level the samples are regrouped: a one-CTA scan over the tiles
// counts each group's left-goers and the next level's tiles, and a partition
// writes every sample into its child's range (left children first, order kept)
// together with the next level's tile list.  The host launches the fixed
// sequence of levels (the trees' depths); tile counts stay on the device, so a
// draw can be captured in a CUDA graph.  Every wait is bounded.
#include "common.cuh"
#include "internal.h"

#include <math.h>

#include <algorithm>

namespace krp {
namespace {

constexpr int NT_THREADS = 256;
constexpr int NT_WAIT_TRIES = 1 << 16;
constexpr float NT_MARGIN = 1e-6f;   // of the stage total C (the team kernel's band)
constexpr int NT_AQ = 8;             // A quads (float4) a thread loads before it stores any
constexpr int NT_BQ = 4;             // B quads likewise

// Tile of the level: positions [t0, t0 + n) of the permutation, all at node c;
// the node's group starts at position g0 and spans tiles [gt0, gt1).
struct TileRec {
    int t0, n, c, g0, gt0, gt1;
};

struct NtWs {  // workspace of a draw, carved from the sampler's buffer
    float* X;          // J x KP: the stage's vector x_s, zero padded
    float* hh;         // J x R: history h (double-float: hh + hl)
    float* hl;
    float* tau;        // 2 J: (hi, lo)
    float* low;        // 2 J
    float* mnode;      // J
    float* margin;     // J
    int* node;         // J: heap index of the current node
    int* ok;           // J: 0 once a stage total was zero or not finite
    int* perm[2];      // position -> sample
    unsigned char* left;   // per position: 1 if the sample went left
    TileRec* tiles[2];
    int* nleft;        // per tile
    int* lsum;         // per tile + 1: exclusive scan of nleft
    int* toff;         // per tile + 1: first next-level tile of the group
    int* ntiles;       // [2]
};

struct NtArgs {
    NtWs W;
    int cur;                 // which perm / tiles buffer is the current level's
    const float* tree;       // the stage's tree (slot stride Tp)
    const float* U;          // the factor's rows (leaf scan)
    int64_t L, nreal;        // leaves, real rows of the stage's tree
    int depth, F, lvl;
    int R, KP, NP, KC, Tp;
    int64_t J;
    int pi, k, sg;           // included-factor position, factor, stage (0: E_k, 1: Z_k)
    int n_incl;
    uint32_t key0, key1, draw;
    int32_t* idx;
    float* trace;
    int64_t n_trace;
    int* status;
    float* weight;           // the final stage's outputs
    float* logq;
    float* SA;
    const int* rank;         // rank(A) and the exponent of G⁺'s scale
};

__device__ __forceinline__ uint32_t nt_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start, leading byte offset
// between core matrices along K, stride byte offset between 8-row groups,
// version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t nt_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major, M = 128.
__device__ __forceinline__ uint32_t nt_idesc(int np) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void nt_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool nt_wait(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < NT_WAIT_TRIES; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(nt_saddr(bar)), "r"(parity), "r"(100000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void nt_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void nt_split(float x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// Operands are K-major with no swizzle: 8-row x 16-byte core matrices, the
// core matrices of an 8-row group adjacent along K (128 bytes apart), then the
// next 8-row group.  Element (p, k) of an operand with kw columns of K sits at
// byte (p / 8) (kw / 4) 128 + (k / 4) 128 + (p mod 8) 16 + (k mod 4) 4, so the
// 16-byte quad e = 8 ((p / 8) (kw / 4) + k / 4) + p mod 8 sits at byte 16 e.

// A sample id read from a permutation: always in [0, J) unless a level kernel
// gave up on a wait (its status then reports it) and left positions unwritten;
// the clamp keeps every later access in bounds.
__device__ __forceinline__ int nt_sample(int s, int64_t J) { return (uint32_t)s < (uint64_t)J ? s : 0; }

__device__ __forceinline__ float* nt_trace(const NtArgs& A, int s) {
    if (!A.trace || s >= A.n_trace) return nullptr;
    return A.trace + (((int64_t)s * A.n_incl + A.pi) * 2 + A.sg) * 66;
}

// ---------------------------------------------------------------------------
// Stage set-up, one warp per sample: the history update by the previous
// factor's row (E_k stage of factors after the first, and the final stage
// sg = 2 after the last factor), the stage's vector x_s (h for E_k and the
// final stage; h ∘ v_u, rounded once from double-float, for Z_k), the root as
// every sample's node, the identity permutation and the root level's tiles.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) nt_init(const __grid_constant__ NtArgs A, const float* __restrict__ Uprev,
                                               int kprev, const float* __restrict__ Vhi,
                                               const float* __restrict__ Vlo, int Rp) {
    const NtWs& W = A.W;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int R = A.R, KP = A.KP;
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < A.J; s += warps) {
        float* hh = W.hh + s * R;
        float* hl = W.hl + s * R;
        float* X = W.X + s * KP;
        if (A.sg != 1) {
            if (A.sg == 0 && A.pi == 0) {
                for (int a = lane; a < R; a += 32) {
                    hh[a] = 1.f;
                    hl[a] = 0.f;
                }
                if (lane == 0) W.ok[s] = 1;
            } else {
                const int64_t row = A.idx[(int64_t)kprev * A.J + s];
                for (int a = lane; a < R; a += 32) {
                    const df nh = df_mul_f(df{hh[a], hl[a]}, __ldg(Uprev + row * R + a));
                    hh[a] = nh.hi;
                    hl[a] = nh.lo;
                }
            }
            for (int a = lane; a < KP; a += 32) X[a] = a < R ? hh[a] + hl[a] : 0.f;
        } else {
            int u = W.node[s] - Rp;
            u = u < 0 ? 0 : (u >= R ? R - 1 : u);   // only a dead sample's node can be out of range
            for (int a = lane; a < KP; a += 32) {
                float x = 0.f;
                if (a < R) {
                    const float vh = __ldg(Vhi + (size_t)u * R + a), vl = __ldg(Vlo + (size_t)u * R + a);
                    const df h{hh[a], hl[a]};
                    const df t = df_add(df_mul_f(h, vh), df_mul_f(h, vl));
                    x = t.hi + t.lo;
                }
                X[a] = x;
            }
        }
        __syncwarp();   // every lane has read the node (u) before it is reset
        if (lane == 0) {
            W.node[s] = 1;
            W.perm[A.cur][s] = (int)s;
        }
    }
    const int64_t nt = (A.J + 127) / 128;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        TileRec rec;
        rec.t0 = (int)(128 * t);
        rec.n = (int)std::min<int64_t>(128, A.J - 128 * t);
        rec.c = 1;
        rec.g0 = 0;
        rec.gt0 = 0;
        rec.gt1 = (int)nt;
        W.tiles[A.cur][t] = rec;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) W.ntiles[A.cur] = (int)nt;
}

// ---------------------------------------------------------------------------
// One level for every tile: MODE 0 the stage total C = m(root) (tau = u C),
// MODE 1 the left child's mass and the decision of Alg. 4, MODE 2 the leaf
// scan (row weights, cumulative edges, first edge >= tau), MODE 3 the
// leverage hᵀG⁺h of the finished samples, their weights and sketch rows.
//
// Shared memory holds B (the node, or the leaf's rows: NP x KP, K-major hi
// and lo copies) and A (the tile's vectors, in chunks of KC columns of K when
// B leaves no room for all of them).  A CTA takes a contiguous run of tiles
// and keeps B while consecutive tiles share the node.  Both operands are
// written row-fastest, so that a warp's 16-byte stores fill 512 contiguous
// bytes of core matrices (no bank conflicts).
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(NT_THREADS, 1) nt_level(const __grid_constant__ NtArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float red[128];
    __shared__ float mAs[128];
    __shared__ int fixl[128];
    __shared__ unsigned char dirs[128];
    __shared__ int sperm[128];
    __shared__ int nfix;
    const NtWs& W = A.W;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = A.R, KP = A.KP, NP = A.NP, KC = A.KC;
    const bool a_whole = KC == KP;   // A holds all of K: the epilogue reads x_s from it
    unsigned char* Bh = smem;
    unsigned char* Bl = Bh + (size_t)NP * KP * 4;
    unsigned char* Ah = Bl + (size_t)NP * KP * 4;
    unsigned char* Al = Ah + (size_t)128 * KC * 4;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(nt_saddr(&tmem_base)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(nt_saddr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = nt_idesc(NP);
    const uint32_t sboB = (uint32_t)(KP >> 2) * 128u;
    uint32_t phase = 0;
    bool alive = true;
    const TileRec* tiles = W.tiles[A.cur];
    const int* perm = W.perm[A.cur];
    const int ntiles = W.ntiles[A.cur];
    const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int tb = (int)blockIdx.x * per, te = min(ntiles, tb + per);
    const int nkq = KP >> 2;
    const int q4 = warp & 3, hf = warp >> 2;
    const int r = 32 * q4 + lane;   // the tile row this thread reads back
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    int64_t bkey = -1;              // the node (or leaf) whose B is resident

    for (int ti = tb; ti < te && alive; ++ti) {
        const TileRec rec = tiles[ti];
        const int c = rec.c, n = rec.n, t0 = rec.t0;
        if (MODE == 1) {
            // an empty right child (padding leaves): every sample goes left
            const int64_t rfirst = (((int64_t)2 * c + 1) << (A.depth - A.lvl - 1)) - A.L;
            if (rfirst * A.F >= A.nreal) {
                if (tid < n) {
                    const int s = nt_sample(perm[t0 + tid], A.J);
                    const float mn = W.mnode[s];
                    W.node[s] = 2 * c;
                    W.left[t0 + tid] = 1;
                    if (float* trc = nt_trace(A, s)) {
                        trc[2 + 2 * A.lvl] = mn;
                        trc[3 + 2 * A.lvl] = mn;
                    }
                }
                if (tid == 0) W.nleft[ti] = n;
                continue;
            }
        }
        int64_t row0 = 0;
        int nrows = 0;
        if (MODE == 2) {
            row0 = ((int64_t)c - A.L) * A.F;
            nrows = (int)std::min<int64_t>(A.F, A.nreal - row0);
        }
        if (tid == 0) nfix = 0;
        if (tid < 128) sperm[tid] = tid < n ? nt_sample(perm[t0 + tid], A.J) : 0;
        __syncthreads();
        const int64_t key = (MODE == 1 || MODE == 2) ? c : 0;
        if (key != bkey) {
            // B: quad e holds row nn = 8 g + (e mod 8), K columns 4 kq .. 4 kq + 3;
            // each thread issues the loads of NT_BQ quads before it uses any
            const float* node = A.tree + (MODE == 1 ? (int64_t)c * A.Tp : 0);
            const int tot = NP * nkq;
            int kq0 = (tid >> 3) % nkq, g0 = (tid >> 3) / nkq;
            for (int e0 = tid; e0 < tot; e0 += NT_BQ * NT_THREADS) {
                float v[NT_BQ][4];
#pragma unroll
                for (int u = 0; u < NT_BQ; ++u) {
                    const int e = e0 + u * NT_THREADS;
                    const int nn = 8 * g0 + (tid & 7), k = 4 * kq0;
                    kq0 += 32;
                    while (kq0 >= nkq) {
                        kq0 -= nkq;
                        ++g0;
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int kk = k + t;
                        v[u][t] = 0.f;
                        if (e < tot && kk < R) {
                            if (MODE == 2) {
                                if (nn < nrows) v[u][t] = __ldg(A.U + (row0 + nn) * R + kk);
                            } else if (nn < R) {
                                v[u][t] = __ldg(node + (nn <= kk ? tri_index(nn, kk, R) : tri_index(kk, nn, R)));
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < NT_BQ; ++u) {
                    const int e = e0 + u * NT_THREADS;
                    if (e < tot) {
                        uint4 h, l;
                        nt_split(v[u][0], h.x, l.x);
                        nt_split(v[u][1], h.y, l.y);
                        nt_split(v[u][2], h.z, l.z);
                        nt_split(v[u][3], h.w, l.w);
                        reinterpret_cast<uint4*>(Bh)[e] = h;
                        reinterpret_cast<uint4*>(Bl)[e] = l;
                    }
                }
            }
            bkey = key;
        }
        // A in chunks of K (rows >= n read as zero), then the products of the chunk
        for (int k0 = 0, kc = 0; k0 < KP; k0 += KC, ++kc) {
            const int kw = KP - k0 < KC ? KP - k0 : KC, nq = kw >> 2;
            // rows of 8-row groups past the tile's last sample stay stale: their
            // rows of D are never read (rows of an MMA are independent)
            const int tot = 8 * nq * ((n + 7) >> 3);
            // quad e = tid + 256 u: row 8 (rest / nq) + tid mod 8, K quad rest mod nq,
            // rest = tid / 8 + 32 u (advanced by 32 per u without a division)
            int q = (tid >> 3) % nq, g = (tid >> 3) / nq;
            for (int e0 = tid; e0 < tot; e0 += NT_AQ * NT_THREADS) {
                float4 v[NT_AQ];
                int qq = q, gg = g;
#pragma unroll
                for (int u = 0; u < NT_AQ; ++u) {
                    const int e = e0 + u * NT_THREADS;
                    const int p = 8 * gg + (tid & 7);
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (e < tot && p < n)
                        v[u] = __ldg(reinterpret_cast<const float4*>(W.X + (int64_t)sperm[p] * KP + k0) + qq);
                    qq += 32;
                    while (qq >= nq) {
                        qq -= nq;
                        ++gg;
                    }
                }
                q = qq;
                g = gg;
#pragma unroll
                for (int u = 0; u < NT_AQ; ++u) {
                    const int e = e0 + u * NT_THREADS;
                    if (e < tot) {
                        uint4 h, l;
                        nt_split(v[u].x, h.x, l.x);
                        nt_split(v[u].y, h.y, l.y);
                        nt_split(v[u].z, h.z, l.z);
                        nt_split(v[u].w, h.w, l.w);
                        reinterpret_cast<uint4*>(Ah)[e] = h;
                        reinterpret_cast<uint4*>(Al)[e] = l;
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ah = nt_saddr(Ah), al = nt_saddr(Al), bh = nt_saddr(Bh), bl = nt_saddr(Bl);
                const uint32_t sboA = (uint32_t)nq * 128u;
                for (int ks = 0; ks < kw / 8; ++ks) {
                    const uint32_t ao = (uint32_t)ks * 256u, bo = (uint32_t)(k0 / 8 + ks) * 256u;
                    const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                    nt_mma(tmem, nt_desc(ah + ao, 128u, sboA), nt_desc(bh + bo, 128u, sboB), idesc, acc);
                    nt_mma(tmem, nt_desc(ah + ao, 128u, sboA), nt_desc(bl + bo, 128u, sboB), idesc, 1u);
                    nt_mma(tmem, nt_desc(al + ao, 128u, sboA), nt_desc(bh + bo, 128u, sboB), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 nt_saddr(&bar))
                             : "memory");
            }
            const bool ok = nt_wait(&bar, phase);
            alive = __syncthreads_and(ok) != 0;
            if (!alive) break;
            phase ^= 1u;
        }
        if (!alive) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (MODE != 2) {
            // m_s = Σ_j D[s, j] x_s[j]: warp w reads rows 32 (w mod 4) .. and
            // the column chunks w / 4, w / 4 + 2, ... of 32 (x_s zero padded to KP)
            const int sr = r < n ? sperm[r] : -1;
            const float4* xs = reinterpret_cast<const float4*>(W.X + (int64_t)(sr < 0 ? 0 : sr) * KP);
            float part = 0.f;
            for (int ch = hf; 32 * ch < NP; ch += 2) {
                float v[32];
                nt_ld32(tmem + lane_base + (uint32_t)(32 * ch), v);
                if (sr >= 0) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j0 = 32 * ch + 4 * q;
                        if (j0 < R) {
                            float4 x;
                            if (a_whole) {   // x = hi + lo from the A copies (quad of row r, K columns j0..)
                                const int e = 8 * ((r >> 3) * nkq + (j0 >> 2)) + (r & 7);
                                const uint4 h = reinterpret_cast<const uint4*>(Ah)[e];
                                const uint4 l = reinterpret_cast<const uint4*>(Al)[e];
                                x = make_float4(__uint_as_float(h.x) + __uint_as_float(l.x),
                                                __uint_as_float(h.y) + __uint_as_float(l.y),
                                                __uint_as_float(h.z) + __uint_as_float(l.z),
                                                __uint_as_float(h.w) + __uint_as_float(l.w));
                            } else {
                                x = __ldg(xs + (j0 >> 2));
                            }
                            part = fmaf(v[4 * q], x.x, part);
                            part = fmaf(v[4 * q + 1], x.y, part);
                            part = fmaf(v[4 * q + 2], x.z, part);
                            part = fmaf(v[4 * q + 3], x.w, part);
                        }
                    }
                }
            }
            if (hf == 1) red[r] = part;
            __syncthreads();
            if (hf == 0 && r < n) {
                const float m = part + red[r];
                const int s = sr;
                if (MODE == 0) {
                    float* trc = nt_trace(A, s);
                    const uint4 rnd = philox4x32_10(make_uint4((uint32_t)s, A.draw, (uint32_t)A.pi, 0u),
                                                    make_uint2(A.key0, A.key1));
                    const float uu = u32_to_unit(A.sg ? rnd.y : rnd.x);
                    float C = m;
                    if (!(C > 0.f) || !isfinite(C)) {
                        if (W.ok[s]) set_status(A.status, isfinite(C) ? KRP_EZERO : KRP_ENUMERIC);
                        W.ok[s] = 0;
                        C = 1.f;
                    }
                    const df tau = df_mul_f(df{C, 0.f}, uu);
                    W.tau[2 * s] = tau.hi;
                    W.tau[2 * s + 1] = tau.lo;
                    W.low[2 * s] = 0.f;
                    W.low[2 * s + 1] = 0.f;
                    W.mnode[s] = C;
                    W.margin[s] = NT_MARGIN * C;
                    if (trc) trc[0] = C;
                } else if (MODE == 3) {
                    // q_s = ℓ_s / rank, ℓ_s = hᵀG⁺h = lv 2^gexp (G⁺ stored scaled by 2^-gexp)
                    const int gexp = A.rank[1];
                    const bool okd = W.ok[s] != 0;
                    const float lv = m / (float)A.rank[0];
                    const float w =
                        okd ? ldexpf(1.0f / sqrtf((float)A.J * lv * ((gexp & 1) ? 2.f : 1.f)), -(gexp >> 1)) : 0.f;
                    A.weight[s] = w;
                    if (A.logq) A.logq[s] = okd ? logf(lv) + (float)gexp * 0.6931471805599453f : -INFINITY;
                    mAs[r] = w;
                } else {
                    float* trc = nt_trace(A, s);
                    const float mn = W.mnode[s];
                    mAs[r] = m;
                    if (trc) {
                        trc[2 + 2 * A.lvl] = m;
                        trc[3 + 2 * A.lvl] = mn;
                    }
                    int dir = 1;
                    if (W.ok[s]) {
                        const float gap = (W.tau[2 * s] - W.low[2 * s]) - m;
                        if (fabsf(gap) > W.margin[s])
                            dir = gap < 0.f ? 1 : 0;
                        else
                            dir = -1;
                    }
                    if (dir < 0) {
                        fixl[atomicAdd(&nfix, 1)] = r;
                    } else {
                        dirs[r] = (unsigned char)dir;
                        if (dir) {
                            W.node[s] = 2 * c;
                            W.mnode[s] = m;
                        } else {
                            const df cut = df_add(df{W.low[2 * s], W.low[2 * s + 1]}, df{m, 0.f});
                            W.node[s] = 2 * c + 1;
                            W.low[2 * s] = cut.hi;
                            W.low[2 * s + 1] = cut.lo;
                            W.mnode[s] = mn - m;
                        }
                    }
                }
            }
            if (MODE == 3 && A.SA) {
                // the sketch rows w_s h (the final stage keeps samples in order: s = t0 + row)
                __syncthreads();
                for (int e = tid; e < n * R; e += NT_THREADS) {
                    const int rr = e / R, a = e - rr * R;
                    const int64_t s = t0 + rr;
                    A.SA[s * R + a] = mAs[rr] * W.X[s * KP + a];
                }
            }
            if (MODE == 1) {
                __syncthreads();
                // near an edge: the left child's mass again in double-float from
                // the packed node, one warp per sample
                const int nf = nfix;
                const float* node = A.tree + (int64_t)c * A.Tp;
                for (int f = warp; f < nf; f += NT_THREADS / 32) {
                    const int rr = fixl[f];
                    const int s = sperm[rr];
                    const float* xs = W.X + (int64_t)s * KP;
                    // FP32 partial per lane over its entries, summed in double-float
                    // across the warp (the team kernel's near-edge arithmetic)
                    float acc = 0.f;
                    for (int i = 0; i < R; ++i) {
                        const float xi = xs[i];
                        const int base = tri_index(i, i, R);
                        for (int j = i + lane; j < R; j += 32) {
                            float w = xi * xs[j];
                            if (j != i) w += w;
                            acc = fmaf(w, __ldg(node + base + (j - i)), acc);
                        }
                    }
                    const df mass = warp_sum_df(df{acc, 0.f});
                    if (lane == 0) {
                        const float m = mAs[rr], mn = W.mnode[s];
                        const df low{W.low[2 * s], W.low[2 * s + 1]};
                        const df cut = df_add(low, mass);
                        const bool lft = df_le(df{W.tau[2 * s], W.tau[2 * s + 1]}, cut);
                        dirs[rr] = lft ? 1 : 0;
                        if (lft) {
                            W.node[s] = 2 * c;
                            W.mnode[s] = m;
                        } else {
                            W.node[s] = 2 * c + 1;
                            W.low[2 * s] = cut.hi;
                            W.low[2 * s + 1] = cut.lo;
                            W.mnode[s] = mn - m;
                        }
                    }
                }
                __syncthreads();
                const bool isl = tid < n && dirs[tid] != 0;
                if (tid < n) W.left[t0 + tid] = isl ? 1 : 0;
                const int cnt = __syncthreads_count(isl);
                if (tid == 0) W.nleft[ti] = cnt;
            }
        } else {
            // leaf scan: thread r of warps 0-3 owns sample r's row of D
            if (hf == 0) {
                const bool mine = r < n;
                const int s = mine ? sperm[r] : 0;
                df tau{0.f, 0.f}, low{0.f, 0.f};
                float target = 0.f, mg = 0.f;
                if (mine) {
                    tau = df{W.tau[2 * s], W.tau[2 * s + 1]};
                    low = df{W.low[2 * s], W.low[2 * s + 1]};
                    const df rel = df_add(tau, df_neg(low));
                    target = rel.hi + rel.lo;
                    mg = W.margin[s];
                }
                float cum = 0.f;
                int first = 0x7fffffff, lastpos = -1;
                bool near = false;
                for (int ch = 0; 32 * ch < NP; ++ch) {
                    float v[32];
                    nt_ld32(tmem + lane_base + (uint32_t)(32 * ch), v);
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int t = 32 * ch + q;
                        if (mine && t < nrows) {
                            const float w = v[q] * v[q];
                            cum += w;
                            if (first == 0x7fffffff && target <= cum) first = t;
                            if (fabsf(cum - target) <= mg) near = true;
                            if (w > 0.f) lastpos = t;
                        }
                    }
                }
                if (__any_sync(0xffffffffu, near)) {
                    // the cumulative edges again in double-float
                    df cd = low;
                    int f2 = 0x7fffffff;
                    for (int ch = 0; 32 * ch < NP; ++ch) {
                        float v[32];
                        nt_ld32(tmem + lane_base + (uint32_t)(32 * ch), v);
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const int t = 32 * ch + q;
                            if (near && t < nrows) {
                                cd = df_add(cd, df{v[q] * v[q], 0.f});
                                if (f2 == 0x7fffffff && df_le(tau, cd)) f2 = t;
                            }
                        }
                    }
                    if (near) first = f2;
                }
                if (mine) {
                    int t_sel = first != 0x7fffffff ? first : lastpos;
                    if (t_sel < 0) {   // no positive weight in the leaf: only through rounding
                        if (W.ok[s]) set_status(A.status, KRP_ENUMERIC);
                        t_sel = 0;
                    }
                    A.idx[(int64_t)A.k * A.J + s] = (int32_t)(row0 + t_sel);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // the accumulator and the A operand are reused by the next tile
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!alive) {
        if (tid == 0) nt_wait(&bar, phase);   // a product may still be in flight: one more bounded wait
        __syncthreads();
        if (tid == 0) set_status(A.status, KRP_ETIMEOUT);
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
    }
}

// Exclusive scan over a 1024-thread block; returns the thread's offset, *total the sum.
__device__ __forceinline__ int nt_block_scan(int v, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int x = wsum[lane];
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        wsum[lane] = xi - x;
        if (lane == 31) wsum[32] = xi;
    }
    __syncthreads();
    const int off = wsum[warp] + inc - v;
    *total = wsum[32];
    __syncthreads();
    return off;
}

// One CTA: lsum = exclusive scan of the tiles' left counts, then per group
// (at its first tile) the next level's tile count, scanned into toff, and the
// next level's tile total.
__global__ void __launch_bounds__(1024) nt_scan(const __grid_constant__ NtArgs A) {
    __shared__ int wsum[33];
    const NtWs& W = A.W;
    const int nt = W.ntiles[A.cur];
    const TileRec* tiles = W.tiles[A.cur];
    const int per = (nt + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(nt, b + per);
    int local = 0;
    for (int i = b; i < e; ++i) local += W.nleft[i];
    int total;
    int run = nt_block_scan(local, wsum, &total);
    for (int i = b; i < e; ++i) {
        W.lsum[i] = run;
        run += W.nleft[i];
    }
    if (threadIdx.x == 0) W.lsum[nt] = total;
    __syncthreads();
    local = 0;
    for (int i = b; i < e; ++i) {
        const TileRec rec = tiles[i];
        int cnt = 0;
        if (rec.gt0 == i) {
            const TileRec last = tiles[rec.gt1 - 1];
            const int ng = last.t0 + last.n - rec.g0;
            // within [0, ng] always, unless a level kernel gave up on a wait (its
            // status is then set): the clamp keeps the next level's tiles in bounds
            const int nl = min(max(W.lsum[rec.gt1] - W.lsum[rec.gt0], 0), ng);
            cnt = (nl + 127) / 128 + (ng - nl + 127) / 128;
        }
        W.toff[i] = cnt;
        local += cnt;
    }
    run = nt_block_scan(local, wsum, &total);
    for (int i = b; i < e; ++i) {
        const int cnt = W.toff[i];
        W.toff[i] = run;
        run += cnt;
    }
    if (threadIdx.x == 0) W.ntiles[A.cur ^ 1] = total;
}

// Partition: every sample to its child's range (left-goers of a group first,
// order kept within each side), and the next level's tiles, written by the
// CTA that holds the group's first tile.
__global__ void __launch_bounds__(128) nt_part(const __grid_constant__ NtArgs A) {
    __shared__ int wtot[4];
    const NtWs& W = A.W;
    const int nt = W.ntiles[A.cur];
    const TileRec* tiles = W.tiles[A.cur];
    const int* pin = W.perm[A.cur];
    int* pout = W.perm[A.cur ^ 1];
    TileRec* tout = W.tiles[A.cur ^ 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
        const TileRec rec = tiles[ti];
        const int p = rec.t0 + tid;
        const int l = tid < rec.n ? W.left[p] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, l);
        if (lane == 0) wtot[warp] = __popc(bal);
        __syncthreads();
        int pre = __popc(bal & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) pre += wtot[w];
        const TileRec last = tiles[rec.gt1 - 1];
        const int ng = last.t0 + last.n - rec.g0;
        const int lbase = W.lsum[rec.gt0];
        const int nl = min(max(W.lsum[rec.gt1] - lbase, 0), ng);   // as in nt_scan
        if (tid < rec.n) {
            const int lb = W.lsum[ti] - lbase + pre;   // left-goers of the group before p
            const int np = l ? rec.g0 + lb : rec.g0 + nl + (p - rec.g0 - lb);
            if (np >= rec.g0 && np < rec.g0 + ng) pout[np] = pin[p];   // always, unless a wait gave up
        }
        if (rec.gt0 == ti) {
            const int nr = ng - nl;
            const int nlt = (nl + 127) / 128, nrt = (nr + 127) / 128, base = W.toff[ti];
            for (int j = tid; j < nlt + nrt; j += blockDim.x) {
                TileRec o;
                if (j < nlt) {
                    o.t0 = rec.g0 + 128 * j;
                    o.n = min(128, nl - 128 * j);
                    o.c = 2 * rec.c;
                    o.g0 = rec.g0;
                    o.gt0 = base;
                    o.gt1 = base + nlt;
                } else {
                    const int jj = j - nlt;
                    o.t0 = rec.g0 + nl + 128 * jj;
                    o.n = min(128, nr - 128 * jj);
                    o.c = 2 * rec.c + 1;
                    o.g0 = rec.g0 + nl;
                    o.gt0 = base + nlt;
                    o.gt1 = base + nlt + nrt;
                }
                tout[base + j] = o;
            }
        }
        __syncthreads();
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of the workspace for J samples; carves it when base != null.
size_t nt_carve(char* base, int64_t J, int R, int KP, NtWs* W) {
    const int64_t ntmax = J + J / 128 + 2;
    size_t o = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + o : nullptr;
        o += align256(bytes);
        return p;
    };
    NtWs w;
    w.X = (float*)take((size_t)J * KP * 4);
    w.hh = (float*)take((size_t)J * R * 4);
    w.hl = (float*)take((size_t)J * R * 4);
    w.tau = (float*)take((size_t)J * 8);
    w.low = (float*)take((size_t)J * 8);
    w.mnode = (float*)take((size_t)J * 4);
    w.margin = (float*)take((size_t)J * 4);
    w.node = (int*)take((size_t)J * 4);
    w.ok = (int*)take((size_t)J * 4);
    w.perm[0] = (int*)take((size_t)J * 4);
    w.perm[1] = (int*)take((size_t)J * 4);
    w.left = (unsigned char*)take((size_t)J);
    w.tiles[0] = (TileRec*)take((size_t)ntmax * sizeof(TileRec));
    w.tiles[1] = (TileRec*)take((size_t)ntmax * sizeof(TileRec));
    w.nleft = (int*)take((size_t)ntmax * 4);
    w.lsum = (int*)take((size_t)(ntmax + 1) * 4);
    w.toff = (int*)take((size_t)(ntmax + 1) * 4);
    w.ntiles = (int*)take(2 * 4);
    if (W) *W = w;
    return o;
}

constexpr size_t NT_SMEM_MAX = 227 * 1024 - 2048;   // dynamic shared memory a CTA may take

size_t nt_smem(int KP, int NP, int KC) { return (size_t)2 * NP * KP * 4 + (size_t)2 * 128 * KC * 4; }

// The K chunk of A and the CTAs per SM: two CTAs per SM if some chunk fits
// half the shared memory, else one with the widest chunk that fits.
bool nt_geometry(int KP, int NP, int* KC, int* per_sm) {
    const int cands[3] = {KP, 64, 32};
    for (int want = 2; want >= 1; --want)
        for (int ci = 0; ci < 3; ++ci) {
            const int kc = std::min(cands[ci], KP);
            if (nt_smem(KP, NP, kc) <= (want == 2 ? NT_SMEM_MAX / 2 - 1024 : NT_SMEM_MAX)) {
                *KC = kc;
                *per_sm = want;
                return true;
            }
        }
    return false;
}

template <int MODE>
cudaError_t nt_launch_level(const NtArgs& A, int per_sm, int num_sms, cudaStream_t st) {
    const size_t sm = nt_smem(A.KP, A.NP, A.KC);
    auto k = nt_level<MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // per_sm comes from the operands' shared memory (the registers allow two
    // CTAs); the occupancy query answers one here, and a grid of one CTA per SM
    // measured 1.5x slower at R = 64
    k<<<(unsigned)(num_sms * per_sm), NT_THREADS, sm, st>>>(A);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

// The tensor-core node-major form; false (the caller takes another form) if
// R is outside 32 < R <= 128, a leaf holds more than 128 rows, a tree has
// more than 2^29 leaves, or the workspace cannot be had (no allocation while
// a graph is being captured).
bool launch_descent_nmtc(krp_sampler* s, int exclude_j, int64_t J, uint64_t seed, uint64_t draw_id, int32_t* idx,
                         float* weight, float* logq, float* SA, float* trace, int64_t n_trace, cudaError_t* err) {
    const int R = s->R;
    if (R <= 32 || R > 128 || s->F > 128 || J < 1 || J > ((int64_t)1 << 30)) return false;
    for (int k = 0; k < s->N; ++k)
        if (s->L[k] > ((int64_t)1 << 29)) return false;
    const int KP = (R + 7) & ~7, NPn = (R + 15) & ~15, NPl = (s->F + 15) & ~15;
    int KCn = 0, KCl = 0, psn = 0, psl = 0;
    if (!nt_geometry(KP, NPn, &KCn, &psn) || !nt_geometry(KP, NPl, &KCl, &psl))
        return false;
    const size_t need = nt_carve(nullptr, J, R, KP, nullptr);
    if (need > s->nm_ws_bytes) {
        if (s->capturing) return false;
        cudaFree(s->nm_ws);
        s->nm_ws = nullptr;
        s->nm_ws_bytes = 0;
        if (cudaMalloc((void**)&s->nm_ws, need) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        s->nm_ws_bytes = need;
    }
    NtArgs A{};
    nt_carve(s->nm_ws, J, R, KP, &A.W);
    A.R = R;
    A.KP = KP;
    A.Tp = s->Tp;
    A.J = J;
    A.key0 = (uint32_t)(seed & 0xffffffffu);
    A.key1 = (uint32_t)(seed >> 32);
    A.draw = (uint32_t)(draw_id & 0xffffffffu);
    A.idx = idx;
    A.trace = trace;
    A.n_trace = trace ? n_trace : 0;
    A.status = s->status;
    A.weight = weight;
    A.logq = logq;
    A.SA = SA;
    A.rank = s->rank_dev;
    int incl[16], n_incl = 0;
    for (int k = 0; k < s->N; ++k)
        if (k != exclude_j) incl[n_incl++] = k;
    A.n_incl = n_incl;
    const int ns = s->num_sms;
    const int64_t init_blocks = std::min<int64_t>((J + 7) / 8, (int64_t)ns * 8);
    const int64_t part_blocks = (int64_t)ns * 8;
    cudaStream_t st = s->stream;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
        return e == cudaSuccess;
    };
    A.cur = 0;
    for (int pi = 0; pi < n_incl && e == cudaSuccess; ++pi) {
        const int k = incl[pi];
        A.pi = pi;
        A.k = k;
        for (int sg = 0; sg < 2 && e == cudaSuccess; ++sg) {
            A.sg = sg;
            A.lvl = 0;
            if (sg == 0) {
                A.tree = s->etree + (size_t)k * s->Rp * s->Tp;
                A.L = s->Rp;
                A.nreal = R;
                A.depth = s->dE;
                A.F = 1;
            } else {
                A.tree = s->tree[k];
                A.U = s->U[k];
                A.L = s->L[k];
                A.nreal = s->I[k];
                A.depth = s->depth[k];
                A.F = s->F;
            }
            const int kprev = pi > 0 ? incl[pi - 1] : 0;
            nt_init<<<(unsigned)init_blocks, 256, 0, st>>>(A, pi > 0 ? s->U[kprev] : nullptr, kprev,
                                                           s->V32 + (size_t)k * R * R, s->V32lo + (size_t)k * R * R,
                                                           s->Rp);
            count_launch();
            if (!chk(cudaGetLastError())) break;
            A.NP = NPn;
            A.KC = KCn;
            if (!chk(nt_launch_level<0>(A, psn, ns, st))) break;
            for (int lvl = 0; lvl < A.depth; ++lvl) {
                A.lvl = lvl;
                if (!chk(nt_launch_level<1>(A, psn, ns, st))) break;
                nt_scan<<<1, 1024, 0, st>>>(A);
                count_launch();
                if (!chk(cudaGetLastError())) break;
                nt_part<<<(unsigned)part_blocks, 128, 0, st>>>(A);
                count_launch();
                if (!chk(cudaGetLastError())) break;
                A.cur ^= 1;
            }
            if (e != cudaSuccess) break;
            if (sg == 1) {
                A.NP = NPl;
                A.KC = KCl;
                if (!chk(nt_launch_level<2>(A, psl, ns, st))) break;
            }
        }
    }
    if (e == cudaSuccess) {
        // final stage: h ∘= the last factor's row, then ℓ_s = hᵀG⁺h on the tensor cores
        const int klast = incl[n_incl - 1];
        A.sg = 2;
        A.tree = s->Gplus32;
        nt_init<<<(unsigned)init_blocks, 256, 0, st>>>(A, s->U[klast], klast, nullptr, nullptr, s->Rp);
        count_launch();
        if (chk(cudaGetLastError())) {
            A.NP = NPn;
            A.KC = KCn;
            chk(nt_launch_level<3>(A, psn, ns, st));
        }
    }
    *err = e;
    return true;
}

}  // namespace krp
