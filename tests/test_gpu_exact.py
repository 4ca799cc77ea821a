"""Exact-decision samplers (KRP_PREC_EXACT) vs the FP64 CPU oracle, through the C ABI.

Bars:
  * trees: each stored slot plus its low part within c_F sqrt(G_ii G_jj) +
    2^-38 (|U|ᵀ|U|) of the FP64 partial Gram G over the node's rows, with
    c_F = 9 F (F + 1) 2^-47 the worst case of the leaves' anchored
    accumulation (carried up the sums by Cauchy-Schwarz) and 2^-38 covering
    the double-float sums; each delta-encoded top slot within 2^-23 |D| plus
    twice that of D_c = G_{2c} - alpha_c G_c formed in FP64 from the oracle's
    partial Grams;
  * indices: fewer than max(1, 1e-4 J) samples differ from the FP64 replay,
    and each that differs has, at its
    first differing factor, a uniform within 1e-5 C of an edge of the oracle's
    bin — at every size, including the 2^22-row launch the benchmark times;
  * weights 1e-4 relative; branch probabilities m_L / m_c within 1e-5 relative
    when >= 1e-3, else 1e-8 absolute.
"""
import numpy as np
import pytest
import torch

from oracle import krp_oracle as O
from paper_2301_12584_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
EXACT = 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2301_12584_gb300 import build as B
    from paper_2301_12584_gb300 import krpls
    if not os.path.exists(krpls.LIB_PATH):
        B.build()
    krpls.lib()


def sampler_for(Us, F=0, prec=EXACT):
    from paper_2301_12584_gb300.krpls import Sampler
    s = Sampler([U.shape[0] for U in Us], Us[0].shape[1], F, prec)
    for k, U in enumerate(Us):
        s.set_factor(k, torch.from_numpy(np.ascontiguousarray(U, dtype=np.float32)).to(DEV))
    return s


def draw(s, Us, excl, J, seed, draw_id):
    N = len(Us)
    idx = torch.full((N, J), -1, dtype=torch.int32, device=DEV)
    w = torch.zeros(J, dtype=torch.float32, device=DEV)
    lq = torch.zeros(J, dtype=torch.float32, device=DEV)
    s.sample(excl, J, seed, draw_id, idx, w, lq, None)
    assert s.sync_status() == 0, s.last_error()
    incl = O.included_factors(N, excl)
    return dict(idx=idx.cpu().numpy()[incl].astype(np.int64), weight=w.cpu().numpy(), logq=lq.cpu().numpy())


def mismatches(gidx, ref, tol=1e-5):
    """Samples whose tuple differs from the oracle's; each must be a near-edge
    flip (tau within tol * C of an edge of the oracle's bin at the first
    differing factor)."""
    diff = gidx != ref["idx"]
    bad = np.nonzero(diff.any(axis=0))[0]
    for s in bad:
        p = int(np.argmax(diff[:, s]))
        near = False
        for st in (0, 1):
            tau, lft, rgt, tot = (ref[k][p, st, s] for k in ("tau", "left", "right", "total"))
            if min(abs(tau - lft), abs(rgt - tau)) <= tol * tot:
                near = True
        assert near, f"sample {s}: factor {p} differs away from any CDF boundary"
    return len(bad)


def index_bar(J):
    return max(1.0, 1e-4 * J)


def unpack(slot, R):
    G = np.zeros((R, R))
    iu = np.triu_indices(R)
    G[iu] = slot[:R * (R + 1) // 2]
    return G + np.triu(G, 1).T


# ----------------------------------------------------------------- trees ----
@pytest.mark.parametrize("I,R,F", [(20000, 32, 32), (3001, 13, 7), (1000, 8, 8), (5, 4, 4), (777, 32, 96)])
def test_exact_tree_matches_partial_grams(I, R, F):
    Us = synth.skewed_row_factors(1, I, R, seed=I + R)
    s = sampler_for(Us, F)
    L, d, Tp = s.tree_info(0)
    hi = s.get_tree(0)
    lo, top = s.get_tree_exact(0)
    U64 = Us[0].astype(np.float64)
    T = R * (R + 1) // 2
    cF = 9 * F * (F + 1) * 2.0 ** -47
    worst = 0.0
    grams = {}

    def gram(v):
        if v not in grams:
            a, b = O.node_rows(v, L, F, I)
            G = U64[a:b].T @ U64[a:b]
            dg = np.sqrt(np.diag(G))
            grams[v] = (G, cF * np.outer(dg, dg) + 2.0 ** -38 * (np.abs(U64[a:b]).T @ np.abs(U64[a:b])))
        return grams[v]
    for slot in range(L):
        h = 1 if slot == 0 else 2 * slot
        G, tol = gram(h)
        got = unpack(hi[slot].astype(np.float64) + lo[slot].astype(np.float64), R)
        # after the packed triangle: the node's trace (it bounds the descent's
        # FP32 rounding error), then zeros
        tr = float(hi[slot][T]) + float(lo[slot][T])
        assert abs(tr - np.trace(G)) <= 1e-5 * np.trace(G) + 1e-30, (slot, tr, np.trace(G))
        assert np.all(hi[slot][T + 1:] == 0) and np.all(lo[slot][T + 1:] == 0)
        worst = max(worst, float((np.abs(got - G) / (tol + 1e-300)).max()))
        assert np.all(np.abs(got - G) <= tol + 1e-30), (slot, float((np.abs(got - G) / (tol + 1e-300)).max()))
    # the delta-encoded top in the tree's slot numbering: [root | D_1 .. D_{2^Ke - 1}]; a
    # right child's Gram is formed as its parent's minus its sibling's, so D carries
    # the double-float rounding of the parent's scale (~2^-44 |U|ᵀ|U| per level;
    # 2^-36 of the root's is still ~1e-11 of C, far inside the decisions' band)
    ke = min(10, d)
    assert np.array_equal(top[0], hi[0])
    root_bar = 2.0 ** -36 * (np.abs(U64).T @ np.abs(U64))
    for c in range(1, 1 << ke):
        depth_c = c.bit_length() - 1
        n_c = O.node_rows(c, L, F, I)
        n_l = O.node_rows(2 * c, L, F, I)
        rows_c, rows_l = n_c[1] - n_c[0], n_l[1] - n_l[0]
        if rows_c == 0:
            continue
        alpha = float(np.float32(rows_l) / np.float32(rows_c))
        Gc, tc = gram(c)
        Gl, _ = gram(2 * c)
        D = Gl - alpha * Gc
        got = unpack(top[c].astype(np.float64), R)
        assert np.all(np.abs(got - D) <= 2.0 ** -23 * np.abs(D) + 2 * tc + root_bar + 1e-30), (c, depth_c)
        # kappa_c = max |D_ab| / sqrt(g_a g_b) over the root's diagonal g: a bound
        # that must hold for the stored D (a little above its largest ratio)
        g = np.diag(gram(1)[0])
        ratio = np.abs(got) / np.sqrt(np.outer(g, g))
        kappa = float(top[c][T])
        assert ratio.max() <= kappa <= ratio.max() * 1.001 + 1e-30, (c, kappa, ratio.max())
        assert np.all(top[c][T + 1:] == 0)
    print(f"I={I} R={R} F={F}: worst |hi+lo - G| / bar = {worst:.2e}")
    s.close()


# ------------------------------------------------------- index parity ----
@pytest.mark.parametrize("case", ["cfg_tiny", "ragged", "excl1", "R5_F3", "N4", "R1", "N1", "R32", "F1",
                                  "R24_F40", "R32_I2p16", "R25_zero_rows_correlated"])
def test_exact_index_parity(case):
    J, excl, F, tree_ref = 1 << 15, -1, 0, False
    if case == "cfg_tiny":      # 3 x (64 x 8), F = 8
        Us, F = synth.gaussian_factors(3, 64, 8, seed=0), 8
    elif case == "ragged":
        Us, F = synth.gaussian_factors(3, [50, 77, 13], 6, seed=3), 4
    elif case == "excl1":
        Us, F, excl = synth.gaussian_factors(3, [40, 90, 33], 7, seed=4), 5, 1
    elif case == "R5_F3":
        Us, F = synth.skewed_entry_factors(3, 30, 5, seed=5), 3
    elif case == "N4":
        Us = synth.uniform_factors(4, 24, 6, seed=6)
    elif case == "R1":
        Us = synth.gaussian_factors(3, 20, 1, seed=7)
    elif case == "N1":
        Us, F = synth.gaussian_factors(1, 500, 8, seed=8), 8
    elif case == "R32":         # 2000 skewed rows per factor
        Us, F, J = synth.skewed_row_factors(3, 2000, 32, seed=9), 32, 1 << 16
    elif case == "F1":
        Us, F = synth.gaussian_factors(2, 40, 4, seed=10), 1
    elif case == "R24_F40":     # F > R (several leaf rows per lane) and uniform entries
        Us = [synth.uniform_factors(1, n, 24, seed=16 + q)[0] for q, n in enumerate((900, 1300, 700))]
        F = 40
    elif case == "R32_I2p16":   # 3 x (2^16 x 32) skewed rows, vs the FP64 segment-tree replay
        Us, F, J, tree_ref = synth.skewed_row_factors(3, 1 << 16, 32, seed=17), 32, 1 << 16, True
    elif case == "R25_zero_rows_correlated":
        # as after a few sparse CP-ALS sweeps: 80% zero rows, strongly correlated
        # unit-norm columns (masses far below |h̃|^2 tr G, so FP32 masses carry
        # large relative errors), R = F = 25 (ragged leaves), vs the tree replay
        Us = synth.correlated_sparse_factors(3, [1 << 18, 1 << 18, 4096], 25, seed=21)
        excl, F, J, tree_ref = 1, 25, 1 << 16, True
    s = sampler_for(Us, F)
    out = draw(s, Us, excl, J, seed=12345, draw_id=3)
    U64 = [U.astype(np.float64) for U in Us]
    if tree_ref:
        ref = O.krp_sample_tree(U64, excl, J, 12345, 3, F=F)
    else:
        ref = O.krp_sample(U64, excl, J, 12345, 3, record=True, chunk=2048)
    assert np.all(np.isfinite(out["weight"])) and np.all(out["weight"] > 0)
    mism = mismatches(out["idx"], ref)
    nx = s.exact_count()
    print(f"{case}: {mism} mismatches / {J}; {nx} exact re-decisions")
    assert mism < index_bar(J), mism
    same = ~(out["idx"] != ref["idx"]).any(axis=0)
    np.testing.assert_allclose(out["weight"][same], ref["weight"][same], rtol=1e-4)
    np.testing.assert_allclose(out["logq"][same], ref["logq"][same], atol=1e-4)
    s.close()


def test_exact_full_size_index_parity():
    """N=3, I=2^22, R=32, F=32 (1% rows x100), J=2^16: the benchmark's launch in
    the exact-decision mode against the FP64 segment-tree replay (Alg. 3/4) of
    every sample."""
    I, R, J = 1 << 22, 32, 1 << 16
    Us = synth.skewed_row_factors(3, I, R, seed=0)
    s = sampler_for(Us, 32)
    out = draw(s, Us, -1, J, seed=1, draw_id=0)
    nx = s.exact_count()
    U64 = [U.astype(np.float64) for U in Us]
    prep = O.SamplerPrep(U64, -1)
    # eigenvectors of G_{>k}: the row stage's distribution depends on V[:, u]
    for k in prep.incl:
        lam, V, _, _ = s.get_prep(k)
        np.testing.assert_allclose(lam, prep.lam[k], rtol=0, atol=1e-12 * prep.lam[k].max())
        dv = np.minimum(np.abs(V - prep.V[k]), np.abs(V + prep.V[k])).max(axis=0)
        print(f"factor {k}: max |V - V_oracle| = {dv.max():.2e}")
    ref = O.krp_sample_tree(U64, -1, J, 1, 0, F=32, prep=prep)
    mism = mismatches(out["idx"], ref)
    print(f"full size, exact mode: {mism} mismatches / {J} ({mism / J:.1e}); "
          f"{nx} exact re-decisions ({nx / (3 * J):.2e} per row stage)")
    assert mism < 1e-4 * J, mism
    same = ~(out["idx"] != ref["idx"]).any(axis=0)
    np.testing.assert_allclose(out["weight"][same], ref["weight"][same], rtol=1e-4)
    s.close()


# ------------------------------------------------ branch probabilities ----
@pytest.mark.parametrize("prec", [EXACT, 0])
def test_branch_probabilities_r32(prec):
    """Per-level m_L / m_c of both stages at R = 32, F = 32 on 3 x (2^16 x 32)
    skewed rows against the FP64 trees (Alg. 4).  Exact-decision mode (prec 2):
    the trace holds double-float masses of the path's nodes, so the bar is
    1e-5 relative (>= 1e-3) or 1e-8 absolute.  FP32 mode (prec 0): m(c) of a
    right child is its parent's mass minus its sibling's, carried in FP32 down
    the path, so it is off by a few ulp of C (its bar adds 4e-7 C / m(c)), and
    its root Grams sum FP32-accumulated leaves (~1e-9 relative), which moves
    the eigenvectors of G_{>k} by up to ~1e-5 where its eigenvalues cluster
    and the eigencomponent stage's probabilities by up to ~1e-4 relative."""
    I, R, F, N, J, n_tr = 1 << 16, 32, 32, 3, 2048, 64
    Us = synth.skewed_row_factors(N, I, R, seed=23)
    s = sampler_for(Us, F, prec)
    idx = torch.zeros((N, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, dtype=torch.float32, device=DEV)
    tr = torch.zeros(n_tr * N * 2 * 66, dtype=torch.float32, device=DEV)
    s.debug_trace(-1, J, 99, 5, idx, w, tr, n_tr)
    assert s.sync_status() == 0, s.last_error()
    trace = tr.cpu().numpy().reshape(n_tr, N, 2, 66)
    gi = idx.cpu().numpy().astype(np.int64)
    U64 = [U.astype(np.float64) for U in Us]
    prep = O.SamplerPrep(U64, -1)
    from oracle.philox import sampler_uniforms
    ue, ur = sampler_uniforms(99, 5, n_tr, N)
    checked = 0
    for sm in range(n_tr):
        h = np.ones(R)
        for p in range(N):
            u_k, tr_u = O.eig_tree_row_sample(prep.lam[p], prep.V[p], prep.grams[p], h, ue[sm, p])
            ht = h * prep.V[p][:, u_k]
            t_k, tr_t = O.tree_row_sample(U64[p], F, np.ones((R, R)), ht, ur[sm, p])
            if t_k != gi[p, sm]:
                break
            for st, trc in ((0, tr_u), (1, tr_t)):
                C = trc[0][1] if trc else 1.0
                for lvl, (ml, mc) in enumerate(trc):
                    pl, gpl = ml / mc, trace[sm, p, st, 2 + 2 * lvl] / trace[sm, p, st, 3 + 2 * lvl]
                    tol = 1e-5 * pl if pl >= 1e-3 else 1e-8
                    if prec == 0:
                        tol = (1e-4 if st == 0 else 1e-5) * pl + 1e-8 + 4e-7 * C / mc
                    assert abs(gpl - pl) <= tol, (prec, sm, p, st, lvl, gpl, pl)
                    checked += 1
            h = h * U64[p][t_k]
    assert checked > 2000, checked
    s.close()


# --------------------------------------------- single-element updates ----
def test_exact_updates_match_rebuild_and_oracle():
    """krp_update_entries on an exact-decision sampler: the (hi, lo) slots and
    the delta-encoded top follow the updated factor to double-float accuracy,
    and later draws keep the index bar."""
    rng = np.random.default_rng(41)
    I, R, F = 3000, 16, 16
    Us = synth.gaussian_factors(3, I, R, seed=42)
    s = sampler_for(Us, F)
    ups = [(int(rng.integers(I)), int(rng.integers(R)), float(rng.standard_normal() * 3)) for _ in range(60)]
    rows = torch.tensor([u[0] for u in ups], dtype=torch.int32, device=DEV)
    cols = torch.tensor([u[1] for u in ups], dtype=torch.int32, device=DEV)
    vals = torch.tensor([u[2] for u in ups], dtype=torch.float32, device=DEV)
    s.update_entries(0, rows, cols, vals)
    assert s.sync_status() == 0, s.last_error()
    U0 = Us[0].astype(np.float64).copy()
    for r, c, v in ups:
        U0[r, c] = np.float32(v)
    L, d, Tp = s.tree_info(0)
    hi = s.get_tree(0)
    lo, top = s.get_tree_exact(0)
    for slot in range(L):
        h = 1 if slot == 0 else 2 * slot
        a, b = O.node_rows(h, L, F, I)
        G = U0[a:b].T @ U0[a:b]
        bound = np.abs(U0[a:b]).T @ np.abs(U0[a:b])
        dg = np.sqrt(np.diag(G))
        tol = 9 * F * (F + 1) * 2.0 ** -47 * np.outer(dg, dg) + 2.0 ** -38 * bound
        got = unpack(hi[slot].astype(np.float64) + lo[slot].astype(np.float64), R)
        assert np.all(np.abs(got - G) <= tol + 1e-30), slot
        T = R * (R + 1) // 2
        tr = float(hi[slot][T]) + float(lo[slot][T])
        assert abs(tr - np.trace(G)) <= 1e-5 * np.trace(G) + 1e-30, (slot, tr, np.trace(G))
    assert np.array_equal(top[0], hi[0])
    Us_new = [U0.astype(np.float32), Us[1], Us[2]]
    J = 1 << 14
    out = draw(s, Us_new, -1, J, seed=5, draw_id=1)
    ref = O.krp_sample([U.astype(np.float64) for U in Us_new], -1, J, 5, 1, record=True, chunk=2048)
    assert mismatches(out["idx"], ref) < index_bar(J)
    s.close()


def test_exact_mode_rejects_large_rank_and_batches():
    from paper_2301_12584_gb300.krpls import Batch, KrpError, Sampler
    with pytest.raises(KrpError):
        Sampler([100, 100], 40, 0, EXACT)
    Us = synth.gaussian_factors(3, 64, 8, seed=1)
    s = sampler_for(Us, 8)
    with pytest.raises(KrpError):
        Batch([s], None)
    s.close()
