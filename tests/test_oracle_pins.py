"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (closed forms, brute force, library routines, invariants
the paper states), so that a dropped term, wrong sign/index or transposed
operand fails at least one of them.  CPU only."""
import itertools
import os

import numpy as np
import pytest

from oracle import krp_oracle as O
from oracle.philox import philox4x32_10, sampler_uniforms, u32_to_open_unit
from paper_2301_12584_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(np.array(v[0:4], np.uint32), np.array(v[4:6], np.uint32))
        assert [int(x) for x in out] == v[6:10]


def test_uniform_mapping_open_and_exact_fp32():
    x = np.array([0, 1, 511, 512, 2**31, 2**32 - 1], dtype=np.uint32)
    u = u32_to_open_unit(x)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == 2.0 ** -24 and u[-1] == 1 - 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    a, b = sampler_uniforms(7, 3, 50000, 3)
    assert abs(a.mean() - 0.5) < 0.01 and abs(b.mean() - 0.5) < 0.01
    assert abs(np.corrcoef(a[:, 0], b[:, 0])[0, 1]) < 0.02


# ------------------------------------------------------ products / Grams ----
def test_khatri_rao_matches_kronecker_columns():
    rng = np.random.default_rng(0)
    Us = [rng.standard_normal((n, 3)) for n in (2, 3, 4)]
    A = O.khatri_rao(Us)
    for r in range(3):
        ref = np.kron(np.kron(Us[0][:, r], Us[1][:, r]), Us[2][:, r])
        np.testing.assert_allclose(A[:, r], ref, rtol=0, atol=1e-15)
    # C order: last factor fastest
    i = (1, 2, 3)
    np.testing.assert_allclose(A[O.linear_index(np.array(i)[:, None], (2, 3, 4))[0]],
                               Us[0][1] * Us[1][2] * Us[2][3])


def test_hadamard_gram_is_AtA():
    rng = np.random.default_rng(1)
    Us = [rng.standard_normal((n, 4)) for n in (5, 6, 7)]
    for excl in (-1, 0, 1, 2):
        incl = O.included_factors(3, excl)
        A = O.khatri_rao([Us[k] for k in incl])
        np.testing.assert_allclose(O.hadamard_gram(Us, excl), A.T @ A, rtol=1e-12)


def test_pinv_eig_matches_library_and_moore_penrose():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((20, 6))
    G = X.T @ X
    Gp, r = O.pinv_eig(G)
    assert r == 6
    np.testing.assert_allclose(Gp, np.linalg.inv(G), rtol=1e-10)
    X[:, 5] = X[:, 0] + X[:, 1]       # rank 5
    G = X.T @ X
    Gp, r = O.pinv_eig(G)
    assert r == 5
    np.testing.assert_allclose(G @ Gp @ G, G, atol=1e-10 * np.abs(G).max())
    np.testing.assert_allclose(Gp @ G @ Gp, Gp, atol=1e-10 * np.abs(Gp).max())
    np.testing.assert_allclose(Gp, np.linalg.pinv(G, hermitian=True), atol=1e-10)


# ------------------------------------------------------- leverage scores ----
def test_leverage_sum_is_rank_and_bounds():
    rng = np.random.default_rng(3)
    Us = [rng.standard_normal((n, 5)) for n in (4, 5, 6)]
    lev, r = O.krp_leverage(Us)
    assert r == 5
    assert abs(lev.sum() - 5) < 1e-10
    assert lev.min() >= -1e-14 and lev.max() <= 1 + 1e-12
    # rank-deficient: duplicate a column in every factor
    Us2 = [np.concatenate([U, U[:, :1]], axis=1) for U in Us]
    lev2, r2 = O.krp_leverage(Us2)
    assert r2 == 5
    np.testing.assert_allclose(lev2, lev, atol=1e-10)


def test_leverage_matches_textbook_qr():
    rng = np.random.default_rng(4)
    Us = [rng.standard_normal((n, 4)) for n in (3, 4, 5)]
    A = O.khatri_rao(Us)
    Q, _ = np.linalg.qr(A)              # full rank: reduced QR (Sec. 2.1)
    np.testing.assert_allclose(O.krp_leverage(Us)[0], (Q * Q).sum(1), atol=1e-12)
    np.testing.assert_allclose(O.leverage_scores_qr(A)[0], (Q * Q).sum(1), atol=1e-12)
    np.testing.assert_allclose(O.leverage_scores_pinv(A)[0], (Q * Q).sum(1), atol=1e-12)
    # N = 1 reduces to the QR row norms of U itself
    lev1, _ = O.krp_leverage([Us[2]])
    Q1, _ = np.linalg.qr(Us[2])
    np.testing.assert_allclose(lev1, (Q1 * Q1).sum(1), atol=1e-12)


def test_leverage_rank_one_closed_form():
    rng = np.random.default_rng(5)
    Us = [rng.standard_normal((n, 1)) for n in (3, 4, 5)]
    a = O.khatri_rao(Us)[:, 0]
    np.testing.assert_allclose(O.krp_leverage(Us)[0], a * a / (a @ a), rtol=1e-12)


def test_leverage_orthogonal_columns_closed_form():
    rng = np.random.default_rng(6)
    Us = []
    for n in (6, 7, 8):
        Q, _ = np.linalg.qr(rng.standard_normal((n, 4)))
        Us.append(Q * rng.uniform(0.5, 3.0, size=4)[None, :])   # G_k diagonal
    lev, _ = O.krp_leverage(Us)
    den = np.prod([np.sum(U * U, axis=0) for U in Us], axis=0)
    A2 = O.khatri_rao([U * U for U in Us])
    np.testing.assert_allclose(lev, (A2 / den[None, :]).sum(1), rtol=1e-10)


# ------------------------------------------------- conditionals (Thm 3.1) ----
def _brute_conditional(Us, prefix, k):
    """p(s_k | s_<k) by marginalising the exact leverage scores."""
    lev, r = O.krp_leverage(Us)
    L = lev.reshape([U.shape[0] for U in Us])
    sub = L[tuple(prefix)]
    other = tuple(range(1, sub.ndim))
    marg = sub.sum(axis=other) if other else sub
    return marg / marg.sum()


@pytest.mark.parametrize("R", [2, 3])
def test_thm31_conditionals_match_marginalised_leverage(R):
    rng = np.random.default_rng(10 + R)
    Us = [rng.standard_normal((n, R)) for n in (3, 4, 3)]
    Gp, rank = O.pinv_eig(O.hadamard_gram(Us))
    for prefix in [(), (1,), (2, 3)]:
        k = len(prefix)
        h = np.ones(R)
        for i, s in enumerate(prefix):
            h = h * Us[i][s]
        q, C = O.conditional_q(h, Us[k], O.g_greater(Us, -1, k, Gp))
        np.testing.assert_allclose(q, _brute_conditional(Us, prefix, k), atol=1e-12)
        if k == 0:
            assert abs(C - rank) < 1e-10       # C at k=1 is the sum of leverage scores


def test_product_of_conditionals_is_leverage_over_rank():
    rng = np.random.default_rng(12)
    Us = [rng.standard_normal((n, 3)) for n in (4, 3, 5)]
    lev, rank = O.krp_leverage(Us)
    Gp, _ = O.pinv_eig(O.hadamard_gram(Us))
    for tup in [(0, 0, 0), (3, 2, 4), (1, 1, 2)]:
        h = np.ones(3)
        p = 1.0
        for k, s in enumerate(tup):
            q, _ = O.conditional_q(h, Us[k], O.g_greater(Us, -1, k, Gp))
            p *= q[s]
            h = h * Us[k][s]
        lin = O.linear_index(np.array(tup)[:, None], (4, 3, 5))[0]
        assert abs(p - lev[lin] / rank) < 1e-12


def test_mixture_identity():
    """q = Σ_u w[u] W[:,u]/||W[:,u]||_1 (Sec. 3.2, Bayes' rule step of App. A.6)."""
    rng = np.random.default_rng(13)
    Us = [rng.standard_normal((n, 4)) for n in (5, 6, 7)]
    Gp, _ = O.pinv_eig(O.hadamard_gram(Us))
    h = Us[0][2] * 1.0
    Ygt = O.g_greater(Us, -1, 1, Gp)
    q, C = O.conditional_q(h, Us[1], Ygt)
    lam, V = O.eig_ascending(Ygt)
    w = O.eigencomponent_weights(h[None, :], lam, V, O.gram(Us[1]))[0]
    assert abs(w.sum() - C) < 1e-10 * C
    W = O.row_weights((h[None, :] * V.T), Us[1])          # W[u, t]
    mix = sum((w[u] / w.sum()) * W[u] / W[u].sum() for u in range(4) if W[u].sum() > 0)
    np.testing.assert_allclose(mix, q, atol=1e-13)


def _enumerate_two_stage(Us, exclude=-1):
    """Exact distribution of the two-stage sampler by enumerating all (u, t) paths."""
    prep = O.SamplerPrep(Us, exclude)
    dims = [Us[k].shape[0] for k in prep.incl]
    P = np.zeros(dims)

    def rec(p, h, prob, tup):
        if p == len(prep.incl):
            P[tuple(tup)] += prob
            return
        k = prep.incl[p]
        w = O.eigencomponent_weights(h[None, :], prep.lam[k], prep.V[k], prep.grams[k])[0]
        for u in range(prep.R):
            if w[u] <= 0:
                continue
            Wt = O.row_weights((h * prep.V[k][:, u])[None, :], prep.Us[k])[0]
            for t in range(dims[p]):
                if Wt[t] > 0:
                    rec(p + 1, h * prep.Us[k][t], prob * (w[u] / w.sum()) * (Wt[t] / Wt.sum()),
                        tup + [t])
    rec(0, np.ones(prep.R), 1.0, [])
    return P.reshape(-1), prep


@pytest.mark.parametrize("R,excl", [(2, -1), (3, -1), (2, 1)])
def test_two_stage_paths_sum_to_leverage(R, excl):
    rng = np.random.default_rng(20 + R)
    Us = [rng.standard_normal((4, R)) for _ in range(3)]
    P, prep = _enumerate_two_stage(Us, excl)
    lev, rank = O.krp_leverage(Us, excl)
    np.testing.assert_allclose(P, lev / rank, atol=1e-12)


# ------------------------------------------------------- inverse CDF ----
def test_inverse_cdf_matches_python_loop():
    rng = np.random.default_rng(30)
    w = rng.random((200, 9)) * (rng.random((200, 9)) > 0.3)
    w[:, 0] += 1e-3
    u = rng.random(200)
    idx, tau, lft, rgt, tot = O.inverse_cdf(w, u)
    for s in range(200):
        t = u[s] * w[s].sum()
        acc = 0.0
        for i in range(9):
            acc += w[s, i]
            if acc >= t:
                break
        assert idx[s] == i and w[s, i] > 0
        assert lft[s] < tau[s] <= rgt[s]


# --------------------------------------------------------- segment tree ----
@pytest.mark.parametrize("I,F", [(37, 4), (64, 8), (5, 8), (33, 1)])
def test_tree_children_sum_and_root(I, F):
    rng = np.random.default_rng(I + F)
    U = rng.standard_normal((I, 3))
    L, d = O.tree_shape(I, F)
    assert L >= -(-I // F) and L < 2 * max(1, -(-I // F))
    np.testing.assert_allclose(O.partial_gram(U, 1, L, F), U.T @ U, rtol=1e-13)
    for v in range(1, L):
        np.testing.assert_allclose(O.partial_gram(U, v, L, F),
                                   O.partial_gram(U, 2 * v, L, F) + O.partial_gram(U, 2 * v + 1, L, F),
                                   rtol=1e-12, atol=1e-12)
    # leaves cover the rows exactly once
    cover = np.zeros(I, int)
    for b in range(L):
        lo, hi = O.node_rows(L + b, L, F, I)
        cover[lo:hi] += 1
    assert np.all(cover == 1)


@pytest.mark.parametrize("I,F", [(37, 4), (64, 8), (100, 7)])
def test_tree_descent_equals_inverse_cdf(I, F):
    """Alg. 4 returns the same bin as a linear inverse-CDF scan (Sec. 3.1)."""
    rng = np.random.default_rng(40 + I)
    R = 4
    U = rng.standard_normal((I, R))
    A = rng.standard_normal((6, R))
    Y = A.T @ A
    for _ in range(40):
        h = rng.standard_normal(R)
        u = rng.random()
        t, trace = O.tree_row_sample(U, F, Y, h, u)
        w = np.einsum("sa,ab,sb->s", U, np.outer(h, h) * Y, U)
        ref, *_ = O.inverse_cdf(w[None, :], np.array([u]))
        assert t == ref[0]
        for ml, mc in trace:
            assert -1e-12 <= ml <= mc * (1 + 1e-12) + 1e-12


def test_eig_tree_equals_eigencomponent_inverse_cdf():
    rng = np.random.default_rng(50)
    Us = [rng.standard_normal((n, 5)) for n in (6, 7, 8)]
    prep = O.SamplerPrep(Us)
    k = 1
    for _ in range(30):
        h = Us[0][rng.integers(6)]
        u = rng.random()
        t, _ = O.eig_tree_row_sample(prep.lam[k], prep.V[k], prep.grams[k], h, u)
        w = O.eigencomponent_weights(h[None, :], prep.lam[k], prep.V[k], prep.grams[k])
        ref, *_ = O.inverse_cdf(w, np.array([u]))
        assert t == ref[0]


# --------------------------------------------------- sampler statistics ----
def test_sampler_histogram_matches_leverage_distribution():
    """App. A.13.2 shape: 3 factors 8 x 8, 1% entries x10, 50,000 draws."""
    Us = [U.astype(np.float64) for U in synth.skewed_entry_factors(3, 8, 8, seed=0)]
    lev, rank = O.krp_leverage(Us)
    p = lev / rank
    out = O.krp_sample(Us, -1, 50000, seed=1, draw_id=0)
    lin = O.linear_index(out["idx"], (8, 8, 8))
    cnt = np.bincount(lin, minlength=512)
    # chi-square on cells with expected count >= 5
    e = 50000 * p
    m = e >= 5
    chi2 = ((cnt[m] - e[m]) ** 2 / e[m]).sum() + ((cnt[~m].sum() - e[~m].sum()) ** 2 / max(e[~m].sum(), 1e-9))
    from scipy.stats import chi2 as C2
    assert C2.sf(chi2, m.sum()) > 1e-3
    # per-sample probabilities are the exact ones
    np.testing.assert_allclose(out["q"], p[lin], rtol=1e-10)
    # marginal TV
    for a in range(3):
        emp = np.bincount(out["idx"][a], minlength=8) / 50000
        ex = p.reshape(8, 8, 8).sum(axis=tuple(b for b in range(3) if b != a))
        assert 0.5 * np.abs(emp - ex).sum() < 0.01


def test_sampling_matrix_is_unbiased():
    """E[(SA)ᵀ(SA)] = AᵀA for S with weights 1/sqrt(J q) (Sec. 2.1)."""
    rng = np.random.default_rng(60)
    Us = [rng.standard_normal((n, 3)) for n in (5, 6, 7)]
    J = 40000
    out = O.krp_sample(Us, -1, J, seed=5, draw_id=1)
    SA = O.sketched_rows(Us, -1, out["idx"], out["weight"])
    G = O.hadamard_gram(Us)
    np.testing.assert_allclose(SA.T @ SA, G, rtol=0.05, atol=0.05 * np.abs(G).max())


def test_excluded_factor_and_draw_id():
    rng = np.random.default_rng(61)
    Us = [rng.standard_normal((n, 3)) for n in (5, 6, 7)]
    out = O.krp_sample(Us, 1, 30000, seed=2, draw_id=9)
    assert out["idx"].shape == (2, 30000)
    lev, rank = O.krp_leverage(Us, 1)
    lin = O.linear_index(out["idx"], (5, 7))
    np.testing.assert_allclose(out["q"], lev[lin] / rank, rtol=1e-10)
    cnt = np.bincount(lin, minlength=35) / 30000
    assert 0.5 * np.abs(cnt - lev / rank).sum() < 0.03
    other = O.krp_sample(Us, 1, 100, seed=2, draw_id=10)
    assert not np.array_equal(other["idx"], out["idx"][:, :100])
    same = O.krp_sample(Us, 1, 100, seed=2, draw_id=9)
    assert np.array_equal(same["idx"], out["idx"][:, :100])
    # a sub-range of samples reproduces the same tuples (counter-based)
    part = O.krp_sample(Us, 1, 50, seed=2, draw_id=9, d0=25)
    assert np.array_equal(part["idx"], out["idx"][:, 25:75])


# --------------------------------------------------- least squares ----
def test_lstsq_normal_equations_and_exact_recovery():
    rng = np.random.default_rng(70)
    A = rng.standard_normal((50, 5))
    X0 = rng.standard_normal((5, 3))
    np.testing.assert_allclose(O.lstsq(A, A @ X0), X0, atol=1e-12)
    B = rng.standard_normal((50, 3))
    X = O.lstsq(A, B)
    np.testing.assert_allclose(A.T @ (A @ X - B), 0, atol=1e-11)


def test_thm21_sketched_residual_close_to_optimal():
    rng = np.random.default_rng(71)
    Us = [rng.standard_normal((8, 4)) for _ in range(3)]
    A = O.khatri_rao(Us)
    b = A @ rng.standard_normal((4, 1)) + 0.1 * rng.standard_normal((512, 1))
    X_opt = O.lstsq(A, b)
    r_opt = np.linalg.norm(A @ X_opt - b)
    out = O.krp_sample(Us, -1, 4000, seed=3, draw_id=0)
    lin = O.linear_index(out["idx"], (8, 8, 8))
    SA = O.sketched_rows(Us, -1, out["idx"], out["weight"])
    SB = b[lin] * out["weight"][:, None]
    X = O.lstsq(SA, SB)
    eps = np.linalg.norm(A @ X - b) / r_opt - 1
    assert 0 <= eps < 0.05


# ---------------------------------------------------------- CP-ALS ----
def test_cp_fit_matches_dense_definition():
    rng = np.random.default_rng(80)
    dims = (4, 5, 3)
    coords = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")).reshape(3, -1)
    keep = rng.random(coords.shape[1]) < 0.5
    coords = coords[:, keep]
    vals = rng.standard_normal(coords.shape[1])
    Us = [rng.standard_normal((d, 2)) for d in dims]
    sigma = np.array([1.5, 0.7])
    T = np.zeros(dims)
    T[tuple(coords)] = vals
    M = np.einsum("r,ir,jr,kr->ijk", sigma, *Us)
    ref = 1 - np.linalg.norm(M - T) / np.linalg.norm(T)
    assert abs(O.cp_fit(coords, vals, sigma, Us) - ref) < 1e-12


def test_cp_als_exact_and_sketched_recover_planted_tensor():
    dims = (6, 7, 5)
    coords, vals = synth.planted_dense_tensor(dims, 2, seed=3)
    U0 = [np.random.default_rng(9).standard_normal((d, 2)) for d in dims]
    _, _, fits = O.cp_als_exact(coords, vals.astype(np.float64), dims, U0, 15)
    assert fits[-1] > 0.999
    _, _, fs = O.cp_als_sketched(coords, vals.astype(np.float64), dims, U0, J=300, sweeps=8, seed=4)
    assert fs[-1] > 0.99


# ------------------------------------------------- planted mistakes ----
def test_planted_mistakes_fail_the_pins(monkeypatch):
    """Each plausible slip in the sampler's arithmetic breaks the brute-force
    path enumeration (the pin is sensitive, not vacuous)."""
    rng = np.random.default_rng(90)
    Us = [rng.standard_normal((4, 3)) for _ in range(3)]
    lev, rank = O.krp_leverage(Us)
    good = O.g_greater
    mistakes = {
        # G_{>k} including factor k itself (index slip m >= k)
        "g_ge": lambda Us_, ex, k, Gp: good(Us_, ex, k - 1, Gp) if k > 0 else good(Us_, ex, k, Gp) * O.gram(Us_[0]),
        # G_{>k} forgetting G⁺
        "no_pinv": lambda Us_, ex, k, Gp: good(Us_, ex, k, np.ones_like(Gp)),
    }
    for name, bad in mistakes.items():
        monkeypatch.setattr(O, "g_greater", bad)
        P, _ = _enumerate_two_stage(Us)
        assert np.abs(P - lev / rank).max() > 1e-4, name
        monkeypatch.setattr(O, "g_greater", good)
    good_w = O.eigencomponent_weights
    # eigenvalue weight dropped
    monkeypatch.setattr(O, "eigencomponent_weights",
                        lambda H, lam, V, Gk: good_w(H, np.ones_like(lam), V, Gk))
    P, _ = _enumerate_two_stage(Us)
    assert np.abs(P - lev / rank).max() > 1e-4
    # transposed eigenvector matrix
    monkeypatch.setattr(O, "eigencomponent_weights",
                        lambda H, lam, V, Gk: good_w(H, lam, V.T, Gk))
    P, _ = _enumerate_two_stage(Us)
    assert np.abs(P - lev / rank).max() > 1e-4


@pytest.mark.parametrize("I,F,excl", [(37, 4, -1), (64, 8, 1), (50, 7, -1)])
def test_batched_tree_replay_equals_inverse_cdf_sampler(I, F, excl):
    """Alg. 3/4 replay gives the same tuples as the plain inverse-CDF replay."""
    Us = synth.skewed_entry_factors(3, I, 5, seed=I)
    U64 = [U.astype(np.float64) for U in Us]
    a = O.krp_sample(U64, excl, 3000, seed=3, draw_id=2, record=True)
    b = O.krp_sample_tree(U64, excl, 3000, seed=3, draw_id=2, F=F)
    assert np.array_equal(a["idx"], b["idx"]) and np.array_equal(a["uidx"], b["uidx"])
    np.testing.assert_allclose(b["total"], a["total"], rtol=1e-12)
    np.testing.assert_allclose(b["tau"], a["tau"], rtol=1e-12)


def test_planted_rhs_noise_is_standard_normal_and_keyed_by_tuple():
    """The planted right-hand side's noise (a workload generator): sigma = 0
    gives A X exactly; repeated tuples get identical rows; over distinct tuples
    the noise passes a Kolmogorov-Smirnov test against N(0, 1)."""
    from scipy.stats import kstest
    rng = np.random.default_rng(3)
    Us = [rng.standard_normal((40, 5)) for _ in range(3)]
    idx = np.stack(np.unravel_index(np.arange(40 ** 3), (40, 40, 40)))   # every tuple once
    X = rng.standard_normal((5, 2))
    A = O.sketched_rows(Us, -1, idx, np.ones(idx.shape[1]))
    np.testing.assert_array_equal(O.planted_rhs(Us, -1, idx, X, 0.0, 11), A @ X)
    xi = O.planted_rhs(Us, -1, idx, X, 1.0, 11) - A @ X
    assert kstest(xi[:, 0], "norm").pvalue > 1e-3
    assert kstest(xi[:, 1], "norm").pvalue > 1e-3
    assert abs(np.corrcoef(xi[:, 0], xi[:, 1])[0, 1]) < 4 / np.sqrt(len(xi))
    rep = idx[:, [5, 77, 5, 77]]
    B = O.planted_rhs(Us, -1, rep, X, 1.0, 11)
    np.testing.assert_array_equal(B[0], B[2])
    np.testing.assert_array_equal(B[1], B[3])
    assert not np.allclose(O.planted_rhs(Us, -1, rep, X, 1.0, 12), B)


def test_single_entry_update_equals_rebuild():
    """UpdateSampler (App. A): after a sequence of single-entry updates, some
    to the same row, every node Gram equals the tree rebuilt from the updated
    matrix (FP64 to 1e-12 relative)."""
    rng = np.random.default_rng(21)
    I, R, F = 37, 5, 4
    U = rng.standard_normal((I, R))
    tree = O.TreeFP64(U.copy(), F)
    U2 = U.copy()
    for r, c in [(0, 0), (36, 4), (17, 2), (17, 3), (17, 2), (5, 1)]:
        val = float(rng.standard_normal()) * 3.0
        O.tree_update_entry(tree, r, c, val)
        U2[r, c] = val
    ref = O.TreeFP64(U2, F)
    scale = np.abs(ref.nodes).max()
    assert np.abs(tree.nodes - ref.nodes).max() <= 1e-12 * scale
    np.testing.assert_array_equal(tree.U, U2)
    # a planted mistake (the d^2 term dropped) is caught
    bad = O.TreeFP64(U.copy(), F)
    x = bad.U[3].copy()
    d = 2.0 - x[1]
    v = bad.L + 3 // F
    bad.nodes[v][1, :] += d * x
    bad.nodes[v][:, 1] += d * x
    U3 = U.copy()
    U3[3, 1] = 2.0
    assert np.abs(bad.nodes[v] - O.TreeFP64(U3, F).nodes[v]).max() > 1e-6


def test_distortion_and_kronecker_residual():
    """Sec. 4.2 accuracy workload: the distortion by its definition (QR basis
    of the materialised A) is 0 for the identity sampler, equals the
    appendix's route kappa(SA V Σ⁻¹) from the eigendecomposition of ⊛ U_kᵀU_k,
    and the Kronecker right-hand side and closed-form residual match the
    materialised b and ||Ax - b||."""
    rng = np.random.default_rng(41)
    Us = [rng.standard_normal((n, 4)) for n in (5, 6, 7)]
    A = O.khatri_rao(Us)
    allidx = np.stack(np.unravel_index(np.arange(A.shape[0]), (5, 6, 7)))
    assert abs(O.sketch_distortion(Us, -1, allidx, np.ones(A.shape[0]))) < 1e-10
    J = 60
    idx = np.stack([rng.integers(0, n, J) for n in (5, 6, 7)])
    w = rng.uniform(0.5, 2.0, J)
    D = O.sketch_distortion(Us, -1, idx, w)
    SA = O.sketched_rows(Us, -1, idx, w)
    lam, V = np.linalg.eigh(O.hadamard_gram(Us))
    sv = np.linalg.svd(SA @ V @ np.diag(lam ** -0.5), compute_uv=False)
    assert abs(D - (sv[0] / sv[-1] - 1.0)) <= 1e-9 * max(1.0, D)
    cs = [rng.standard_normal(n) for n in (5, 6, 7)]
    b = np.kron(np.kron(cs[0], cs[1]), cs[2])
    lin = O.linear_index(idx, (5, 6, 7))
    np.testing.assert_allclose(O.kron_rows(cs, -1, idx), b[lin], rtol=1e-14)
    x = rng.standard_normal(4)
    res, G, Atb = O.kron_lstsq_residual(Us, -1, cs, x)
    np.testing.assert_allclose(Atb, A.T @ b, rtol=1e-12)
    assert abs(res - np.linalg.norm(A @ x - b)) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("excl", [-1, 1])
def test_sample_probability_is_leverage_over_rank(excl):
    """sample_probability(q_s = ℓ_s / rank, Sec. 2.1) against the textbook
    QR leverage scores of the materialised A (Thm 1.1): every tuple's q equals
    the row's leverage over rank(A), and q sums to 1 over all tuples; also with
    a factor excluded (A over the included factors) and rank-deficient."""
    rng = np.random.default_rng(17)
    Us = [rng.standard_normal((n, 3)) for n in (3, 4, 2)]
    Us[2][:, 2] = Us[2][:, 0]                           # factor 2's Gram has rank 2
    incl = [k for k in range(3) if k != excl]
    A = O.khatri_rao([Us[k] for k in incl])
    lev, r = O.leverage_scores_qr(A)
    tuples = np.array(list(itertools.product(*[range(Us[k].shape[0]) for k in incl]))).T   # C order
    q, rank = O.sample_probability(Us, excl, tuples)
    assert rank == r
    np.testing.assert_allclose(q, lev / r, rtol=1e-10, atol=1e-14)
    assert abs(q.sum() - 1.0) < 1e-12
