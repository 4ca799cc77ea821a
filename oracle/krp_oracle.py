"""Plain FP64 CPU oracle for exact Khatri-Rao-product leverage-score sampling.

TEST INFRASTRUCTURE ONLY.  This package checks the CUDA library; it is not
part of it.  Only the test suite, the smoke check and the CPU-baseline leg of
the benchmark may import it.  It shares no code with the device path.

Every function is written for a reader checking it against the paper
(Bharadwaj et al., "Fast Exact Leverage Score Sampling from Khatri-Rao
Products with Applications to Tensor Decomposition", NeurIPS 2023):
nothing is blocked, fused or reordered beyond what the cited passage states.
Library primitives (matmul, eigh, qr, svd, lstsq, cumsum) serve as steps.

Conventions (readings of the paper, each listed in the design notes):
  * Row order of A = U_1 (.) ... (.) U_N is C order over (i_1..i_N): the
    last factor's index varies fastest (Table 6, Khatri-Rao row).
  * G^+ is the eigen-pseudo-inverse with eigenvalues <= R * 2^-52 * lam_max
    treated as zero; rank = number of kept eigenvalues.
  * Eigenvalues in ascending order; negative ones clamped to zero.
  * Inverse-CDF search: tau = u * total, pick the first bin whose right
    edge (cumulative sum) is >= tau; zero-weight bins are never picked.
  * G_{>k} = G^+ (*) prod_{m > k, m included} G_m (Eq. G_geq_k_defn).

Parity status: every function below is pinned by a CPU test against closed
forms, brute force or a library routine (tests/test_oracle_pins.py), except
where its docstring says "parity unpinned".
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32_10, sampler_uniforms, u32_to_open_unit

EPS64 = 2.0 ** -52


# ---------------------------------------------------------------------------
# Products and Grams (Table 6; Section 3 opening: G = AᵀA = ⊛ G_k)
# ---------------------------------------------------------------------------
def khatri_rao(Us):
    """A = U_1 ⊙ ... ⊙ U_N, rows in C order over (i_1..i_N) (Table 6)."""
    A = np.asarray(Us[0], dtype=np.float64)
    for U in Us[1:]:
        U = np.asarray(U, dtype=np.float64)
        # column r of the result is A[:, r] ⊗ U[:, r]; U's index is fastest
        A = (A[:, None, :] * U[None, :, :]).reshape(-1, A.shape[1])
    return A


def gram(U):
    """G_k = U_kᵀ U_k (Section 3)."""
    U = np.asarray(U, dtype=np.float64)
    return U.T @ U


def included_factors(N, exclude):
    """Included factors in ascending order, skipping `exclude` (Alg. 2)."""
    return [k for k in range(N) if k != exclude]


def hadamard_gram(Us, exclude=-1):
    """G = ⊛_{k != exclude} G_k, which equals AᵀA for A the KRP (Section 3)."""
    incl = included_factors(len(Us), exclude)
    G = np.ones((Us[0].shape[1],) * 2)
    for k in incl:
        G = G * gram(Us[k])
    return G


def pinv_eig(G):
    """Eigen-pseudo-inverse of a symmetric p.s.d. matrix.

    Returns (G⁺, rank).  Eigenvalues <= R * 2^-52 * lam_max are dropped.
    """
    lam, V = np.linalg.eigh(np.asarray(G, dtype=np.float64))
    R = G.shape[0]
    lam_max = max(float(lam.max()), 0.0)
    keep = lam > R * EPS64 * lam_max
    inv = np.zeros_like(lam)
    inv[keep] = 1.0 / lam[keep]
    return (V * inv) @ V.T, int(keep.sum())


# ---------------------------------------------------------------------------
# Leverage scores (Eq. leverage_definition and its QR restatement, Sec. 2.1)
# ---------------------------------------------------------------------------
def leverage_scores_qr(A):
    """ℓ_i = squared row norm of an orthonormal basis Q of range(A) (Sec. 2.1).

    The basis is the left singular vectors with nonzero singular values, so a
    rank-deficient A is handled; for full-rank A this is the reduced-QR Q.
    """
    A = np.asarray(A, dtype=np.float64)
    Uq, s, _ = np.linalg.svd(A, full_matrices=False)
    r = int((s > max(A.shape) * EPS64 * s.max()).sum()) if s.size else 0
    Q = Uq[:, :r]
    return (Q * Q).sum(axis=1), r


def leverage_scores_pinv(A):
    """ℓ_i = A[i,:] (AᵀA)⁺ A[i,:]ᵀ (Eq. leverage_definition)."""
    A = np.asarray(A, dtype=np.float64)
    Gp, r = pinv_eig(A.T @ A)
    return np.einsum("ia,ab,ib->i", A, Gp, A), r


def krp_leverage(Us, exclude=-1):
    """Exact leverage scores of every row of the KRP of the included factors,
    via ℓ_s = a_sᵀ G⁺ a_s with G = ⊛ G_k (Eq. krp_leverage; Section 3)."""
    incl = included_factors(len(Us), exclude)
    A = khatri_rao([Us[k] for k in incl])
    Gp, r = pinv_eig(hadamard_gram(Us, exclude))
    return np.einsum("ia,ab,ib->i", A, Gp, A), r


# ---------------------------------------------------------------------------
# Conditional distributions (Thm 3.1; Eqs. first_dist, second_conditional_dist)
# ---------------------------------------------------------------------------
def g_greater(Us, exclude, k, Gplus):
    """G_{>k} = G⁺ ⊛ ⊛_{m>k, m included} G_m (Eq. G_geq_k_defn)."""
    Gk = np.array(Gplus, dtype=np.float64, copy=True)
    for m in included_factors(len(Us), exclude):
        if m > k:
            Gk = Gk * gram(Us[m])
    return Gk


def eig_ascending(M):
    """Symmetric eigendecomposition, eigenvalues ascending, negatives clamped
    to zero (G_{>k} is p.s.d. by the Schur product theorem)."""
    lam, V = np.linalg.eigh(np.asarray(M, dtype=np.float64))
    return np.maximum(lam, 0.0), V


def conditional_q(h, U, Ygt):
    """q_{h,U,Y}[s] = ⟨hhᵀ, U[s]ᵀU[s], Y⟩ / C, C = ⟨hhᵀ, UᵀU, Y⟩ (Thm 3.1).

    Returns (q, C) for every row s of U.
    """
    U = np.asarray(U, dtype=np.float64)
    M = np.outer(h, h) * Ygt
    num = np.einsum("sa,ab,sb->s", U, M, U)
    C = float(np.sum(M * gram(U)))
    return num / C, C


def eigencomponent_weights(H, lam, V, Gk):
    """Unnormalised u-stage weights, one row per history vector h (Eq. first_dist):
    w[u] = λ_u (h ∘ V[:,u])ᵀ G_k (h ∘ V[:,u]).   H: (J, R) -> (J, R)."""
    X = H[:, :, None] * V[None, :, :]            # X[s, a, u] = h_a V[a, u]
    Xt = np.transpose(X, (0, 2, 1))              # (J, u, a)
    quad = np.einsum("sua,ab,sub->su", Xt, Gk, Xt)
    return quad * lam[None, :]


def row_weights(Ht, U):
    """Unnormalised t-stage weights (U[t] · h̃)² (Eq. second_conditional_dist,
    rank-1 leaf rule of Lemma 3.2 point 3).   Ht: (J, R), U: (I, R) -> (J, I)."""
    return (Ht @ np.asarray(U, dtype=np.float64).T) ** 2


def inverse_cdf(weights, u):
    """Inverse-CDF draw, one per row of `weights` (J, n), uniforms u (J,).

    tau = u * total; returns the first index whose cumulative sum reaches tau
    (the bin containing tau).  Also returns tau, the chosen bin's left and
    right edges and the total, for boundary analysis.
    """
    cum = np.cumsum(weights, axis=1)
    total = cum[:, -1]
    tau = u * total
    idx = (cum < tau[:, None]).sum(axis=1)
    n = weights.shape[1]
    # tau < total always holds in FP64 for u <= 1 - 2^-24; guard anyway:
    over = idx >= n
    if np.any(over):
        pos = weights[over] > 0
        idx[over] = n - 1 - np.argmax(pos[:, ::-1], axis=1)
    rows = np.arange(weights.shape[0])
    right = cum[rows, idx]
    left = np.where(idx > 0, cum[rows, np.maximum(idx - 1, 0)], 0.0)
    return idx, tau, left, right, total


# ---------------------------------------------------------------------------
# Alg. 1 + Alg. 2 replay (two-stage sampler, plain inverse CDF per stage)
# ---------------------------------------------------------------------------
class SamplerPrep:
    """Everything Alg. 2 computes before the per-sample loop:
    G, G⁺, rank, and for each included k: G_{>k} = V_k Λ_k V_kᵀ."""

    def __init__(self, Us, exclude=-1, eig_override=None):
        self.Us = [np.asarray(U, dtype=np.float64) for U in Us]
        self.N = len(Us)
        self.R = self.Us[0].shape[1]
        self.exclude = exclude
        self.incl = included_factors(self.N, exclude)
        self.grams = {k: gram(self.Us[k]) for k in self.incl}
        G = np.ones((self.R, self.R))
        for k in self.incl:
            G = G * self.grams[k]
        self.G = G
        self.Gplus, self.rank = pinv_eig(G)
        self.Ggt, self.lam, self.V = {}, {}, {}
        for k in self.incl:
            self.Ggt[k] = g_greater(self.Us, exclude, k, self.Gplus)
            if eig_override is not None and k in eig_override:
                lam, V = eig_override[k]
                self.lam[k] = np.maximum(np.asarray(lam, np.float64), 0.0)
                self.V[k] = np.asarray(V, np.float64)
            else:
                self.lam[k], self.V[k] = eig_ascending(self.Ggt[k])


def krp_sample(Us, exclude, J, seed, draw_id, d0=0, eig_override=None,
               chunk=16384, record=False, prep=None):
    """Draw samples d0..d0+J-1 by Alg. 2 with Philox uniforms.

    Returns dict with idx (n_incl, J) int64, weight (J,), q (J,), logq (J,),
    rank, and (if record) per-stage tau/left/right/total arrays
    shaped (n_incl, 2, J) with stage 0 = eigencomponent, 1 = row.
    The weight is 1/sqrt(J_total * q) with q = ℓ_s / rank (Sec. 2.1), where
    J_total is `J` (callers drawing a sub-range pass their own scaling).
    A SamplerPrep built for the same factors may be passed to skip the preparation
    (G, G⁺, the G_{>k} and their eigendecompositions).
    """
    if prep is None:
        prep = SamplerPrep(Us, exclude, eig_override)
    incl = prep.incl
    ni = len(incl)
    R = prep.R
    idx = np.zeros((ni, J), dtype=np.int64)
    uidx = np.zeros((ni, J), dtype=np.int64)
    rec = {key: np.zeros((ni, 2, J)) for key in ("tau", "left", "right", "total")}
    lev = np.zeros(J)
    for c0 in range(0, J, chunk):
        c1 = min(J, c0 + chunk)
        n = c1 - c0
        u_eig, u_row = sampler_uniforms(seed, draw_id, n, ni, d0=d0 + c0)
        H = np.ones((n, R))
        for p, k in enumerate(incl):
            # eigencomponent stage: draw u from w (Eq. first_dist)
            w = eigencomponent_weights(H, prep.lam[k], prep.V[k], prep.grams[k])
            u_k, tau, lft, rgt, tot = inverse_cdf(w, u_eig[:, p])
            uidx[p, c0:c1] = u_k
            for key, val in zip(("tau", "left", "right", "total"), (tau, lft, rgt, tot)):
                rec[key][p, 0, c0:c1] = val
            # row stage: draw t from (U_k[t] · (h ∘ V[:,u]))² (Eq. second_conditional_dist)
            Ht = H * prep.V[k][:, u_k].T
            wt = row_weights(Ht, prep.Us[k])
            t_k, tau, lft, rgt, tot = inverse_cdf(wt, u_row[:, p])
            idx[p, c0:c1] = t_k
            for key, val in zip(("tau", "left", "right", "total"), (tau, lft, rgt, tot)):
                rec[key][p, 1, c0:c1] = val
            H = H * prep.Us[k][t_k, :]          # h ∘= U_k[t_k, :]
        lev[c0:c1] = np.einsum("sa,ab,sb->s", H, prep.Gplus, H)
    q = lev / prep.rank
    out = dict(idx=idx, uidx=uidx, q=q, logq=np.log(q), weight=1.0 / np.sqrt(J * q),
               rank=prep.rank, prep=prep)
    if record:
        out.update(rec)
    return out


def sample_probability(Us, exclude, idx):
    """q_s = ℓ_s / rank for given index tuples (n_incl, J) (Sec. 2.1, Thm 1.1)."""
    prep = SamplerPrep(Us, exclude)
    H = np.ones((idx.shape[1], prep.R))
    for p, k in enumerate(prep.incl):
        H = H * prep.Us[k][idx[p], :]
    lev = np.einsum("sa,ab,sb->s", H, prep.Gplus, H)
    return lev / prep.rank, prep.rank


def linear_index(idx, dims):
    """C-order linear row index of the KRP for tuples idx (n_incl, J)."""
    lin = np.zeros(idx.shape[1], dtype=np.int64)
    for p, I in enumerate(dims):
        lin = lin * int(I) + idx[p]
    return lin


# ---------------------------------------------------------------------------
# Segment tree T_{I,F} (Sec. 3.1, Alg. 3, Alg. 4) in FP64
# ---------------------------------------------------------------------------
def tree_shape(I, F):
    """Leaves = ceil(I/F) padded to a power of two L; depth d = log2 L.
    Heap numbering: root 1, children 2v and 2v+1; leaf b is node L + b and
    holds rows [bF, min((b+1)F, I))."""
    nleaf = max(1, -(-I // F))
    L = 1
    while L < nleaf:
        L *= 2
    return L, L.bit_length() - 1


def node_rows(v, L, F, I):
    """Row range [lo, hi) of S(v): the union of its leaves' segments."""
    depth = v.bit_length() - 1
    d = L.bit_length() - 1
    span = 1 << (d - depth)                      # leaves under v
    b0 = (v - (1 << depth)) * span
    return min(b0 * F, I), min((b0 + span) * F, I)


def partial_gram(U, v, L, F):
    """G^v = Σ_{i ∈ S(v)} U[i]ᵀ U[i] (Eq. partial_gram), by definition."""
    U = np.asarray(U, dtype=np.float64)
    lo, hi = node_rows(v, L, F, U.shape[0])
    return U[lo:hi].T @ U[lo:hi]


def tree_row_sample(U, F, Y, h, u):
    """Alg. 4 (RowSample) in FP64 for one history vector h and uniform u.

    Node masses m(v) = ⟨hhᵀ, G^v, Y⟩; descend left iff tau <= low + m(L(c));
    a right child whose segment is empty (padding) is never entered.  At the
    leaf, scan rows with q̃[i] = U[i] (hhᵀ ∘ Y) U[i]ᵀ and return the first row
    whose cumulative edge reaches tau; zero-weight rows are skipped.
    Returns (row, [(m_left, m_node), ...] per level).
    """
    U = np.asarray(U, dtype=np.float64)
    I = U.shape[0]
    L, d = tree_shape(I, F)
    M = np.outer(h, h) * Y
    mass = lambda v: float(np.sum(M * partial_gram(U, v, L, F)))
    C = mass(1)
    tau = u * C
    c, low, m_c = 1, 0.0, C
    trace = []
    while c < L:
        m_left = mass(2 * c)
        trace.append((m_left, m_c))
        cutoff = low + m_left
        right_lo, _ = node_rows(2 * c + 1, L, F, I)
        if tau <= cutoff or right_lo >= I:
            c, m_c = 2 * c, m_left
        else:
            c, low, m_c = 2 * c + 1, cutoff, m_c - m_left
    lo, hi = node_rows(c, L, F, I)
    q = np.einsum("sa,ab,sb->s", U[lo:hi], M, U[lo:hi])
    cum = low + np.cumsum(q)
    hit = np.nonzero(cum >= tau)[0]
    if hit.size:
        return lo + int(hit[0]), trace
    pos = np.nonzero(q > 0)[0]
    return lo + int(pos[-1]), trace


def eig_tree_row_sample(lam, V, Gk, h, u):
    """Eigencomponent draw through Alg. 4 on E_k = BuildSampler(√Λ Vᵀ, F=1, G_k)
    (Alg. 2).  Rows of √Λ Vᵀ are √λ_u V[:,u]ᵀ."""
    W = (np.sqrt(np.maximum(lam, 0.0))[:, None] * V.T)
    return tree_row_sample(W, 1, Gk, h, u)


# ---------------------------------------------------------------------------
# Sketched least squares (Sec. 2.1, Thm 2.1); solved by QR-based lstsq.
# ---------------------------------------------------------------------------
def sketched_rows(Us, exclude, idx, weight):
    """SA[s,:] = w_s · ⊛_{k incl} U_k[s_k, :]."""
    incl = included_factors(len(Us), exclude)
    H = np.ones((idx.shape[1], Us[0].shape[1]))
    for p, k in enumerate(incl):
        H = H * np.asarray(Us[k], dtype=np.float64)[idx[p], :]
    return H * np.asarray(weight, np.float64)[:, None]


def lstsq(A, B):
    """argmin_X ||A X - B||_F in FP64 (library least squares)."""
    X, *_ = np.linalg.lstsq(np.asarray(A, np.float64), np.asarray(B, np.float64), rcond=None)
    return X


# ---------------------------------------------------------------------------
# Sparse CP-ALS with the sketched solve (Alg. 6; Sec. 3.3; fit, Sec. 4.3)
# ---------------------------------------------------------------------------
def fiber_table(coords, vals, j):
    """Map each tuple of the modes other than j to its mode-j fiber
    [(i_j, value), ...] (the nonzeros of one row of mat(T, j)ᵀ, App. A.9)."""
    N = coords.shape[0]
    others = [k for k in range(N) if k != j]
    table = {}
    for e in range(coords.shape[1]):
        key = tuple(int(coords[k, e]) for k in others)
        table.setdefault(key, []).append((int(coords[j, e]), float(vals[e])))
    return table


def cp_fit(coords, vals, sigma, Us):
    """fit = 1 - ||T̃ - T||_F / ||T||_F (Sec. 4.3), with
    ||T̃ - T||² = ||T||² - 2⟨T, T̃⟩ + ||T̃||², ||T̃||² = σᵀ(⊛ G_k)σ and
    ⟨T, T̃⟩ = Σ_nnz T[i] Σ_r σ_r Π_k U_k[i_k, r]."""
    vals = np.asarray(vals, np.float64)
    sigma = np.asarray(sigma, np.float64)
    normT2 = float(vals @ vals)
    G = np.ones((len(sigma),) * 2)
    for U in Us:
        G = G * gram(U)
    normM2 = float(sigma @ G @ sigma)
    P = np.ones((coords.shape[1], len(sigma)))
    for k, U in enumerate(Us):
        P = P * np.asarray(U, np.float64)[coords[k], :]
    inner = float(vals @ (P @ sigma))
    resid2 = max(normT2 - 2.0 * inner + normM2, 0.0)
    return 1.0 - np.sqrt(resid2) / np.sqrt(normT2)


def column_normalize(U):
    """σ[i] = ||U[:, i]||_2 and U[:, i] /= σ[i] (Alg. 6)."""
    U = np.asarray(U, np.float64)
    sigma = np.sqrt((U * U).sum(axis=0))
    safe = np.where(sigma > 0, sigma, 1.0)
    return U / safe[None, :], sigma


def sketched_mode_solve(Us, coords, vals, dims, j, J, seed, draw_id, table=None):
    """One sketched least-squares solve of Alg. 6 for mode j:
    U_j = argmin_X ||S U_{≠j} Xᵀ - S mat(T,j)ᵀ||_F with S drawn by Alg. 2
    (excluding j).  Returns (U_j unnormalised, sample dict)."""
    smp = krp_sample(Us, j, J, seed, draw_id)
    SA = sketched_rows(Us, j, smp["idx"], smp["weight"])
    if table is None:
        table = fiber_table(coords, vals, j)
    SB = np.zeros((J, dims[j]))
    for s in range(J):
        key = tuple(int(x) for x in smp["idx"][:, s])
        for (ij, v) in table.get(key, ()):
            SB[s, ij] += smp["weight"][s] * v
    X = lstsq(SA, SB)             # R x I_j
    return X.T, smp


def cp_als_sketched(coords, vals, dims, Us0, J, sweeps, seed, draw_base=0):
    """STS-CP (Alg. 6 with the exact-leverage sketched solve).
    Draw ids: draw_base + sweep * N + j.  Returns (sigma, Us, fits per sweep)."""
    N = len(dims)
    Us = [column_normalize(U)[0] for U in Us0]
    sigma = np.ones(Us[0].shape[1])
    tables = [fiber_table(coords, vals, j) for j in range(N)]
    fits = []
    for it in range(sweeps):
        for j in range(N):
            Uj, _ = sketched_mode_solve(Us, coords, vals, dims, j, J, seed,
                                        draw_base + it * N + j, tables[j])
            Us[j], sigma = column_normalize(Uj)
        fits.append(cp_fit(coords, vals, sigma, Us))
    return sigma, Us, fits


def cp_als_exact(coords, vals, dims, Us0, sweeps):
    """Non-randomised CP-ALS (Alg. 6) on a small sparse tensor, materialising
    mat(T, j) and U_{≠j}; used to pin the sketched sweep's fixed point."""
    N = len(dims)
    Us = [column_normalize(U)[0] for U in Us0]
    sigma = np.ones(Us[0].shape[1])
    T = np.zeros(dims)
    T[tuple(coords)] = vals
    fits = []
    for _ in range(sweeps):
        for j in range(N):
            others = [k for k in range(N) if k != j]
            A = khatri_rao([Us[k] for k in others])              # C order over others
            B = np.moveaxis(T, j, -1).reshape(-1, dims[j])        # rows: others in C order
            Uj = lstsq(A, B).T
            Us[j], sigma = column_normalize(Uj)
        fits.append(cp_fit(coords, vals, sigma, Us))
    return sigma, Us, fits


# ---------------------------------------------------------------------------
# Batched FP64 replay of Alg. 3 (BuildSampler) + Alg. 4 (RowSample) for many
# samples at once, for factors too tall for the linear inverse CDF.  In exact
# arithmetic it returns the same indices as krp_sample (Sec. 3.1); the pin
# test checks that on small cases.
# ---------------------------------------------------------------------------
class TreeFP64:
    """All node Grams of T_{I,F} in FP64, heap-numbered (root 1, children 2v, 2v+1;
    leaf b = node L + b), built bottom-up by Alg. 3 (leaf Grams, then parent =
    left + right).  Empty padding leaves hold zero."""

    def __init__(self, U, F):
        U = np.asarray(U, dtype=np.float64)
        self.I, self.R = U.shape
        self.F = F
        self.L, self.d = tree_shape(self.I, F)
        nleaf_rows = self.L * F
        Up = np.zeros((nleaf_rows, self.R))
        Up[: self.I] = U
        blocks = Up.reshape(self.L, F, self.R)
        nodes = np.zeros((2 * self.L, self.R, self.R))
        nodes[self.L:] = np.matmul(np.transpose(blocks, (0, 2, 1)), blocks)      # leaf Grams
        for v in range(self.L - 1, 0, -1):
            nodes[v] = nodes[2 * v] + nodes[2 * v + 1]
        self.nodes = nodes
        self.U = U

    def masses(self, v, Y_h):
        """m(v) = ⟨hhᵀ, G^v, Y⟩ for node ids v (J,) and matrices Y_h = hhᵀ ∘ Y (J,R,R)."""
        return np.einsum("sab,sab->s", self.nodes[v], Y_h)


def tree_update_entry(tree, r, c, u_new):
    """UpdateSampler (App. A, efficient single-element updates) on an FP64 tree:
    U[r, c] := u_new.  With d = u_new - U[r, c] and the old row x = U[r, :],
    the leaf holding row r gets G[c, :] += d x, G[:, c] += d xᵀ, G[c, c] += d²;
    every ancestor is then the sum of its two children again, which changes
    only its row and column c.  Modifies tree.nodes and tree.U in place."""
    U = tree.U if tree.U.flags.writeable else tree.U.copy()
    x = U[r].copy()
    d = float(u_new) - x[c]
    v = tree.L + r // tree.F
    G = tree.nodes[v]
    G[c, :] += d * x
    G[:, c] += d * x
    G[c, c] += d * d
    while v > 1:
        prev, v = v, v // 2
        sib = prev ^ 1
        tree.nodes[v] = tree.nodes[sib] + tree.nodes[prev]
    U[r, c] = u_new
    tree.U = U
    return tree


def tree_sample_batch(tree, Y, H, u):
    """Alg. 4 for J history vectors H (J,R) and uniforms u (J,), Y p.s.d.
    Returns (rows, tau, left_edges, right_edges, C) — edges of the chosen bin."""
    J = H.shape[0]
    M = H[:, :, None] * H[:, None, :] * Y[None, :, :]
    C = tree.masses(np.ones(J, dtype=np.int64), M)
    tau = u * C
    c = np.ones(J, dtype=np.int64)
    low = np.zeros(J)
    L, d, F, I = tree.L, tree.d, tree.F, tree.I
    for lvl in range(d):
        mL = tree.masses(2 * c, M)
        cutoff = low + mL
        span = 1 << (d - lvl - 1)
        right_first_row = ((2 * c + 1) * span - L) * F
        go_left = (tau <= cutoff) | (right_first_row >= I)
        low = np.where(go_left, low, cutoff)
        c = np.where(go_left, 2 * c, 2 * c + 1)
    b = c - L
    rows = np.zeros(J, dtype=np.int64)
    left = np.zeros(J)
    right = np.zeros(J)
    for s in range(J):
        lo, hi = b[s] * F, min(b[s] * F + F, I)
        Ub = tree.U[lo:hi]
        q = np.einsum("sa,ab,sb->s", Ub, M[s], Ub)
        cum = low[s] + np.cumsum(q)
        hit = np.nonzero(cum >= tau[s])[0]
        t = hit[0] if hit.size else np.nonzero(q > 0)[0][-1]
        rows[s] = lo + t
        right[s] = cum[t]
        left[s] = cum[t] - q[t]
    return rows, tau, left, right, C


def krp_sample_tree(Us, exclude, J, seed, draw_id, F, d0=0, prep=None, trees=None):
    """Alg. 2 with every stage drawn through Alg. 4 on FP64 segment trees
    (E_k with F = 1 and Y = G_k; Z_k with leaf size F and Y = [1]).
    Returns the same dict fields as krp_sample(record=True)."""
    if prep is None:
        prep = SamplerPrep(Us, exclude)
    incl = prep.incl
    R = prep.R
    if trees is None:
        trees = {k: TreeFP64(prep.Us[k], F) for k in incl}
    u_eig, u_row = sampler_uniforms(seed, draw_id, J, len(incl), d0=d0)
    H = np.ones((J, R))
    out = {key: np.zeros((len(incl), 2, J)) for key in ("tau", "left", "right", "total")}
    idx = np.zeros((len(incl), J), dtype=np.int64)
    uidx = np.zeros((len(incl), J), dtype=np.int64)
    for p, k in enumerate(incl):
        Wk = np.sqrt(np.maximum(prep.lam[k], 0.0))[:, None] * prep.V[k].T
        etree = TreeFP64(Wk, 1)
        u_k, tau, lft, rgt, C = tree_sample_batch(etree, prep.grams[k], H, u_eig[:, p])
        uidx[p] = u_k
        for key, val in zip(("tau", "left", "right", "total"), (tau, lft, rgt, C)):
            out[key][p, 0] = val
        Ht = H * prep.V[k][:, u_k].T
        t_k, tau, lft, rgt, C = tree_sample_batch(trees[k], np.ones((R, R)), Ht, u_row[:, p])
        idx[p] = t_k
        for key, val in zip(("tau", "left", "right", "total"), (tau, lft, rgt, C)):
            out[key][p, 1] = val
        H = H * prep.Us[k][t_k, :]
    lev = np.einsum("sa,ab,sb->s", H, prep.Gplus, H)
    q = lev / prep.rank
    out.update(idx=idx, uidx=uidx, q=q, logq=np.log(q), weight=1.0 / np.sqrt(J * q), rank=prep.rank, prep=prep)
    return out


def planted_rhs(Us, exclude, idx, X_true, sigma, seed):
    """Rows of a planted right-hand side B = A X_true + sigma * xi at the sampled
    tuples idx (n_incl x J): row s is a_s X_true + sigma xi(s, :), a_s the row of
    A = ⊙ U_k (included factors).  xi(s, c) is a standard normal by Box–Muller
    from Philox4x32-10 (key = seed halves, counter = (lin lo32, lin hi32, c,
    0x9E3779B9), lin = the C-order linear index of the tuple mod 2^64), so a
    repeated tuple gets the same noise.  A workload generator, not part of the
    method: the sketched solve of Thm 2.1 sees only these rows."""
    incl = included_factors(len(Us), exclude)
    idx = np.asarray(idx, dtype=np.int64)
    J = idx.shape[1]
    A = sketched_rows(Us, exclude, idx, np.ones(J))
    lin = np.zeros(J, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for p, k in enumerate(incl):
            lin = lin * np.uint64(Us[k].shape[0]) + idx[p].astype(np.uint64)
    X_true = np.asarray(X_true, dtype=np.float64)
    nrhs = X_true.shape[1]
    seed = int(seed)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    ctr = np.zeros((J, nrhs, 4), dtype=np.uint32)
    ctr[..., 0] = (lin & np.uint64(0xFFFFFFFF)).astype(np.uint32)[:, None]
    ctr[..., 1] = (lin >> np.uint64(32)).astype(np.uint32)[:, None]
    ctr[..., 2] = np.arange(nrhs, dtype=np.uint32)[None, :]
    ctr[..., 3] = np.uint32(0x9E3779B9)
    w = philox4x32_10(ctr, key)
    u1, u2 = u32_to_open_unit(w[..., 0]), u32_to_open_unit(w[..., 1])
    xi = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return A @ X_true + float(sigma) * xi


def sketch_distortion(Us, exclude, idx, weight):
    """Distortion D(S, A) = kappa(SQ) - 1 (Sec. 4.2, Eq. distortion_defn) by its
    definition: Q = orthonormal basis of range(A) from the SVD of the
    materialised A (rank from the SVD), SQ = the sampled, reweighted rows of Q,
    kappa = largest / smallest nonzero singular value.  Small cases only."""
    incl = included_factors(len(Us), exclude)
    A = khatri_rao([np.asarray(Us[k], np.float64) for k in incl])
    Uq, sv, _ = np.linalg.svd(A, full_matrices=False)
    r = int((sv > A.shape[1] * np.finfo(float).eps * sv[0]).sum())
    Q = Uq[:, :r]
    lin = linear_index(np.asarray(idx, np.int64), tuple(Us[k].shape[0] for k in incl))
    SQ = np.asarray(weight, np.float64)[:, None] * Q[lin]
    s = np.linalg.svd(SQ, compute_uv=False)
    s = s[s > s[0] * 1e-13]
    return s[0] / s[-1] - 1.0


def kron_rows(cs, exclude, idx):
    """Entries of b = c_1 ⊗ ... ⊗ c_N (Sec. 4.2's right-hand side) at the sampled
    tuples: b[t] = Π_k c_k[t_k] over the included factors."""
    incl = included_factors(len(cs), exclude)
    out = np.ones(np.asarray(idx).shape[1])
    for p, k in enumerate(incl):
        out = out * np.asarray(cs[k], np.float64)[np.asarray(idx[p], np.int64)]
    return out


def kron_lstsq_residual(Us, exclude, cs, x):
    """||A x - b|| for A = ⊙ U_k and b = ⊗ c_k without materialising either:
    ||Ax - b||² = xᵀ(⊛ U_kᵀU_k)x - 2 xᵀ(⊛ U_kᵀ c_k) + Π ||c_k||², with the
    column identity Aᵀb = ⊛_k U_kᵀ c_k (each column of A is ⊗_k U_k[:, r])."""
    incl = included_factors(len(Us), exclude)
    G = hadamard_gram([Us[k] for k in incl])
    Atb = np.ones(np.asarray(Us[incl[0]]).shape[1])
    bb = 1.0
    for k in incl:
        U = np.asarray(Us[k], np.float64)
        c = np.asarray(cs[k], np.float64)
        Atb = Atb * (U.T @ c)
        bb *= float(c @ c)
    x = np.asarray(x, np.float64)
    return float(np.sqrt(max(x @ G @ x - 2.0 * x @ Atb + bb, 0.0))), G, Atb
