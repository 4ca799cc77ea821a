"""Sparse path (sampled-fiber lookup, SBᵀSA, Y M⁻¹, ALS sweep, fit) vs the
FP64 oracle, through the C ABI; plus the bounded-wait status path."""
import numpy as np
import pytest
import torch

from oracle import krp_oracle as O
from paper_2301_12584_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2301_12584_gb300 import build as B
    from paper_2301_12584_gb300 import krpls
    if not os.path.exists(krpls.LIB_PATH):
        B.build()
    krpls.lib()


def make(dims, R, coords, vals, Us, prec=0):
    from paper_2301_12584_gb300.krpls import Sampler, SparseTensor
    s = Sampler(list(dims), R, 0, prec)
    for k, U in enumerate(Us):
        s.set_factor(k, torch.from_numpy(np.ascontiguousarray(U, np.float32)).to(DEV))
    t = SparseTensor(dims, coords, vals)
    return s, t


# I_j spans several row tiles of Y M⁻¹ (64, 128 or 256 rows) with a ragged
# tail; R covers each padded width (32, 64, 128) and R % 4 != 0.  prec 1 and
# 3 (BF16x3, TF32x3 samplers) take Y M⁻¹ on the tensor cores as TF32x3 for
# 64 <= R <= 104.
@pytest.mark.parametrize("prec", [0, 1, 3])
@pytest.mark.parametrize("dims,R,J,nnz", [((60, 50, 20), 6, 3000, 4000), ((700, 40, 30), 40, 3000, 20000),
                                          ((300, 33, 29), 50, 3000, 15000), ((520, 30, 24), 100, 4000, 20000),
                                          ((1100, 40, 30), 104, 4000, 30000)])
def test_sparse_solve_matches_oracle_on_gpu_samples(dims, R, J, nnz, prec):
    coords, vals = synth.sparse_zipf_tensor(dims, nnz, seed=3)
    Us = synth.gaussian_factors(3, list(dims), R, seed=4)
    s, t = make(dims, R, coords, vals, Us, prec)
    U64 = [U.astype(np.float64) for U in Us]
    for j in range(3):
        idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
        w = torch.zeros(J, device=DEV)
        SA = torch.zeros((J, R), device=DEV)
        s.sample(j, J, 7, j, idx, w, None, SA)
        Uo = torch.zeros((dims[j], R), device=DEV)
        s.solve_sparse(t, j, J, idx, w, SA, Uo)
        assert s.sync_status() == 0, s.last_error()
        gi = idx.cpu().numpy().astype(np.int64)[[k for k in range(3) if k != j]]
        wg = w.cpu().numpy().astype(np.float64)
        SAg = SA.cpu().numpy().astype(np.float64)
        table = O.fiber_table(coords, vals.astype(np.float64), j)
        SB = np.zeros((J, dims[j]))
        for sm in range(J):
            for (ij, v) in table.get(tuple(int(x) for x in gi[:, sm]), ()):
                SB[sm, ij] += wg[sm] * v
        X = O.lstsq(SAg, SB).T
        got = Uo.cpu().numpy()
        err = np.linalg.norm(got - X) / np.linalg.norm(X)
        assert err < 1e-4, (j, err)
    s.close()
    t.close()


def test_fit_kernel_matches_oracle():
    dims = (30, 40, 25)
    coords, vals = synth.sparse_zipf_tensor(dims, 3000, seed=5)
    R = 5
    Us = synth.gaussian_factors(3, list(dims), R, seed=6)
    s, t = make(dims, R, coords, vals, Us)
    sigma = np.array([1.0, 0.5, 2.0, 0.3, 1.2], np.float32)
    fit = s.cp_fit(t, torch.from_numpy(sigma).to(DEV))
    ref = O.cp_fit(coords, vals.astype(np.float64), sigma.astype(np.float64), [U.astype(np.float64) for U in Us])
    assert abs(fit - ref) <= 1e-6 * max(1.0, abs(ref)), (fit, ref)
    s.close()
    t.close()


@pytest.mark.parametrize("dims,R", [((300, 200, 40), 37), ((520, 300, 90), 100)])
def test_sweep_normalises_columns(dims, R):
    """After a sweep every factor has unit columns and sigma holds the norms
    the last solve produced (column sums of squares fused into Y M⁻¹)."""
    from paper_2301_12584_gb300.krpls import Sampler, SparseTensor
    coords, vals = synth.sparse_zipf_tensor(dims, 30000, seed=12)
    Us = synth.gaussian_factors(3, list(dims), R, seed=13)
    s, t = make(dims, R, coords, vals, Us)
    J = 2048
    idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, device=DEV)
    SA = torch.zeros((J, R), device=DEV)
    sigma = torch.zeros(R, device=DEV)
    s.cp_als_sweep(t, J, 5, 0, sigma)
    assert s.sync_status() == 0, s.last_error()
    for k in range(3):
        U = s.get_factor(k).astype(np.float64)
        np.testing.assert_allclose(np.linalg.norm(U, axis=0), 1.0, rtol=2e-6)
    # sigma: norms of the last mode's U_j = Y M⁻¹ before scaling, replayed on a
    # second sampler holding the swept factors 0 and 1 (same seed and draw id)
    s2, t2 = make(dims, R, coords, vals, Us)
    for k in range(2):
        s2.set_factor(k, torch.from_numpy(np.ascontiguousarray(s.get_factor(k), np.float32)).to(DEV))
    s2.set_factor(2, torch.from_numpy(np.ascontiguousarray(Us[2], np.float32)).to(DEV))
    s2.sample(2, J, 5, 2, idx, w, None, SA)
    Uo = torch.zeros((dims[2], R), device=DEV)
    s2.solve_sparse(t2, 2, J, idx, w, SA, Uo)
    assert s2.sync_status() == 0, s2.last_error()
    norms = np.linalg.norm(Uo.cpu().numpy().astype(np.float64), axis=0)
    np.testing.assert_allclose(sigma.cpu().numpy(), norms, rtol=1e-4)
    for x in (s, t, s2, t2):
        x.close()


@pytest.mark.parametrize("dims,rank,sweeps,converges", [((12, 10, 8), 3, 6, False), ((6, 7, 5), 2, 8, True)])
def test_als_sweeps_match_oracle(dims, rank, sweeps, converges):
    """STS-CP sweeps (Alg. 6) on a planted exactly-low-rank tensor: the fit after
    every sweep matches the oracle's sketched ALS (same Philox draws) within
    1e-3 relative.  The rank-3 start stalls in an ALS swamp (so does exact ALS,
    fit 0.653); the rank-2 case converges (fit > 0.99)."""
    coords, vals = synth.planted_dense_tensor(dims, rank, seed=7 if rank == 3 else 3)
    R, J = rank, 400 if rank == 3 else 300
    if rank == 3:
        U0 = synth.gaussian_factors(3, list(dims), R, seed=8)
    else:   # the start of the CPU pin test, which converges
        U0 = [np.random.default_rng(9).standard_normal((d, 2)).astype(np.float32) for d in dims]
    U0n = [O.column_normalize(U.astype(np.float64))[0].astype(np.float32) for U in U0]
    s, t = make(dims, R, coords, vals, U0n)
    sigma = torch.zeros(R, device=DEV)
    fits = []
    for it in range(sweeps):
        s.cp_als_sweep(t, J, 11, it * 3, sigma)
        assert s.sync_status() == 0, s.last_error()
        fits.append(s.cp_fit(t, sigma))
    _, _, ofits = O.cp_als_sketched(coords, vals.astype(np.float64), dims, [U.astype(np.float64) for U in U0n],
                                   J=J, sweeps=sweeps, seed=11)
    np.testing.assert_allclose(fits, ofits, rtol=1e-3)
    if converges:
        assert fits[-1] > 0.99, fits
    s.close()
    t.close()


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2301_12584_gb300.krpls import Sampler
    s = Sampler([16, 16], 4, 0)
    s.debug_wait_timeout(20)
    assert s.sync_status() == -7          # KRP_ETIMEOUT
    # the context is still usable
    Us = synth.gaussian_factors(2, 16, 4, seed=1)
    for k in range(2):
        s.set_factor(k, torch.from_numpy(Us[k]).to(DEV))
    idx = torch.zeros((2, 64), dtype=torch.int32, device=DEV)
    w = torch.zeros(64, device=DEV)
    s.sample(-1, 64, 1, 0, idx, w)
    assert s.sync_status() == 0
    s.close()


def test_graph_replay_of_sampler_calls():
    """Sampler calls captured as a CUDA graph replay bit for bit: a dense
    sketch-and-solve sequence, and a whole STS-CP sweep (the sparse solve adds
    in a fixed order: sorted runs instead of atomics), whose factors, trees,
    sigma and fit equal the direct sweep's exactly."""
    from paper_2301_12584_gb300.krpls import Sampler, SparseTensor
    dims, R, J = (40, 30, 20), 4, 2000
    coords, vals = synth.sparse_zipf_tensor(dims, 3000, seed=8)
    Us = synth.gaussian_factors(3, list(dims), R, seed=9)
    stream = torch.cuda.Stream()
    s = Sampler(list(dims), R, 0, stream=stream)
    t = SparseTensor(dims, coords, vals)
    sigma = torch.zeros(R, device=DEV)

    def reset():
        for k, U in enumerate(Us):
            s.set_factor(k, torch.from_numpy(U).to(DEV))
        torch.cuda.synchronize()

    # (1) dense sequence, bit for bit
    reset()
    idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, device=DEV)
    SA = torch.zeros((J, R), device=DEV)
    B = torch.zeros((J, 2), device=DEV)
    X = torch.zeros((R, 2), device=DEV)
    Xt = torch.from_numpy(synth.planted_solution(R, 2, seed=1)).to(DEV)

    def dense():
        s.sample(-1, J, 4, 1, idx, w, None, SA)
        s.planted_rows(-1, J, idx, Xt, 2, 0.01, 3, B)
        s.solve_dense(J, SA, w, B, 2, X)

    dense()
    assert s.sync_status() == 0
    ref = [x.clone() for x in (idx, w, SA, B, X)]
    for x in (idx, w, SA, B, X):
        x.zero_()
    torch.cuda.synchronize()
    s.capture_begin()
    dense()
    assert s.capture_end() >= 4
    assert float(X.abs().sum()) == 0.0                 # recorded, not run
    s.replay()
    assert s.sync_status() == 0
    for a, b in zip(ref, (idx, w, SA, B, X)):
        assert torch.equal(a, b)
    # (2) a whole sweep
    reset()
    s.cp_als_sweep(t, J, 5, 0, sigma)                 # allocates the sweep buffers
    assert s.sync_status() == 0, s.last_error()
    reset()
    s.cp_als_sweep(t, J, 5, 10, sigma)
    assert s.sync_status() == 0
    direct_trees = [s.get_tree(k).copy() for k in range(3)]
    direct_factors = [s.get_factor(k).copy() for k in range(3)]
    direct_sigma = sigma.clone()
    direct_fit = s.cp_fit(t, sigma)
    reset()
    sigma.zero_()
    torch.cuda.synchronize()
    s.capture_begin()
    s.cp_als_sweep(t, J, 5, 10, sigma)
    assert s.capture_end() > 10
    assert float(sigma.abs().sum()) == 0.0
    s.replay()
    assert s.sync_status() == 0
    for k in range(3):
        assert np.array_equal(s.get_factor(k), direct_factors[k])
        assert np.array_equal(s.get_tree(k), direct_trees[k])
    assert torch.equal(sigma, direct_sigma)
    assert s.cp_fit(t, sigma) == direct_fit
    s.close()
    t.close()


@pytest.mark.parametrize("n,bits", [(1, 8), (100, 8), (2047, 13), (2048, 22), (2049, 32), (100003, 22),
                                    (1 << 20, 32)])
def test_radix_sort_is_stable(n, bits):
    """The sort behind the deterministic sparse solve against NumPy's stable
    argsort, on keys with many repeats (values = input positions)."""
    from paper_2301_12584_gb300.krpls import debug_sort_pairs
    rng = np.random.default_rng(n + bits)
    hi = min(1 << bits, max(2, n // 7))
    keys = rng.integers(0, hi, n, dtype=np.uint64).astype(np.uint32)
    keys[rng.random(n) < 0.1] = np.uint32((1 << bits) - 1)          # the largest key, repeated
    kd = torch.from_numpy(keys.view(np.int32).copy()).to(DEV)
    vd = torch.arange(n, dtype=torch.int32, device=DEV)
    debug_sort_pairs(kd, vd, bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kd.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(vd.cpu().numpy(), order.astype(np.int32))


def test_sparse_solve_repeats_bit_for_bit():
    """The same sparse solve twice (and a fresh tensor index) gives identical
    U_j: every sum of the solve is taken in a fixed order."""
    from paper_2301_12584_gb300.krpls import SparseTensor
    dims, R, J = (3000, 2000, 60), 24, 1 << 15
    coords, vals = synth.sparse_zipf_tensor(dims, 200000, seed=21)
    Us = synth.gaussian_factors(3, list(dims), R, seed=22)
    s, t = make(dims, R, coords, vals, Us)
    t2 = SparseTensor(dims, coords, vals)
    for j in range(3):
        idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
        w = torch.zeros(J, device=DEV)
        SA = torch.zeros((J, R), device=DEV)
        s.sample(j, J, 3, j, idx, w, None, SA)
        outs = []
        for tt in (t, t, t2):
            Uo = torch.zeros((dims[j], R), device=DEV)
            s.solve_sparse(tt, j, J, idx, w, SA, Uo)
            assert s.sync_status() == 0, s.last_error()
            outs.append(Uo)
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    for x in (s, t, t2):
        x.close()


def test_sparse_solve_full_key_width():
    """Dims 2^22 x 2^22 x 2^14 (keys of 22 + 22 and 22 + 14 bits), J = 2^16
    samples per solve.  The factors are N(0,1) on 40 rows per mode spread over
    the whole index range (the largest index included) and zero elsewhere, so
    every sample lands on a tuple of those rows, and the ~7000 nonzeros lie on
    them too, several fibers holding every one of their mode's 40 rows.  Each
    mode's U_j against the FP64 lstsq on the GPU's own samples, restricted to
    the rows the sampled fibers touch (every other row of U_j must be 0)."""
    dims = (1 << 22, 1 << 22, 1 << 14)
    R, J, nsup = 8, 1 << 16, 40
    rng = np.random.default_rng(51)
    sup = [np.sort(np.concatenate([rng.choice(d - 1, nsup - 1, replace=False), [d - 1]])) for d in dims]
    full = set()
    for _ in range(25):                      # long fibers: all 40 rows of the third mode
        a, b = rng.integers(nsup, size=2)
        full.update((int(sup[0][a]), int(sup[1][b]), int(sup[2][c])) for c in range(nsup))
    for _ in range(25):                      # and of the first
        b, c = rng.integers(nsup, size=2)
        full.update((int(sup[0][a]), int(sup[1][b]), int(sup[2][c])) for a in range(nsup))
    while len(full) < 7000:
        a, b, c = rng.integers(nsup, size=3)
        full.add((int(sup[0][a]), int(sup[1][b]), int(sup[2][c])))
    coords = np.array(sorted(full), dtype=np.int32).T.copy()
    vals = rng.lognormal(0.0, 0.5, coords.shape[1]).astype(np.float32)
    Us = []
    for k, d in enumerate(dims):
        U = np.zeros((d, R), np.float32)
        U[sup[k]] = rng.standard_normal((nsup, R)).astype(np.float32)
        Us.append(U)
    s, t = make(dims, R, coords, vals, Us)
    for j in range(3):
        idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
        w = torch.zeros(J, device=DEV)
        SA = torch.zeros((J, R), device=DEV)
        s.sample(j, J, 11, j, idx, w, None, SA)
        Uo = torch.zeros((dims[j], R), device=DEV)
        s.solve_sparse(t, j, J, idx, w, SA, Uo)
        assert s.sync_status() == 0, s.last_error()
        gi = idx.cpu().numpy().astype(np.int64)[[k for k in range(3) if k != j]]
        wg = w.cpu().numpy().astype(np.float64)
        SAg = SA.cpu().numpy().astype(np.float64)
        table = O.fiber_table(coords, vals.astype(np.float64), j)
        cols = {int(x): q for q, x in enumerate(sup[j])}
        SB = np.zeros((J, nsup))
        hits = 0
        for sm in range(J):
            fib = table.get(tuple(int(x) for x in gi[:, sm]), ())
            hits += bool(fib)
            for (ij, v) in fib:
                SB[sm, cols[ij]] += wg[sm] * v
        assert hits > J // 10, hits              # the sampled tuples do reach the fibers
        X = O.lstsq(SAg, SB).T                    # rows of U_j at the support rows
        got = Uo.cpu().numpy()
        err = np.linalg.norm(got[sup[j]] - X) / np.linalg.norm(X)
        assert err < 1e-4, (j, err)
        off = np.ones(got.shape[0], dtype=bool)
        off[sup[j]] = False
        assert not np.any(got[off])               # every other row is exactly 0
    s.close()
    t.close()
