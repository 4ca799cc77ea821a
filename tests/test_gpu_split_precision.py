"""Split-precision segment trees (BF16x3 and TF32x3 leaf Grams on tcgen05) vs
the FP64 oracle, through the C ABI.

Error bar of a BF16x3 product: with x = hi + lo + d, |x - hi| <= 2^-9 |x| and
|d| <= 2^-18 |x|, the three products miss lo*lo' and the d terms, at most
3 * 2^-18 |x||y| ~ 1.2e-5 |x||y|.  The tensor cores' FP32 accumulation does
not round each addition to nearest (measured worst total 2.5e-5), so every
tree entry must lie within 5e-5 * (|U|ᵀ|U| over the node's rows) of the exact
Gram (the FP32 build's bar is 2e-5).  Node masses inherit
~1e-5 relative error, so sampled indices may flip where a uniform lies within
about 1e-4 C of a bin edge; every mismatch must be such a flip.

TF32x3: |x - hi| <= 2^-11 |x| and the split keeps ~22 bits, so the three
products miss at most ~3 * 2^-22 |x||y| ~ 7e-7 |x||y|; with the tensor
cores' accumulation the trees are held to the FP32 build's 2e-5 bar
(measured worst 3.2e-6).  A node mass sums R^2 such entries of both signs,
so at R = 64 its relative error can reach ~1e-5 and flips are exempted
within 1e-4 C of an edge, as for BF16x3.
"""
import numpy as np
import pytest
import torch

from oracle import krp_oracle as O
from paper_2301_12584_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
BF16X3 = 1
TF32X3 = 3
TREE_BAR = {BF16X3: 5e-5, TF32X3: 2e-5}
EDGE_TOL = {BF16X3: 1e-4, TF32X3: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2301_12584_gb300 import build as B
    from paper_2301_12584_gb300 import krpls
    if not os.path.exists(krpls.LIB_PATH):
        B.build()
    krpls.lib()


def sampler_for(Us, F, prec):
    from paper_2301_12584_gb300.krpls import Sampler
    s = Sampler([U.shape[0] for U in Us], Us[0].shape[1], F, prec)
    for k, U in enumerate(Us):
        s.set_factor(k, torch.from_numpy(np.ascontiguousarray(U, dtype=np.float32)).to(DEV))
    return s


def unpack(slot, R):
    G = np.zeros((R, R))
    iu = np.triu_indices(R)
    G[iu] = slot[:len(iu[0])]
    return G + np.triu(G, 1).T


@pytest.mark.parametrize("I,R,F", [(64, 8, 8), (1000, 8, 8), (37, 5, 3), (5, 8, 8), (20000, 32, 32),
                                   (3001, 25, 25), (700, 64, 64), (300, 128, 128), (100, 3, 1), (4096, 16, 16),
                                   (5000, 32, 20), (999, 50, 50), (3000, 100, 100), (1001, 70, 70),
                                   (777, 90, 60)])
@pytest.mark.parametrize("prec", [BF16X3, TF32X3])
def test_split_tree_matches_partial_grams(I, R, F, prec):
    rng = np.random.default_rng(I * 7 + R)
    U = rng.standard_normal((I, R)).astype(np.float32)
    U[rng.choice(I, max(1, I // 100), replace=False)] *= 100.0
    s = sampler_for([U], F, prec)
    assert s.sync_status() == 0, s.last_error()
    # the leaf kernel also wrote the sampler's copy of the rows (ragged tails included)
    assert np.array_equal(s.get_factor(0), U)
    L, d, Tp = s.tree_info(0)
    tree = s.get_tree(0)
    U64 = U.astype(np.float64)
    T = R * (R + 1) // 2
    worst = 0.0
    for slot in range(L):
        h = 1 if slot == 0 else 2 * slot
        lo, hi = O.node_rows(h, L, F, I)
        ref = U64[lo:hi].T @ U64[lo:hi]
        bound = np.abs(U64[lo:hi]).T @ np.abs(U64[lo:hi])
        got = unpack(tree[slot], R)
        assert np.all(tree[slot][T:] == 0)
        err = np.abs(got - ref)
        assert np.all(err <= TREE_BAR[prec] * bound + 1e-30), (slot, (err / (bound + 1e-300)).max())
        worst = max(worst, float((err / (bound + 1e-300)).max()))
    print(f"prec {prec} I={I} R={R} F={F}: worst |err| / (|U|ᵀ|U|) = {worst:.2e}")
    s.close()


@pytest.mark.parametrize("prec", [BF16X3, TF32X3])
def test_split_fused_copy_and_gather(prec):
    """set_factor from a device buffer copies the rows inside the tensor-core
    leaf kernel; the gathered sketch rows must be the oracle's rows exactly."""
    Us = synth.gaussian_factors(3, [300, 257, 129], 32, seed=21)
    s = sampler_for(Us, 32, prec)
    J, R = 2048, 32
    idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, device=DEV)
    SA = torch.zeros((J, R), device=DEV)
    s.sample(-1, J, 3, 0, idx, w, None, SA)
    assert s.sync_status() == 0, s.last_error()
    gi = idx.cpu().numpy().astype(np.int64)
    U64 = [U.astype(np.float64) for U in Us]
    rows = O.sketched_rows(U64, -1, gi, w.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(SA.cpu().numpy(), rows, rtol=2e-6, atol=1e-30)
    s.close()


@pytest.mark.parametrize("prec", [BF16X3, TF32X3])
@pytest.mark.parametrize("case", ["cfg_tiny", "R32", "R64"])
def test_split_sampler_parity(case, prec):
    if case == "cfg_tiny":
        Us, F, J = synth.gaussian_factors(3, 64, 8, seed=0), 8, 1 << 15
    elif case == "R32":
        Us, F, J = synth.skewed_row_factors(3, 2000, 32, seed=9), 32, 1 << 14
    else:
        Us, F, J = synth.uniform_factors(3, 300, 64, seed=11), 64, 1 << 12
    s = sampler_for(Us, F, prec)
    N = len(Us)
    idx = torch.zeros((N, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, device=DEV)
    s.sample(-1, J, 12345, 3, idx, w)
    assert s.sync_status() == 0, s.last_error()
    gi = idx.cpu().numpy().astype(np.int64)
    U64 = [U.astype(np.float64) for U in Us]
    ref = O.krp_sample(U64, -1, J, 12345, 3, record=True, chunk=2048)
    diff = gi != ref["idx"]
    bad = np.nonzero(diff.any(axis=0))[0]
    for sm in bad:
        p = int(np.argmax(diff[:, sm]))
        near = any(min(abs(ref["tau"][p, st, sm] - ref["left"][p, st, sm]),
                       abs(ref["right"][p, st, sm] - ref["tau"][p, st, sm])) <= EDGE_TOL[prec] * ref["total"][p, st, sm]
                   for st in (0, 1))
        assert near, f"sample {sm}: factor {p} differs away from any CDF boundary"
    assert len(bad) <= 0.01 * J
    same = ~diff.any(axis=0)
    np.testing.assert_allclose(w.cpu().numpy()[same], ref["weight"][same], rtol=1e-4)
    print(f"prec {prec} {case}: {len(bad)} near-edge mismatches / {J}")
    s.close()


def test_bf16x3_bad_input_is_reported():
    """A NaN row reaches the leaf Grams through the tensor cores too; the
    sampler must report it on the device status, not hang or fault."""
    U = torch.randn(256, 16, device=DEV)
    U[17, 3] = float("nan")
    from paper_2301_12584_gb300.krpls import Sampler
    s = Sampler([256, 64], 16, 16, BF16X3)
    s.set_factor(0, U)
    s.set_factor(1, torch.randn(64, 16, device=DEV))
    idx = torch.zeros((2, 64), dtype=torch.int32, device=DEV)
    w = torch.zeros(64, device=DEV)
    s.sample(-1, 64, 1, 0, idx, w)
    assert s.sync_status() in (-6, -4)
    s.close()
