"""Least-squares accuracy workload (Sec. 4.2) on the GPU against the FP64
oracle: the sketch distortion computed without forming A (appendix route)
against its definition through a basis of range(A), the Kronecker
right-hand side's entries, and the sketched solution's residual ratio.

Tolerances: D within 1e-5 (1 + D) relative (SAᵀSA from FP32 sums of FP32
rows); Kronecker entries 1e-6 relative (FP32 products of N terms).
"""
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


@pytest.mark.parametrize("dims,R,J,excl", [((6, 7, 8), 4, 500, -1), ((30, 40, 20), 16, 3000, -1),
                                           ((25, 20, 30), 8, 2000, 1)])
def test_distortion_and_kron_rows_match_oracle(dims, R, J, excl):
    from paper_2301_12584_gb300.krpls import Sampler
    Us = synth.skewed_entry_factors(3, list(dims), R, seed=sum(dims) + R)
    s = Sampler(list(dims), R, 0)
    for k, U in enumerate(Us):
        s.set_factor(k, torch.from_numpy(U).to(DEV))
    idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, device=DEV)
    SA = torch.zeros((J, R), device=DEV)
    s.sample(excl, J, 9, 0, idx, w, None, SA)
    D, rank = s.sketch_distortion(excl, J, SA)
    assert s.sync_status() == 0
    incl = [k for k in range(3) if k != excl]
    gi = idx.cpu().numpy().astype(np.int64)[incl]
    U64 = [U.astype(np.float64) for U in Us]
    Dref = O.sketch_distortion(U64, excl, gi, w.cpu().numpy().astype(np.float64))
    assert rank == R
    assert abs(D - Dref) <= 1e-5 * (1.0 + Dref), (D, Dref)
    rng = np.random.default_rng(3)
    cs = [rng.standard_normal(n).astype(np.float32) for n in dims]
    cd = [torch.from_numpy(c).to(DEV) for c in cs]
    B = torch.zeros(J, device=DEV)
    s.kron_rows(excl, J, idx, cd, B)
    assert s.sync_status() == 0
    ref = O.kron_rows([c.astype(np.float64) for c in cs], excl, gi)
    np.testing.assert_allclose(B.cpu().numpy(), ref, rtol=1e-6, atol=1e-30)
    # the sketched solution's residual is close to optimal (Thm 2.1; Sec. 4.2 reports eps ~ 1e-2)
    X = torch.zeros((R, 1), device=DEV)
    s.solve_dense(J, SA, w, B.view(J, 1), 1, X)
    assert s.sync_status() == 0
    res, G, Atb = O.kron_lstsq_residual(U64, excl, [c.astype(np.float64) for c in cs], X.cpu().numpy()[:, 0])
    x_opt = np.linalg.solve(G, Atb)
    res_opt, _, _ = O.kron_lstsq_residual(U64, excl, [c.astype(np.float64) for c in cs], x_opt)
    eps = res / res_opt - 1.0
    assert -1e-9 <= eps < 0.5, eps
    s.close()


def test_distortion_requires_a_preparation():
    from paper_2301_12584_gb300.krpls import KrpError, Sampler
    s = Sampler([10, 12], 4, 0)
    for k in range(2):
        s.set_factor(k, torch.randn(s.I[k], 4, device=DEV))
    SA = torch.zeros((8, 4), device=DEV)
    with pytest.raises(KrpError) as e:
        s.sketch_distortion(-1, 8, SA)
    assert e.value.code == -8
    s.close()
