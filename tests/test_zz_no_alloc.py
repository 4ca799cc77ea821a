"""krp_solve_dense_noalloc (the dense sketched solve with fixed device scratch)
against krp_solve_dense and against the FP64 oracle's lstsq of the same
weighted sketch: two calls in a row, different shapes (including one whose
partial sums fill the most CTAs the solve uses, 2 per SM), then the status
word's reset after a singular system.

Tolerance: 1e-4 relative Frobenius, the dense solve's bar.  Collected last so
that it also runs after every other GPU test in one process.
"""
import numpy as np
import pytest
import torch

from oracle import krp_oracle as O
from paper_2301_12584_gb300 import synth

DEV = "cuda:0"


@pytest.fixture(scope="module")
def krpls():
    import os
    from paper_2301_12584_gb300 import build as B
    from paper_2301_12584_gb300 import krpls as K
    if not os.path.exists(K.LIB_PATH):
        B.build()
    K.lib()
    return K


def sketch(K, Us, J, seed, nrhs):
    """A sampled sketch (SA, weight) of the full KRP and random rows B, on the device."""
    s = K.Sampler([U.shape[0] for U in Us], Us[0].shape[1], 0, 0)
    for k, U in enumerate(Us):
        s.set_factor(k, torch.from_numpy(U).to(DEV))
    N, R = len(Us), Us[0].shape[1]
    idx = torch.zeros((N, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, device=DEV)
    SA = torch.zeros((J, R), device=DEV)
    s.sample(-1, J, seed, 0, idx, w, SA=SA)
    g = torch.Generator(device="cpu").manual_seed(seed)
    B = torch.randn((J, nrhs), generator=g).to(DEV)
    return s, SA, w, B


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.gpu
def test_noalloc_matches_solve_dense_twice(krpls):
    # (R, nrhs, J, seed): the limits; the limits with J >= 256 x 2 x SMs (every
    # partial the solve can use, exponents at the end of the used scratch);
    # a small ragged case
    cases = [(32, 16, 30001, 3), (32, 16, 1 << 18, 5), (13, 3, 777, 4)]
    for R, nrhs, J, seed in cases:
        Us = synth.gaussian_factors(3, 40, R, seed=seed)
        s, SA, w, B = sketch(krpls, Us, J, seed, nrhs)
        X_ref = torch.zeros((R, nrhs), device=DEV)
        s.solve_dense(J, SA, w, B, nrhs, X_ref)
        assert s.sync_status() == 0
        X_o = O.lstsq(SA.double().cpu().numpy(), (w[:, None] * B).double().cpu().numpy())
        status = torch.full((1,), 12345, dtype=torch.int32, device=DEV)
        for _ in range(2):
            X = torch.full((R, nrhs), float("nan"), device=DEV)
            krpls.solve_dense_noalloc(J, R, SA, w, B, nrhs, X, status)
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert torch.isfinite(X).all()
            assert rel(X, X_ref) <= 1e-4
            Xn = X.double().cpu().numpy()
            assert np.linalg.norm(Xn - X_o) <= 1e-4 * np.linalg.norm(X_o)
        s.close()


@pytest.mark.gpu
def test_noalloc_singular_then_clean(krpls):
    R, nrhs, J = 6, 2, 4000
    Us = synth.gaussian_factors(3, 30, R, seed=31)
    for U in Us:
        U[:, 5] = U[:, 0]                       # rank-deficient KRP: M singular
    s, SA, w, B = sketch(krpls, Us, J, 1, nrhs)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    X = torch.ones((R, nrhs), device=DEV)
    krpls.solve_dense_noalloc(J, R, SA, w, B, nrhs, X, status, flags=0)
    torch.cuda.synchronize()
    assert int(status.item()) == -5             # KRP_ESINGULAR
    assert np.all(X.cpu().numpy() == 0)
    X_ref = torch.zeros((R, nrhs), device=DEV)
    s.solve_dense(J, SA, w, B, nrhs, X_ref, flags=1)
    assert s.sync_status() == 0
    krpls.solve_dense_noalloc(J, R, SA, w, B, nrhs, X, status, flags=1)   # pseudo-inverse fallback
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert rel(SA @ X, SA @ X_ref) <= 1e-4
    s.close()


def test_noalloc_rejects_oversize_on_host(krpls):
    fake = 256                                   # never dereferenced: the call is rejected first
    for R, nrhs in ((33, 1), (32, 17), (0, 1), (4, 0)):
        with pytest.raises(krpls.KrpError) as e:
            krpls.solve_dense_noalloc(100, R, fake, fake, fake, nrhs, fake, fake, stream=0)
        assert e.value.code == -1                # KRP_EINVAL
        assert "R must be in [1, 32]" in str(e.value)
    with pytest.raises(krpls.KrpError) as e:
        krpls.solve_dense_noalloc(100, 4, fake, fake, fake, 1, fake, None, stream=0)
    assert e.value.code == -1
