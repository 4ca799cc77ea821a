"""Batched problems (one launch per phase over many samplers, CUDA-graph
replay) and the planted right-hand side, against the FP64 oracle and against
the single-problem path.

Per problem the batch draws the same uniforms as krp_sample(seed, draw_id), so
the index parity bar of the single path applies (every mismatch within 1e-5 C
of an edge of the oracle's bin, fewer than 1e-4 J of them); the solve must be
within 1e-4 relative Frobenius of FP64 lstsq on the batch's own sketch.
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


def make_problems(P, seed, I_range=(256, 1500), Rs=(8, 16, 32)):
    rng = np.random.default_rng(seed)
    probs = []
    for p in range(P):
        R = int(Rs[p % len(Rs)])
        I = [int(np.exp(rng.uniform(np.log(I_range[0]), np.log(I_range[1])))) for _ in range(3)]
        Us = synth.gaussian_factors(3, I, R, seed=1000 + p)
        probs.append((I, R, Us))
    return probs


def samplers_for(probs):
    from paper_2301_12584_gb300.krpls import Sampler
    out = []
    for I, R, Us in probs:
        s = Sampler(I, R, R)
        for k, U in enumerate(Us):
            s.set_factor(k, torch.from_numpy(U).to(DEV))
        out.append(s)
    torch.cuda.synchronize()
    return out


def near_edge(ref, p, sm, tol):
    return any(min(abs(ref["tau"][p, st, sm] - ref["left"][p, st, sm]),
                   abs(ref["right"][p, st, sm] - ref["tau"][p, st, sm])) <= tol * ref["total"][p, st, sm]
               for st in (0, 1))


def run_batch(batch, J, nrhs, seed, X_true):
    P, N, off = batch.P, batch.N, batch.row_off
    idx = torch.zeros((P, N, J), dtype=torch.int32, device=DEV)
    w = torch.zeros((P, J), device=DEV)
    SA = torch.zeros(J * off[-1], device=DEV)
    B = torch.zeros((P, J, nrhs), device=DEV)
    X = torch.zeros(off[-1] * nrhs, device=DEV)
    batch.build()
    batch.sample(J, seed, 2, idx, w, SA)
    batch.planted_rows(J, idx, X_true, nrhs, 1e-3, seed + 1, B)
    batch.solve_dense(J, SA, w, B, nrhs, X)
    return idx, w, SA, B, X


def test_planted_rows_single_matches_oracle():
    from paper_2301_12584_gb300.krpls import Sampler
    Us = synth.gaussian_factors(3, [50, 37, 64], 8, seed=5)
    s = Sampler([50, 37, 64], 8, 8)
    for k, U in enumerate(Us):
        s.set_factor(k, torch.from_numpy(U).to(DEV))
    J, nrhs = 4096, 4
    idx = torch.zeros((3, J), dtype=torch.int32, device=DEV)
    w = torch.zeros(J, device=DEV)
    s.sample(1, J, 3, 0, idx, w)
    X = synth.planted_solution(8, nrhs, seed=2)
    B = torch.zeros((J, nrhs), device=DEV)
    s.planted_rows(1, J, idx, torch.from_numpy(X).to(DEV), nrhs, 0.5, 99, B)
    assert s.sync_status() == 0
    U64 = [U.astype(np.float64) for U in Us]
    gi = idx.cpu().numpy().astype(np.int64)[[0, 2]]
    ref = O.planted_rhs(U64, 1, gi, X.astype(np.float64), 0.5, 99)
    np.testing.assert_allclose(B.cpu().numpy(), ref, rtol=1e-5, atol=2e-5 * np.abs(ref).max())
    s.close()


def test_batch_matches_oracle_per_problem():
    P, J, nrhs = 6, 2048, 4
    probs = make_problems(P, seed=1)
    sams = samplers_for(probs)
    from paper_2301_12584_gb300.krpls import Batch
    stream = torch.cuda.Stream()
    batch = Batch(sams, stream)
    X_true = np.concatenate([synth.planted_solution(R, nrhs, seed=50 + p).ravel()
                             for p, (_, R, _) in enumerate(probs)]).astype(np.float32)
    fresh = [synth.gaussian_factors(3, I, R, seed=2000 + p) for p, (I, R, _) in enumerate(probs)]
    src = [torch.from_numpy(U).to(DEV) for Us in fresh for U in Us]
    batch.set_sources(src)
    with torch.cuda.stream(stream):
        idx, w, SA, B, X = run_batch(batch, J, nrhs, 7, torch.from_numpy(X_true).to(DEV))
    stream.synchronize()
    assert batch.sync_status() == 0
    idx, w, SA, B, X = (t.cpu().numpy() for t in (idx, w, SA, B, X))
    off = batch.row_off
    total_mism = 0
    for p, (I, R, _) in enumerate(probs):
        U64 = [U.astype(np.float64) for U in fresh[p]]
        # trees rebuilt from the new sources (and the samplers' copies updated)
        root = sams[p].get_tree(0)[0]
        G = U64[0].T @ U64[0]
        iu = np.triu_indices(R)
        bound = (np.abs(U64[0]).T @ np.abs(U64[0]))[iu]
        assert np.all(np.abs(root[:len(iu[0])] - G[iu]) <= 2e-5 * bound)
        ref = O.krp_sample(U64, -1, J, 7, 2, record=True)
        gi = idx[p].astype(np.int64)
        diff = gi != ref["idx"]
        bad = np.nonzero(diff.any(axis=0))[0]
        for sm in bad:
            assert near_edge(ref, int(np.argmax(diff[:, sm])), sm, 1e-5), (p, sm)
        total_mism += len(bad)
        same = ~diff.any(axis=0)
        np.testing.assert_allclose(w[p][same], ref["weight"][same], rtol=1e-4)
        SAp = SA[J * off[p]: J * off[p + 1]].reshape(J, R)
        rows = O.sketched_rows(U64, -1, gi, w[p].astype(np.float64))
        np.testing.assert_allclose(SAp, rows, rtol=2e-6, atol=1e-30)
        Xt = X_true[off[p] * nrhs: off[p + 1] * nrhs].reshape(R, nrhs).astype(np.float64)
        Bref = O.planted_rhs(U64, -1, gi, Xt, 1e-3, 8)
        np.testing.assert_allclose(B[p], Bref, rtol=1e-5, atol=1e-5 * np.abs(Bref).max())
        Xp = X[off[p] * nrhs: off[p + 1] * nrhs].reshape(R, nrhs)
        Xo = O.lstsq(SAp.astype(np.float64), w[p][:, None].astype(np.float64) * B[p].astype(np.float64))
        assert np.linalg.norm(Xp - Xo) <= 1e-4 * np.linalg.norm(Xo)
        assert np.linalg.norm(Xp - Xt) <= 0.05 * np.linalg.norm(Xt)   # the planted solution is recovered
    assert total_mism < max(1.0, 1e-4 * P * J)
    batch.close()
    for s in sams:
        s.close()


def test_batch_graph_replay_and_tuning_reproduce_direct_run():
    P, J, nrhs = 9, 1024, 4
    probs = make_problems(P, seed=2)
    sams = samplers_for(probs)
    from paper_2301_12584_gb300.krpls import Batch
    stream = torch.cuda.Stream()
    batch = Batch(sams, stream)
    X_true = torch.from_numpy(np.concatenate([synth.planted_solution(R, nrhs, seed=p).ravel()
                                              for p, (_, R, _) in enumerate(probs)]).astype(np.float32)).to(DEV)
    with torch.cuda.stream(stream):
        direct = [t.clone() for t in run_batch(batch, J, nrhs, 3, X_true)]
        bufs = run_batch(batch, J, nrhs, 3, X_true)            # warm-up of the same buffers
        stream.synchronize()
        for t in bufs:
            t.zero_()
        stream.synchronize()
        batch.capture_begin()
        P_, N_, off = batch.P, batch.N, batch.row_off
        idx, w, SA, B, X = bufs
        batch.build()
        batch.sample(J, 3, 2, idx, w, SA)
        batch.planted_rows(J, idx, X_true, nrhs, 1e-3, 4, B)
        batch.solve_dense(J, SA, w, B, nrhs, X)
        nodes = batch.capture_end()
        assert nodes >= 6
        assert float(X.abs().sum()) == 0.0                     # captured, not run
        batch.replay()
    stream.synchronize()
    assert batch.sync_status() == 0
    for a, b in zip(direct, bufs):
        assert torch.equal(a, b)
    best = batch.autotune(J)
    assert best in (1, 2, 4, 8, 16)
    with torch.cuda.stream(stream):
        tuned = run_batch(batch, J, nrhs, 3, X_true)
    stream.synchronize()
    for a, b in zip(direct, tuned):
        assert torch.equal(a, b)                               # CTAs per problem change no result
    batch.close()
    for s in sams:
        s.close()


def test_batch_rejects_unsupported_samplers():
    from paper_2301_12584_gb300.krpls import Batch, KrpError, Sampler
    s = Sampler([300, 300], 64, 64)
    for k in range(2):
        s.set_factor(k, torch.randn(300, 64, device=DEV))
    with pytest.raises(KrpError) as e:
        Batch([s], torch.cuda.Stream())
    assert e.value.code == -1
    t = Sampler([300, 300], 8, 8)
    t.set_factor(0, torch.randn(300, 8, device=DEV))
    with pytest.raises(KrpError) as e:
        Batch([t], torch.cuda.Stream())                        # factor 1 unset
    assert e.value.code == -8
    s.close()
    t.close()


def test_throughput_probes_are_plausible():
    """The measurement build's krp_probe_peaks (libkrpprobe.so): the SIMT FP32,
    FP64 and L2 rooflines' denominators (positive, finite, FP64 well below FP32,
    L2 above the HBM copy rate)."""
    from paper_2301_12584_gb300.profile_cases import probe_peaks
    p = probe_peaks()
    assert all(np.isfinite(v) and v > 0 for v in p.values()), p
    assert p["fp64_tflops"] < p["fp32_tflops"], p
    assert p["l2_read_gbs"] > 1000.0, p
