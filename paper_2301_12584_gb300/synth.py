"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random arrays (NumPy PCG64); it contains none of the
sampler's or solver's arithmetic, so both the CUDA path and the CPU oracle
can be fed identical inputs from it.

Workloads (all seeded; see the design notes for the recipes):
  * tiny exact case: N=3 factors of 64 x 8, N(0,1), seed 0, with a planted
    8 x 4 solution and 0.01 noise on a materialised B (Sec. 4.2 style);
  * sampler at scale: N=3 factors of 2^22 x 32, N(0,1), with 1% of rows
    scaled by 100 (skewed leverage), fresh N(0,1) rows for one factor per
    draw;
  * rank sweep: N=4 factors of 2^20 x R, U(-1,1);
  * sparse 3-mode tensor with Zipf(1.1) mode indices, duplicates dropped,
    values from a rank-16 U(0,1) model times lognormal(0, 0.5) noise
    (stand-in for the FROSTT tensors of Sec. 4.3);
  * skewed small factors (8 x 8, 1% of entries x10) as in App. A.13.2.
"""
from __future__ import annotations

import numpy as np


def gaussian_factors(N, I, R, seed, dtype=np.float32):
    """N factors I_k x R with i.i.d. N(0,1) entries. I may be an int or list."""
    rng = np.random.default_rng(seed)
    dims = [I] * N if np.isscalar(I) else list(I)
    return [rng.standard_normal((int(n), R), dtype=np.float64).astype(dtype) for n in dims]


def skewed_row_factors(N, I, R, seed, frac=0.01, scale=100.0, dtype=np.float32):
    """N(0,1) factors with floor(frac*I) rows per factor (chosen without
    replacement) multiplied by `scale`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(N):
        U = rng.standard_normal((I, R), dtype=np.float32)
        rows = rng.choice(I, size=int(frac * I), replace=False)
        U[rows] *= np.float32(scale)
        out.append(U.astype(dtype, copy=False))
    return out


def fresh_factor(I, R, seed, dtype=np.float32):
    """Fresh N(0,1) rows replacing one factor between draws."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((I, R), dtype=np.float32).astype(dtype, copy=False)


def uniform_factors(N, I, R, seed, dtype=np.float32):
    """N factors I x R with i.i.d. U(-1, 1) entries."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, size=(I, R)).astype(dtype) for _ in range(N)]


def skewed_entry_factors(N, I, R, seed, frac=0.01, scale=10.0, dtype=np.float32):
    """N(0,1) factors with a random `frac` of all entries multiplied by
    `scale` (App. A.13.2 / Sec. 4.2 recipe)."""
    rng = np.random.default_rng(seed)
    Is = list(I) if np.ndim(I) else [I] * N
    out = []
    for k in range(N):
        U = rng.standard_normal((Is[k], R))
        mask = rng.random((Is[k], R)) < frac
        U[mask] *= scale
        out.append(U.astype(dtype))
    return out


def correlated_sparse_factors(N, I, R, seed, zero_frac=0.8, common=3.0, dtype=np.float32):
    """Factors shaped like those of later sparse CP-ALS sweeps: a random
    `zero_frac` of each factor's rows are zero (indices that no sampled
    nonzero touched), the others N(0,1) plus `common` times one N(0,1) value
    shared by the row's entries (strongly correlated columns, so an
    ill-conditioned Gram), then every column scaled to unit norm.  I may be
    an int or a list."""
    rng = np.random.default_rng(seed)
    dims = [I] * N if np.isscalar(I) else list(I)
    out = []
    for n in dims:
        U = rng.standard_normal((int(n), R)) + common * rng.standard_normal((int(n), 1))
        U[rng.random(int(n)) < zero_frac] = 0.0
        U /= np.maximum(np.linalg.norm(U, axis=0), 1e-300)
        out.append(U.astype(dtype))
    return out


def planted_solution(R, nrhs, seed, dtype=np.float32):
    """X_true (R x nrhs), i.i.d. N(0,1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((R, nrhs)).astype(dtype)


def noise(shape, seed, scale, dtype=np.float32):
    """scale * N(0,1) array."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(shape)).astype(dtype)


def zipf_cdf(dim, s):
    """CDF of Zipf(s) truncated to ranks 1..dim."""
    ranks = np.arange(1, dim + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-s))
    return cdf / cdf[-1]


def zipf_indices(rng, n, dim, s, perm=None, cdf=None):
    """n draws from Zipf(s) truncated to [0, dim) by inverse CDF, then mapped
    through a seeded permutation so that hot indices are not contiguous (one
    permutation per mode: pass the same `perm` for every batch of a mode)."""
    if cdf is None:
        cdf = zipf_cdf(dim, s)
    if perm is None:
        perm = rng.permutation(dim)
    u = rng.random(n)
    r = np.searchsorted(cdf, u, side="left")
    r = np.minimum(r, dim - 1)
    return perm[r].astype(np.int32)


def sparse_zipf_tensor(dims, nnz, seed, s=1.1, model_rank=16, batch=None, device=None):
    """Synthetic sparse tensor: coordinates with Zipf(s) per mode, repeats
    dropped in draw order until `nnz` unique coordinates; values are a
    rank-`model_rank` CP model with U(0,1) factors evaluated at each
    coordinate, times lognormal(0, 0.5) noise.

    All random draws come from NumPy's PCG64(seed).  With `device` (a torch
    device) the inverse-CDF lookups, the removal of repeats and the model
    values run there instead (same draws and coordinates; values equal up to
    the order of FP64 summation) — for tensors of 10^8 nonzeros.

    Returns (coords int32 [N, nnz], vals float32 [nnz]).
    """
    rng = np.random.default_rng(seed)
    N = len(dims)
    bits = [int(np.ceil(np.log2(max(d, 2)))) for d in dims]
    assert sum(bits) <= 63
    batch = batch or max(1024, nnz // 2)
    perms = [rng.permutation(d) for d in dims]
    cdfs = [zipf_cdf(d, s) for d in dims]
    if device is not None:
        import torch
        tcdf = [torch.from_numpy(c).to(device) for c in cdfs]
        tperm = [torch.from_numpy(p).to(device) for p in perms]
        seen = torch.zeros(0, dtype=torch.int64, device=device)
        acc = [torch.zeros(0, dtype=torch.int32, device=device) for _ in range(N)]
        while seen.numel() < nnz:
            cs = []
            for k, d in enumerate(dims):
                u = torch.from_numpy(rng.random(batch)).to(device)
                r = torch.clamp(torch.searchsorted(tcdf[k], u, right=False), max=d - 1)
                cs.append(tperm[k][r].to(torch.int32))
            key = torch.zeros(batch, dtype=torch.int64, device=device)
            for k in range(N):
                key = (key << bits[k]) | cs[k].to(torch.int64)
            uniq, inv = torch.unique(key, sorted=True, return_inverse=True)
            first = torch.full((uniq.numel(),), batch, dtype=torch.int64, device=device)
            first.scatter_reduce_(0, inv, torch.arange(batch, device=device), reduce="amin")
            first = torch.sort(first).values
            key = key[first]
            cs = [c[first] for c in cs]
            fresh = ~torch.isin(key, seen)
            key = key[fresh]
            cs = [c[fresh] for c in cs]
            take = min(key.numel(), nnz - seen.numel())
            seen = torch.cat([seen, key[:take]])
            acc = [torch.cat([a, c[:take]]) for a, c in zip(acc, cs)]
        del seen
        coords_t = torch.stack(acc)
        V = [torch.from_numpy(rng.random((d, model_rank))).to(device) for d in dims]
        noise = rng.lognormal(0.0, 0.5, size=nnz)
        vals = np.empty(nnz, dtype=np.float32)
        step = 1 << 24
        for a in range(0, nnz, step):
            b = min(nnz, a + step)
            P = torch.ones((b - a, model_rank), dtype=torch.float64, device=device)
            for k in range(N):
                P *= V[k][coords_t[k, a:b].long()]
            vals[a:b] = (P.sum(dim=1).cpu().numpy() * noise[a:b]).astype(np.float32)
        return coords_t.cpu().numpy(), vals
    keys_seen = np.zeros(0, dtype=np.int64)
    coords_acc = [np.zeros(0, np.int32) for _ in range(N)]
    while keys_seen.size < nnz:
        cs = [zipf_indices(rng, batch, d, s, perm=pm, cdf=cf) for d, pm, cf in zip(dims, perms, cdfs)]
        key = np.zeros(batch, dtype=np.int64)
        for k in range(N):
            key = (key << bits[k]) | cs[k].astype(np.int64)
        # keep the first occurrence of each key, in draw order
        _, first = np.unique(key, return_index=True)
        first.sort()
        key = key[first]
        cs = [c[first] for c in cs]
        fresh = ~np.isin(key, keys_seen)
        key = key[fresh]
        cs = [c[fresh] for c in cs]
        take = min(key.size, nnz - keys_seen.size)
        keys_seen = np.concatenate([keys_seen, key[:take]])
        coords_acc = [np.concatenate([a, c[:take]]) for a, c in zip(coords_acc, cs)]
    coords = np.stack(coords_acc).astype(np.int32)
    V = [rng.random((d, model_rank)) for d in dims]
    noise = rng.lognormal(0.0, 0.5, size=nnz)
    vals = np.empty(nnz, dtype=np.float32)
    step = 1 << 22
    for a in range(0, nnz, step):  # the CP model in chunks (nnz x model_rank would not fit at scale)
        b = min(nnz, a + step)
        P = np.ones((b - a, model_rank))
        for k in range(N):
            P *= V[k][coords[k, a:b]]
        vals[a:b] = (P.sum(axis=1) * noise[a:b]).astype(np.float32)
    return coords, vals


def planted_dense_tensor(dims, rank, seed):
    """Small exactly-low-rank tensor (no noise), returned as a full-coordinate
    sparse tensor: CP model with N(0,1) factors."""
    rng = np.random.default_rng(seed)
    Vs = [rng.standard_normal((d, rank)) for d in dims]
    grids = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    coords = np.stack([g.reshape(-1) for g in grids]).astype(np.int32)
    P = np.ones((coords.shape[1], rank))
    for k in range(len(dims)):
        P *= Vs[k][coords[k]]
    return coords, P.sum(axis=1).astype(np.float32)
