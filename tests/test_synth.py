"""Seeded input generators: the torch path of the sparse tensor generator
(used for 10^8-nonzero tensors) reproduces the NumPy path exactly."""
import numpy as np
import torch

from paper_2301_12584_gb300 import synth


def test_sparse_generator_torch_path_matches_numpy():
    dims = (1 << 12, 1 << 10, 300)
    a = synth.sparse_zipf_tensor(dims, 50_000, seed=3)
    b = synth.sparse_zipf_tensor(dims, 50_000, seed=3, device=torch.device("cpu"))
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-6)
    keys = (a[0][0].astype(np.int64) << 22) | (a[0][1].astype(np.int64) << 10) | a[0][2]
    assert np.unique(keys).size == keys.size          # coordinates are unique
    assert (a[0] >= 0).all() and all((a[0][k] < d).all() for k, d in enumerate(dims))
