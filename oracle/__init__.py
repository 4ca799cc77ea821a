"""CPU oracle for the KRP leverage-score sampler and sketched solve.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py, never by the library.  It shares no code
with the CUDA path; the two meet only through seeded input arrays.

Modules:
  philox      Philox4x32-10 (Salmon et al., SC'11) and the uniform mapping.
  krp_oracle  FP64 leverage scores, Alg. 2 replay, Alg. 3/4 segment tree,
              sketched least squares, sparse STS-CP (Alg. 6) and the fit.

Every function is pinned by tests/test_oracle_pins.py; none is "parity
unpinned".
"""
from . import philox, krp_oracle  # noqa: F401
