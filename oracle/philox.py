"""Philox4x32-10 counter-based generator, written out from its published definition.

Test infrastructure only: this module belongs to the CPU oracle.  Nothing on
the product path imports it.

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 3.3): a 4x32-bit counter block is transformed by 10
rounds.  Each round multiplies words 0 and 2 by two fixed odd constants,
splits each 64-bit product into high and low halves, and permutes/xors them
with the other two words and the round key.  The 2x32-bit key is bumped by
two Weyl constants between rounds.

The sampler draws every uniform from one Philox block, so the oracle and
the device path start from identical bits (the reading of "Uniform(0,1)" in
Alg. 4 that this library adopts):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (sample index d, draw_id & 0xffffffff, position p of the factor
             among the included factors, 0)
  word 0 -> uniform for the eigencomponent stage, word 1 -> uniform for the
  row stage, each mapped to (2*(x >> 9) + 1) * 2^-24, an open-interval value
  that is exact in both FP32 and FP64.
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Apply Philox4x32 with 10 rounds.

    ctr: uint32 array of shape (..., 4); key: uint32 array of shape (..., 2)
    (broadcastable).  Returns uint32 array of shape (..., 4).
    """
    ctr = np.asarray(ctr, dtype=np.uint32)
    key = np.asarray(key, dtype=np.uint32)
    c0, c1, c2, c3 = (ctr[..., i].astype(np.uint64) for i in range(4))
    k0 = key[..., 0].astype(np.uint64)
    k1 = key[..., 1].astype(np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK32
        p0 = PHILOX_M0 * c0          # < 2^64, exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        n0 = hi1 ^ c1 ^ k0
        n1 = lo1
        n2 = hi0 ^ c3 ^ k1
        n3 = lo0
        c0, c1, c2, c3 = n0, n1, n2, n3
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def u32_to_open_unit(x):
    """Map a uint32 word to the open interval (0, 1): (2*(x>>9)+1) * 2^-24."""
    x = np.asarray(x, dtype=np.uint32)
    return ((2.0 * (x >> np.uint32(9)).astype(np.float64)) + 1.0) * 2.0 ** -24


def sampler_uniforms(seed, draw_id, J, n_incl, d0=0):
    """Uniforms for samples d0..d0+J-1 and included positions 0..n_incl-1.

    Returns (u_eig, u_row), each float64 of shape (J, n_incl).
    """
    seed = int(seed)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    d = (np.arange(J, dtype=np.uint64) + np.uint64(d0)).astype(np.uint32)
    ctr = np.zeros((J, n_incl, 4), dtype=np.uint32)
    ctr[..., 0] = d[:, None]
    ctr[..., 1] = np.uint32(int(draw_id) & 0xFFFFFFFF)
    ctr[..., 2] = np.arange(n_incl, dtype=np.uint32)[None, :]
    out = philox4x32_10(ctr, key)
    return u32_to_open_unit(out[..., 0]), u32_to_open_unit(out[..., 1])
