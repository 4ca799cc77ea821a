"""One sampler replica per GPU: weak scaling with no data-path collective.

Samples are i.i.d. given the segment trees (Sec. 4, batch-parallel sampling),
so every rank holds its own copy of the factors and trees and draws with draw
ids of its own.  Ranks never exchange data; the only collectives are the timing
barrier and the maximum over ranks of the elapsed time, which makes the
whole-job rate (samples of all ranks) / (slowest rank's time).
"""
from __future__ import annotations

import os

# Draw ids of rank r are r * DRAW_STRIDE + d for d < DRAW_STRIDE; with Philox
# counters keyed by the draw id, the ranks' uniforms never overlap.
DRAW_STRIDE = 1_000_000


def rank_env():
    """(rank, local_rank, world_size) from the torchrun environment; (0, 0, 1) alone."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def draw_base(rank: int) -> int:
    return rank * DRAW_STRIDE


def draw_ids(rank: int, first: int, count: int) -> range:
    """The draw ids rank `rank` uses for its draws first .. first + count - 1."""
    if first < 0 or first + count > DRAW_STRIDE:
        raise ValueError(f"draws {first}..{first + count} leave the rank's id range of {DRAW_STRIDE}")
    return range(draw_base(rank) + first, draw_base(rank) + first + count)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks (the value itself without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms_max: float) -> float:
    """Units processed by all ranks per second, timed by the slowest rank."""
    if ms_max <= 0:
        raise ValueError("elapsed time must be positive")
    return units_per_rank * world / (ms_max / 1e3)
