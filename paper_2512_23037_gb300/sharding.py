"""Shot-range sharding across ranks (weak scaling, no data-path collective).

Shots are independent and every random draw is keyed on (seed, shot index),
so rank r of `world` simply owns shots [r * stride, r * stride + n_per_rank);
the only cross-rank step is one sum of the five tally counters.
"""
from __future__ import annotations

RANK_STRIDE = 1 << 40  # shot-index stride between ranks


def shot_range(rank: int, world: int, n_per_rank: int, stride: int = RANK_STRIDE):
    if not (0 <= rank < world) or n_per_rank < 0 or n_per_rank > stride:
        raise ValueError("bad shard")
    return rank * stride, n_per_rank


def reduce_tallies(tallies):
    """Element-wise sum of [shots, discarded, overflow, kept, logical] lists."""
    out = [0, 0, 0, 0, 0]
    for t in tallies:
        for i in range(5):
            out[i] += int(t[i])
    return out
