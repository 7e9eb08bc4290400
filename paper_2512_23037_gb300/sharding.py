"""Shot-range sharding across ranks (no data-path collective).

Shots are independent and every random draw is keyed on (seed, shot index)
(Sec. IV-B: shots share no state), so a job of N shots starting at shot
`first` splits into contiguous ranges: rank r of G runs
[first + floor(r N / G), first + floor((r + 1) N / G)). A G-rank run of N
shots therefore gives exactly the 1-rank run of the same N shots. The only
cross-rank step is one sum of the tally (five u64 counters and two FP64
sums).
"""
from __future__ import annotations

TALLY_COUNTS = ("shots", "discarded", "overflow", "kept", "logical_errors")
TALLY_SUMS = ("sum_fidelity", "sum_weight")


def shot_range(rank: int, world: int, n_total: int, first: int = 0):
    """(first shot, shot count) of rank `rank` in a job of n_total shots."""
    if not (0 <= rank < world) or n_total < 0 or first < 0:
        raise ValueError("bad shard")
    lo = (rank * n_total) // world
    hi = ((rank + 1) * n_total) // world
    return first + lo, hi - lo


def reduce_tallies(tallies):
    """Sum of tallies given as dicts (soft_tally's keys) or as
    [shots, discarded, overflow, kept, logical_errors] lists; returns the
    same kind as the first."""
    tallies = list(tallies)
    if tallies and isinstance(tallies[0], dict):
        out = {k: 0 for k in TALLY_COUNTS}
        out.update({k: 0.0 for k in TALLY_SUMS})
        for t in tallies:
            for k in TALLY_COUNTS:
                out[k] += int(t[k])
            for k in TALLY_SUMS:
                out[k] += float(t.get(k, 0.0))
        return out
    out = [0, 0, 0, 0, 0]
    for t in tallies:
        for i in range(5):
            out[i] += int(t[i])
    return out


def all_reduce_tally(tally: dict, dist, device=None) -> dict:
    """The job's tally: this rank's tally (a soft_tally dict) summed over the
    ranks of the default process group with one all-reduce of the counters
    (int64) and one of the FP64 sums."""
    import torch
    cnt = torch.tensor([int(tally[k]) for k in TALLY_COUNTS], dtype=torch.int64, device=device)
    sums = torch.tensor([float(tally.get(k, 0.0)) for k in TALLY_SUMS], dtype=torch.float64, device=device)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    out = {k: int(v) for k, v in zip(TALLY_COUNTS, cnt.tolist())}
    out.update({k: float(v) for k, v in zip(TALLY_SUMS, sums.tolist())})
    return out
