"""Autotuner for the shot kernel's launch shape.

Times short runs of the real workload (a sample of shots far from the shots a
caller will run, so nothing is reused) for every candidate of

  - first_cap: capacity of the first pass's on-chip map (shots above it and
    below their circuit's cap rerun at the full cap),
  - groups_per_block: shots resident per 128-thread block (2 or 4 for 32-lane
    groups, 8 for 16-lane groups),
  - group_size: lanes per shot (32 = one warp per shot, 16 = two shots per warp;
    0 = the library default: one shot per lane where that applies, with
    first_cap the capacity of the warp pass that takes shots outgrowing a lane),

and keeps the fastest. Results are cached per circuit signature.
"""
from __future__ import annotations

import itertools

from . import soft_compile_circuit  # noqa: F401  (re-exported for callers)
from . import soft_run_batch, soft_run_timing, soft_tally

_CACHE: dict = {}

DEFAULT_SPACE = {"first_cap": [16, 32, 64], "groups_per_block": [2, 4, 8], "group_size": [0, 32, 16]}


def signature(circs, precision):
    return (precision,) + tuple((c.n, c.info["coeff_cap"], c.info["n_events"], c.info["n_sites"]) for c in circs)


def autotune(circs, precision="fp32", sample_shots=1 << 18, space=None, seed=0x5eed, stream=None, repeats=2):
    """Return the fastest launch options (kwargs for soft_run_shots /
    soft_run_batch) for this list of compiled circuits, and the timings."""
    key = signature(circs, precision)
    if key in _CACHE:
        return _CACHE[key]
    space = space or DEFAULT_SPACE
    n = len(circs)
    per = max(1, sample_shots // n)
    names = list(space)
    results, seen = [], set()
    for values in itertools.product(*[space[k] for k in names]):
        kw = dict(zip(names, values))
        gs, gpb = kw.get("group_size", 32), kw.get("groups_per_block", 0)
        if gs == 0:  # the library default shape: groups per block do not apply
            kw["groups_per_block"] = 0
            if tuple(sorted(kw.items())) in seen:
                continue
            seen.add(tuple(sorted(kw.items())))
        elif gpb and gpb > 128 // gs:
            continue  # more groups than a 128-thread block holds
        if gs == 16 and gpb and gpb != 8:
            continue  # 16-lane groups run full blocks
        best = None
        for rep in range(repeats + 1):
            first = [(1 << 50) + rep * per] * n
            r = soft_run_batch(circs, [per] * n, first, seed, precision=precision, stream=stream, **kw)
            soft_tally(r)
            ms, _ = soft_run_timing(r)
            r.free()
            if rep > 0:  # the first run warms up
                best = ms if best is None else min(best, ms)
        results.append((best, kw))
    results.sort(key=lambda t: t[0])
    out = {"best": results[0][1], "ms": results[0][0], "table": results}
    _CACHE[key] = out
    return out
