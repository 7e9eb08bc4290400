"""Host logic of the autotuner, on the CPU: which candidate shapes it times (the
library default once per first-pass capacity, no group count larger than a
128-thread block holds, full blocks for 16-lane groups), that it keeps the
fastest by the best repeat after the warm-up run, and that it caches per
circuit signature. The runs are stand-ins that report scripted timings."""
import pytest

import paper_2512_23037_gb300.autotune as at


class _Circ:
    def __init__(self, n, cap, n_events, n_sites):
        self.n = n
        self.info = {"coeff_cap": cap, "n_events": n_events, "n_sites": n_sites}


class _Run:
    def __init__(self, ms):
        self.ms = ms

    def free(self):
        pass


@pytest.fixture
def fake_runs(monkeypatch):
    calls = []

    def run_batch(circs, shots, firsts, seed, precision=None, stream=None, **kw):
        calls.append(dict(kw))
        gs, fc, gpb = kw["group_size"], kw["first_cap"], kw["groups_per_block"]
        # scripted: the library default is fastest at first_cap 64; the first call of each
        # shape (the warm-up) is slow and must not count
        ms = (5.0 if gs == 0 else 9.0 + gpb) + (0.0 if fc == 64 else 1.0)
        if sum(1 for c in calls if c == kw) == 1:
            ms += 100.0
        return _Run(ms)

    monkeypatch.setattr(at, "soft_run_batch", run_batch)
    monkeypatch.setattr(at, "soft_tally", lambda r: {})
    monkeypatch.setattr(at, "soft_run_timing", lambda r: (r.ms, 1))
    at._CACHE.clear()
    yield calls
    at._CACHE.clear()


def test_candidates_and_choice(fake_runs):
    circs = [_Circ(42, 256, 365, 3401), _Circ(30, 64, 120, 900)]
    res = at.autotune(circs, precision="fp32", sample_shots=1 << 10, repeats=2)
    shapes = [kw for _, kw in res["table"]]
    # the library default (group_size 0) once per first_cap, with groups_per_block 0
    default = [kw for kw in shapes if kw["group_size"] == 0]
    assert sorted(kw["first_cap"] for kw in default) == sorted(at.DEFAULT_SPACE["first_cap"])
    assert all(kw["groups_per_block"] == 0 for kw in default)
    # 32-lane groups: at most 4 per block; 16-lane groups: full blocks of 8
    assert all(kw["groups_per_block"] <= 4 for kw in shapes if kw["group_size"] == 32)
    assert all(kw["groups_per_block"] == 8 for kw in shapes if kw["group_size"] == 16)
    assert len({tuple(sorted(kw.items())) for kw in shapes}) == len(shapes)
    # each shape ran 1 warm-up + 2 timed repeats; the choice ignores the warm-up
    assert len(fake_runs) == 3 * len(shapes)
    assert res["best"] == {"first_cap": 64, "groups_per_block": 0, "group_size": 0}
    assert res["ms"] == pytest.approx(5.0)
    assert [ms for ms, _ in res["table"]] == sorted(ms for ms, _ in res["table"])


def test_cache_per_signature(fake_runs):
    circs = [_Circ(42, 256, 365, 3401)]
    a = at.autotune(circs, precision="fp32", sample_shots=1 << 10, repeats=1)
    n = len(fake_runs)
    b = at.autotune(circs, precision="fp32", sample_shots=1 << 10, repeats=1)
    assert b is a and len(fake_runs) == n  # cached: no new runs
    at.autotune(circs, precision="fp64", sample_shots=1 << 10, repeats=1)
    assert len(fake_runs) > n  # another precision is another signature
