"""GPU path (through the C ABI) against the FP64 oracle, shot for shot.

Bars (written here, used below):
  - records, status and tallies bit-exact, except shots whose first
    differing outcome had |p - u| <= BAND (counted, must be rare);
  - tableau words (compiled X/Z + per-shot signs) bit-exact;
  - coefficients: same key set, values within 1e-12 (FP64) / 1e-5 (FP32);
    the FP32 comparison drops oracle entries with |v|^2 < 1e-10, the FP32
    pruning threshold.
"""
import numpy as np
import pytest

import oracle
from paper_2512_23037_gb300 import circuits as C

pytestmark = pytest.mark.gpu

BAND = {"fp64": 1e-9, "fp32": 1e-5}
VTOL = {"fp64": 1e-12, "fp32": 1e-5}
TAU = {"fp64": 1e-20, "fp32": 1e-10}


@pytest.fixture(scope="module")
def soft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_23037_gb300 as S
    S.load()
    return S


def _bits(words, nrec):
    return [(int(words[r // 64]) >> (r % 64)) & 1 for r in range(nrec)]


def _band_ok(circ, noise, seed, shot, band, gpu_rec=None):
    """True if the oracle's shot has a sampled outcome with |p - u| <= band at
    or before the measurement of the first record bit where the GPU's record
    differs (anywhere in the shot when the records agree or are not given):
    only an outcome decided within rounding may start a divergence."""
    tr = oracle.trace(circ, circ.n, noise, circ.cap, seed, shot)
    ev = tr["events"]
    stop = len(ev)
    if gpu_rec is not None:
        diff = [r for r in range(64 * len(gpu_rec))
                if ((int(gpu_rec[r // 64]) ^ int(tr["records"][r // 64])) >> (r % 64)) & 1]
        if diff:
            hit = [i for i, e in enumerate(ev) if e["kind"] == 3 and e["b"] == diff[0]]
            stop = hit[0] + 1 if hit else len(ev)
    for e in ev[:stop]:
        if e["kind"] == 3 and not e["det"] and abs(e["p_plus"] - e["u"]) <= band:
            return True
    return False


def _random40():
    """40 qubits and every op kind (T, T^dag, Rz, M, R, MR, Pauli products of
    weight 1-4, feedback Paulis, observables), with measurements frequent
    enough that the noiseless run's maps fit a lane (16 entries) and noisy
    shots stay below the cap (2^8), so that they run to the end."""
    circ = C.random_circuit(4040, 40, 400, t_frac=0.08, meas_frac=0.2, detectors=True, mpp_frac=0.05)
    circ.cap = 256
    return circ


def run_both(S, circ, noise, n_shots, seed, precision, first_shot=0, capture=0, group=0, first_cap=0,
             chunk=0):
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, n_shots, first_shot, seed, precision=precision, record_mode=S.REC_ALL,
                         capture_k=capture, group_size=group, first_cap=first_cap, chunk_shots=chunk)
    rec, st = S.soft_get_records(r, n_shots)
    tal = S.soft_tally(r)
    ref = oracle.run(circ, circ.n, noise, circ.cap, seed, first_shot, n_shots, threads=8)
    return c, r, rec, st, tal, ref


def compare_records(circ, noise, seed, first_shot, rec, st, ref, precision):
    nrec = ref["n_records"]
    band_events = 0
    for i in range(len(st)):
        same = st[i] == ref["status"][i] and np.array_equal(rec[i], ref["records"][i])
        if not same:
            assert _band_ok(circ, noise, seed, first_shot + i, BAND[precision], rec[i]), (
                f"shot {first_shot + i}: status {st[i]} vs {ref['status'][i]}, records "
                f"{_bits(rec[i], nrec)} vs {_bits(ref['records'][i], nrec)}")
            band_events += 1
    return band_events


def compare_states(S, c, r, circ, noise, seed, first_shot, k, precision, statuses=(0,), rec=None, st=None):
    """Final GS state of the first k shots against the oracle's: tableau words
    (kept shots), signs, key set, values. statuses: the oracle statuses
    compared (0 kept, 1 discarded: the state where the failed detector stopped
    the shot, signs and map relative to the shot-invariant X/Z words there). With the
    GPU's records and statuses given, a shot whose outcomes diverged at an
    outcome decided within rounding (the records' band rule) is skipped.
    Returns (states compared, of those the shots whose map outgrew 16 entries,
    i.e. left a first-round lane)."""
    xw, zw = c.tableau()
    n = circ.n
    compared = left = 0
    for off in range(k):
        tr = oracle.trace(circ, n, noise, circ.cap, seed, first_shot + off)
        signs, keys, vals = S.soft_get_state(r, off)
        if tr["status"] not in statuses:
            continue
        if rec is not None and (st[off] != tr["status"] or not np.array_equal(rec[off], tr["records"])):
            assert _band_ok(circ, noise, seed, first_shot + off, BAND[precision], rec[off])
            continue
        compared += 1
        if len(tr["events"]) and int(np.max(tr["events"]["nnz_after"])) > 16:
            left += 1
        # tableau words: compiled X/Z (the circuit's end: kept shots only; the X/Z words are
        # shot-invariant, so a discarded shot shares the oracle's at its stop) + per-shot signs
        if tr["status"] == 0:
            assert np.array_equal(xw, tr["rows_x"]) and np.array_equal(zw, tr["rows_z"])
        rd = [(int(signs[i // 64]) >> (i % 64)) & 1 for i in range(n)]
        rs = [(int(signs[2 + i // 64]) >> (i % 64)) & 1 for i in range(n)]
        assert rd + rs == [int(v) for v in tr["rows_r"]], f"signs differ at shot {first_shot + off}"
        # coefficient map
        ok = np.abs(tr["vals"]) ** 2 >= TAU[precision]
        ok_keys = tr["keys"][ok]
        ok_vals = tr["vals"][ok]
        order = np.lexsort((keys[:, 0], keys[:, 1]))
        keys, vals = keys[order], vals[order]
        assert np.array_equal(keys, ok_keys), f"key sets differ at shot {first_shot + off}"
        assert np.max(np.abs(vals - ok_vals)) <= VTOL[precision], f"values differ at shot {first_shot + off}"
    return compared, left


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiny_workload(soft, precision):
    circ, noise = C.workload("tiny6")
    noise = C.Noise.uniform(0.02)
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 3000, 0, precision, capture=64)
    assert compare_records(circ, noise, 0, 0, rec, st, ref, precision) <= 3
    assert [tal["shots"], tal["discarded"], tal["overflow"], tal["kept"], tal["logical_errors"]][0] == 3000
    compare_states(soft, c, r, circ, noise, 0, 0, 64, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(6))
def test_random_circuits(soft, precision, seed):
    """Every op kind: T/T^dag/Rz, case-A and case-B measurements, resets,
    feedback Paulis, observables; several tiles and a ragged tail."""
    n = [3, 5, 8, 12, 40, 70][seed]
    circ = C.random_circuit(1000 + seed, n, 60 + 8 * n, t_frac=0.2, detectors=True)
    circ.cap = 256
    noise = C.Noise(0.01, 0.01, 0.01, 0.01)
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 777, seed, precision, capture=48)
    assert compare_records(circ, noise, seed, 0, rec, st, ref, precision) <= 3
    compare_states(soft, c, r, circ, noise, seed, 0, 48, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_w42_prefix(soft, precision):
    circ, noise = C.workload("w42")
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 10000, 0, precision, capture=32)
    band = compare_records(circ, noise, 0, 0, rec, st, ref, precision)
    assert band <= 5
    t = ref["tally"]
    if band == 0:
        assert [tal["shots"], tal["discarded"], tal["overflow"], tal["kept"], tal["logical_errors"]] == t
    compare_states(soft, c, r, circ, noise, 0, 0, 32, precision)


def test_w42_far_shot_range(soft):
    """Shot indices far from 0 (counter words above 2^32) and a chunked run."""
    circ, noise = C.workload("w42")
    first = (1 << 40) + 12345
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 3000, 7, "fp64", first_shot=first, chunk=1000)
    assert compare_records(circ, noise, 7, first, rec, st, ref, "fp64") == 0


def test_rerun_pass_matches_single_pass(soft):
    """A tiny first-pass capacity forces most shots through the rerun pass."""
    circ, noise = C.workload("w42")
    for fc in (2, 8):
        c, r, rec, st, tal, ref = run_both(soft, circ, noise, 2000, 3, "fp64", first_cap=fc)
        assert compare_records(circ, noise, 3, 0, rec, st, ref, "fp64") == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("group", [16, 32])
def test_group_sizes(soft, group, precision):
    circ, noise = C.workload("w42")
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 2000, 5, precision, group=group, capture=64)
    assert compare_records(circ, noise, 5, 0, rec, st, ref, precision) <= 2
    compare_states(soft, c, r, circ, noise, 5, 0, 64, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(4))
def test_two_shots_per_warp_random_circuits(soft, precision, seed):
    """16-lane groups: register maps of up to 16 entries, spills to the shared
    hash beyond, two shots of one warp on different paths."""
    n = [4, 9, 30, 80][seed]
    circ = C.random_circuit(3000 + seed, n, 60 + 8 * n, t_frac=0.22, detectors=True, mpp_frac=0.05)
    circ.cap = 256
    noise = C.Noise(0.01, 0.01, 0.01, 0.01)
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 900, seed, precision, capture=48, group=16)
    assert compare_records(circ, noise, seed, 0, rec, st, ref, precision) <= 3
    compare_states(soft, c, r, circ, noise, seed, 0, 48, precision)


def test_overflow_status(soft):
    c = C.Circuit(6, cap=8)
    for q in range(6):
        c.gate(C.H, q)
        c.gate(C.T, q)
    c.measure(0)
    _, _, rec, st, tal, ref = run_both(soft, c, C.Noise(), 50, 0, "fp64")
    assert list(st) == list(ref["status"]) == [2] * 50
    assert tal["overflow"] == 50


def test_noiseless_w42_all_kept(soft):
    circ, _ = C.workload("w42")
    S = soft
    c = S.soft_compile_circuit(circ.array(), circ.n, C.Noise(), circ.cap)
    r = S.soft_run_shots(c, 20000, 0, 0, precision="fp32")
    t = S.soft_tally(r)
    assert (t["shots"], t["discarded"], t["overflow"], t["kept"], t["logical_errors"]) == (20000, 0, 0, 20000, 0)


def test_zero_and_one_shot(soft):
    circ, noise = C.workload("tiny6")
    S = soft
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, 0, 0, 0)
    assert S.soft_tally(r)["shots"] == 0
    c2, r2, rec, st, tal, ref = run_both(S, circ, noise, 1, 0, "fp64")
    assert tal["shots"] == 1 and compare_records(circ, noise, 0, 0, rec, st, ref, "fp64") == 0


def test_bench_config_sampled(soft):
    """The bench's launch configuration (w42, FP32, 2^24 shots in one chunk,
    default tuning: lane per shot, eviction rounds, handover, middle pass):
    tallies are consistent and sampled shots match the oracle."""
    S = soft
    circ, noise = C.workload("w42")
    n = 1 << 24
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, n, 0, 0, precision="fp32", record_mode=S.REC_ALL)
    rec, st = S.soft_get_records(r, n)
    t = S.soft_tally(r)
    assert t["shots"] == n and t["discarded"] + t["overflow"] + t["kept"] == n
    assert np.sum(st == 1) == t["discarded"] and np.sum(st == 0) == t["kept"]
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(n, size=300, replace=False))
    band = 0
    for s in sample:
        ref = oracle.run(circ, circ.n, noise, circ.cap, 0, int(s), 1)
        if not (ref["status"][0] == st[s] and np.array_equal(ref["records"][0], rec[s])):
            assert _band_ok(circ, noise, 0, int(s), BAND["fp32"])
            band += 1
    assert band <= 2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_w97_two_word_keys(soft, precision):
    """97 qubits (two-word keys and signs), cap 2^12: the rerun pass runs from
    a global-memory slab because that state does not fit in shared memory."""
    circ, noise = C.workload("w97")
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 1500, 0, precision, capture=16)
    assert compare_records(circ, noise, 0, 0, rec, st, ref, precision) <= 2
    compare_states(soft, c, r, circ, noise, 0, 0, 16, precision)


def test_global_memory_rerun_forced(soft):
    """cap 8192 (FP64) cannot live in shared memory; first_cap 2 sends almost
    every shot through the global-memory rerun pass."""
    circ = C.random_circuit(4242, 10, 140, t_frac=0.35, meas_frac=0.05, detectors=True)
    circ.cap = 8192
    noise = C.Noise(0.01, 0.01, 0.01, 0.01)
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 400, 11, "fp64", capture=24, first_cap=2)
    assert compare_records(circ, noise, 11, 0, rec, st, ref, "fp64") <= 1
    compare_states(soft, c, r, circ, noise, 11, 0, 24, "fp64")


def _small_batch():
    """Windowed circuits with different qubit counts, windows (caps), block
    counts and noise levels."""
    specs = [(17, 2, 3, 2e-3), (21, 3, 4, 1e-3), (26, 4, 3, 3e-3), (19, 5, 2, 5e-4), (30, 2, 5, 2e-3),
             (23, 6, 2, 1e-3)]
    out = []
    for k, (n, w, blocks, p) in enumerate(specs):
        circ, noise = C.windowed(300 + k, n_data=n - 4, n_anc=4, blocks=blocks, w=w, n_cliff=30, checks=4, p=p)
        out.append((circ, noise, 300 + 97 * k))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_runs_and_oracle(soft, precision):
    """One launch over six circuits: per-circuit tallies equal the circuits'
    own runs, and (FP64) the oracle's."""
    S = soft
    batch = _small_batch()
    circs = [S.soft_compile_circuit(c.array(), c.n, nz, c.cap) for c, nz, _ in batch]
    shots = [n for _, _, n in batch]
    firsts = [1000 * k for k in range(len(batch))]
    r = S.soft_run_batch(circs, shots, firsts, 21, precision=precision)
    for i, ((circ, noise, n), h) in enumerate(zip(batch, circs)):
        tb = S.soft_tally_batch(r, i)
        r1 = S.soft_run_shots(h, n, firsts[i], 21, precision=precision)
        t1 = S.soft_tally(r1)
        key = ("shots", "discarded", "overflow", "kept", "logical_errors")
        assert [tb[k] for k in key] == [t1[k] for k in key], i
        if precision == "fp64":
            ref = oracle.run(circ, circ.n, noise, circ.cap, 21, firsts[i], n, threads=8, records=False)
            assert [tb[k] for k in key] == ref["tally"], i
    tot = S.soft_tally(r)
    assert tot["shots"] == sum(shots)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mixed", [False, True])
def test_batch_lane_per_shot(soft, precision, mixed):
    """A batch of windowed circuits of different sizes runs lane per shot (a
    bucket range per circuit, warps moving between circuits); mixed: circuits
    with 5- and 6-qubit windows (maps beyond a lane) among them, whose shots go
    straight to the warp pass. Per-circuit tallies against the warp-per-shot
    batch, and (FP64) the oracle's."""
    S = soft
    batch = [C.windowed(40 + k, blocks=2 + k % 4, n_data=30 + 4 * k, p=3e-3) for k in range(5)]
    if mixed:
        batch.insert(1, C.windowed(50, blocks=3, n_data=28, w=5, p=2e-3))
        batch.insert(4, C.windowed(51, blocks=2, n_data=32, w=6, p=2e-3))
    circs = [S.soft_compile_circuit(c.array(), c.n, nz, c.cap) for c, nz in batch]
    shots = [3000 + 500 * k for k in range(len(batch))]
    firsts = [777 * k for k in range(len(batch))]
    r = S.soft_run_batch(circs, shots, firsts, 8, precision=precision, time_passes=True)
    assert S.soft_run_pass_timing(r)[0][0] > 0.0  # the lane pre-pass ran
    rw = S.soft_run_batch(circs, shots, firsts, 8, precision=precision, lanes=False)
    key = ("shots", "discarded", "overflow", "kept", "logical_errors")
    for i, ((circ, noise), n) in enumerate(zip(batch, shots)):
        tb, tw = S.soft_tally_batch(r, i), S.soft_tally_batch(rw, i)
        assert tb["shots"] == tw["shots"] == n
        assert all(abs(tb[k] - tw[k]) <= 2 for k in key), (i, tb, tw)
        if precision == "fp64":
            ref = oracle.run(circ, circ.n, noise, circ.cap, 8, firsts[i], n, threads=8, records=False)
            assert all(abs(a - b) <= 2 for a, b in zip([tb[k] for k in key], ref["tally"])), (i, tb, ref["tally"])
    assert S.soft_tally(r)["shots"] == sum(shots)


def test_autotune_choice_is_valid_and_exact(soft):
    """The autotuner times every candidate shape of a reduced space (the library
    default, lane per shot, among them) on a batch and returns the fastest; a run
    with its choice gives the default run's per-circuit tallies (up to outcomes
    within rounding)."""
    from paper_2512_23037_gb300.autotune import autotune
    S = soft
    batch = [C.windowed(60 + k, blocks=2, n_data=30, p=3e-3) for k in range(3)]
    circs = [S.soft_compile_circuit(c.array(), c.n, nz, c.cap) for c, nz in batch]
    space = {"first_cap": [32, 64], "groups_per_block": [4], "group_size": [0, 32]}
    res = autotune(circs, precision="fp32", sample_shots=1 << 14, space=space, repeats=1)
    assert len(res["table"]) == 4 and res["best"] in [kw for _, kw in res["table"]]
    assert all(ms > 0 for ms, _ in res["table"])
    shots, firsts = [4000] * 3, [0, 5000, 10000]
    r = S.soft_run_batch(circs, shots, firsts, 2, precision="fp32", **res["best"])
    r0 = S.soft_run_batch(circs, shots, firsts, 2, precision="fp32")
    for i in range(3):
        a, b = S.soft_tally_batch(r, i), S.soft_tally_batch(r0, i)
        assert a["shots"] == b["shots"] == 4000
        assert all(abs(a[k] - b[k]) <= 2 for k in ("discarded", "kept", "logical_errors"))


def test_batch_with_global_memory_reruns(soft):
    """A batch where one circuit's cap (2^12) forces global-memory reruns."""
    S = soft
    batch = _small_batch()
    circs = [S.soft_compile_circuit(c.array(), c.n, nz, c.cap) for c, nz, _ in batch]
    shots = [n for _, _, n in batch]
    r = S.soft_run_batch(circs, shots, [0] * len(batch), 3, precision="fp64", first_cap=4)
    for i, (circ, noise, n) in enumerate(batch):
        ref = oracle.run(circ, circ.n, noise, circ.cap, 3, 0, n, threads=8, records=False)
        t = S.soft_tally_batch(r, i)
        assert [t["shots"], t["discarded"], t["overflow"], t["kept"], t["logical_errors"]] == ref["tally"], i


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replayed_chunks(soft, precision):
    """Chunks replayed from one captured CUDA graph give the same records."""
    import torch
    S = soft
    circ, noise = C.workload("w42")
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    stream = torch.cuda.Stream()
    n, chunk = 5000, 1000
    r = S.soft_run_shots(c, n, 77, 4, precision=precision, record_mode=S.REC_ALL, chunk_shots=chunk,
                         stream=stream, graph=True)
    rec, st = S.soft_get_records(r, n)
    ms, launches = S.soft_run_timing(r)
    assert launches >= 5 * 2
    ref = oracle.run(circ, circ.n, noise, circ.cap, 4, 77, n, threads=8)
    assert compare_records(circ, noise, 4, 77, rec, st, ref, precision) <= 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_workspace_reuse_is_clean(soft, precision):
    """Runs borrow the device's cached workspace, left dirty by the run before
    (another circuit, other shots, records, captured states): records, statuses,
    tallies and states equal those of a run on a freshly allocated workspace."""
    S = soft
    circ, noise = C.workload("w42")
    small, nz2 = C.workload("tiny6")
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    c2 = S.soft_compile_circuit(small.array(), small.n, nz2, small.cap)

    def run(cc, n, first, **kw):
        r = S.soft_run_shots(cc, n, first, 5, precision=precision, record_mode=S.REC_ALL, **kw)
        rec, st = S.soft_get_records(r, n)
        states = [S.soft_get_state(r, k) for k in range(kw.get("capture_k", 0))]
        t = S.soft_tally(r)
        r.free()
        return rec, st, t, states

    S.soft_release_workspace()
    fresh = run(c, 6000, 100, chunk_shots=2000)
    S.soft_release_workspace()
    fresh_cap = run(c, 300, 7, capture_k=16)
    # dirty the cache with other circuits and shots, then repeat both
    run(c2, 20000, 0)
    run(c, 9000, 50000, chunk_shots=3000)
    again = run(c, 6000, 100, chunk_shots=2000)
    again_cap = run(c, 300, 7, capture_k=16)
    for a, b in ((fresh, again), (fresh_cap, again_cap)):
        assert (a[0] == b[0]).all() and (a[1] == b[1]).all() and a[2] == b[2]
        for (s1, k1, v1), (s2, k2, v2) in zip(a[3], b[3]):
            assert (s1 == s2).all() and (k1 == k2).all() and (v1 == v2).all()
    S.soft_release_workspace()
    c.free()
    c2.free()


@pytest.mark.parametrize("lanes", [True, False])
def test_pass_timing(soft, lanes):
    """Per-pass events: one set per chunk, each pass non-negative, the sum within
    the run's own events; the pre-pass runs only with lane-per-shot scheduling;
    runs without the flag, or replayed from a graph, report SOFT_E_ARG."""
    S = soft
    circ, noise = C.workload("w42")
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, 30000, 0, 1, precision="fp32", chunk_shots=10000, lanes=lanes, time_passes=True)
    t = S.soft_tally(r)
    assert t["shots"] == 30000
    ms, chunks, n_rerun = S.soft_run_pass_timing(r)
    total, _ = S.soft_run_timing(r)
    assert chunks == 3 and min(ms) >= 0.0 and ms[1] > 0.0
    assert (ms[0] > 0.0) == lanes
    assert 0 <= n_rerun <= 30000 and (n_rerun == 0 or ms[2] > 0.0)
    assert sum(ms) <= total * 1.01 + 0.01
    r.free()
    r = S.soft_run_shots(c, 1000, 0, 1, precision="fp32")
    with pytest.raises(S.SoftError):
        S.soft_run_pass_timing(r)
    r.free()


def _run_prefix(S, c, n, seed, precision, prefix, **kw):
    # a warp per shot on both sides: the lane kernel always starts from the prefix
    r = S.soft_run_shots(c, n, 0, seed, precision=precision, record_mode=S.REC_ALL, capture_k=48, prefix=prefix,
                         lanes=False, **kw)
    rec, st = S.soft_get_records(r, n)
    states = [S.soft_get_state(r, off) for off in range(48)]
    return rec, st, S.soft_tally(r), states


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["w42", "tiny6", "random40", "w42_rerun", "w97"])
def test_prefix_start_is_bit_identical(soft, precision, case):
    """Starting each shot from the noiseless run's state at its first error
    (the default) gives exactly the records, statuses, tallies and final states
    of running it from the first event."""
    S = soft
    kw = {}
    if case in ("w42", "w42_rerun"):
        circ, noise = C.workload("w42")
        if case == "w42_rerun":
            kw = {"first_cap": 8}
    elif case == "w97":  # two-word keys, snapshots above 32 entries held in shared memory
        circ, noise = C.workload("w97")
    elif case == "tiny6":
        circ, noise = C.workload("tiny6")
        noise = C.Noise.uniform(0.02)
    else:
        circ = _random40()
        noise = C.Noise(0.005, 0.005, 0.005, 0.005)
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    a = _run_prefix(S, c, 3000, 9, precision, True, **kw)
    b = _run_prefix(S, c, 3000, 9, precision, False, **kw)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2]
    for (s1, k1, v1), (s2, k2, v2) in zip(a[3], b[3]):
        assert np.array_equal(s1, s2) and np.array_equal(k1, k2) and np.array_equal(v1, v2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_maximum_qubits_128(soft, precision):
    """n = 128, the largest register the two-word keys hold."""
    circ = C.random_circuit(6128, 128, 700, t_frac=0.04, meas_frac=0.2, detectors=True, mpp_frac=0.04)
    circ.cap = 256
    noise = C.Noise(0.004, 0.004, 0.004, 0.004)
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 400, 3, precision, capture=24)
    assert compare_records(circ, noise, 3, 0, rec, st, ref, precision) <= 2
    compare_states(soft, c, r, circ, noise, 3, 0, 24, precision)


def _many_records(n_rounds):
    rng = np.random.default_rng(77)
    c = C.Circuit(12, cap=256)
    for _ in range(n_rounds):
        for q in range(12):
            c.gate([C.H, C.S, C.T, C.T_DAG][int(rng.integers(4))], q)
        a, b = (int(v) for v in rng.choice(12, size=2, replace=False))
        c.gate(C.CX, a, b)
        for q in range(12):
            c.measure(q, reset=bool(rng.integers(2)))
    return c


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_maximum_records_1020(soft, precision):
    """85 rounds of 12 measurements: 1020 records, 16 record words per shot."""
    circ = _many_records(85)
    assert circ.n_records == 1020
    noise = C.Noise(0.01, 0.01, 0.01, 0.01)
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 300, 4, precision)
    assert rec.shape[1] == 16
    assert compare_records(circ, noise, 4, 0, rec, st, ref, precision) <= 2


def test_more_than_1024_records_rejected(soft):
    circ = _many_records(86)  # 1032 records
    with pytest.raises(soft.SoftError):
        soft.soft_compile_circuit(circ.array(), circ.n, C.Noise(), circ.cap)


@pytest.mark.parametrize("case", ["empty", "clifford_only", "no_measurements", "one_qubit"])
def test_degenerate_circuits(soft, case):
    """An empty op list, a Clifford-only circuit (the map stays one entry), a
    circuit without measurements, a one-qubit circuit: tallies and records
    equal the oracle's."""
    n = 1 if case == "one_qubit" else 5
    c = C.Circuit(n, cap=16)
    rng = np.random.default_rng(5)
    if case != "empty":
        for _ in range(40):
            q = int(rng.integers(n))
            if case == "clifford_only" or n == 1:
                c.gate([C.H, C.S, C.X, C.Z, C.S_DAG][int(rng.integers(5))], q)
            elif rng.random() < 0.3:
                c.gate(C.CX, q, (q + 1) % n)
            else:
                c.gate([C.H, C.T, C.S][int(rng.integers(3))], q)
        if case == "one_qubit":
            c.gate(C.T, 0)
            c.measure(0)
        elif case == "clifford_only":
            for q in range(n):
                c.measure(q)
    noise = C.Noise(0.05, 0.05, 0.05, 0.05)
    cc, r, rec, st, tal, ref = run_both(soft, c, noise, 500, 2, "fp64")
    assert [tal["shots"], tal["discarded"], tal["overflow"], tal["kept"], tal["logical_errors"]] == ref["tally"]
    assert compare_records(c, noise, 2, 0, rec, st, ref, "fp64") == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["w42", "random40"])
def test_wide_round_matches_oracle(soft, precision, case):
    """Shots whose maps outgrow a lane continue in the wide round's lanes (32
    entries) before any warp: records and statuses against the oracle, tallies
    against runs without the wide round."""
    S = soft
    if case == "w42":
        circ, noise = C.workload("w42")
        noise = C.Noise.uniform(3e-3)  # more errors: more maps outgrow a lane
    else:
        circ = _random40()
        noise = C.Noise(0.005, 0.005, 0.005, 0.005)
    n_shots = 6000
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, n_shots, 0, 13, precision=precision, record_mode=S.REC_ALL, time_passes=True, wide=True)
    rec, st = S.soft_get_records(r, n_shots)
    t = S.soft_tally(r)
    assert S.soft_run_diagnostics(r)[0] == 0
    ms, _, n_left = S.soft_run_pass_timing(r)
    assert ms[0] > 0.0  # lanes ran
    if case == "w42":
        assert n_left > 0  # and some shots left them (random40's maps stay within a lane)
    ref = oracle.run(circ, circ.n, noise, circ.cap, 13, 0, n_shots, threads=8)
    assert compare_records(circ, noise, 13, 0, rec, st, ref, precision) <= 2
    t2 = S.soft_tally(S.soft_run_shots(c, n_shots, 0, 13, precision=precision, wide=False))
    assert all(abs(t[k] - t2[k]) <= 2 for k in ("discarded", "overflow", "kept", "logical_errors"))


@pytest.mark.parametrize("precision,wide", [("fp64", None), ("fp32", None), ("fp32", True)])
@pytest.mark.parametrize("n_data,n_anc", [(72, 4), (120, 8)])
def test_lane_per_shot_two_word_keys(soft, precision, wide, n_data, n_anc):
    """Above 64 qubits (two-word keys, signs and spill records) in the lane
    kernel, and (wide) in the wide round's lanes: windowed circuits of 76 and
    128 qubits, whose noiseless maps fit a lane, against the oracle."""
    S = soft
    circ, noise = C.windowed(11, n_data=n_data, n_anc=n_anc, blocks=4, p=4e-3)
    n_shots = 3000
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, n_shots, 0, 9, precision=precision, record_mode=S.REC_ALL, time_passes=True,
                         wide=wide)
    rec, st = S.soft_get_records(r, n_shots)
    assert S.soft_run_diagnostics(r)[0] == 0
    ms, _, n_left = S.soft_run_pass_timing(r)
    assert ms[0] > 0.0  # the lane pre-pass ran
    if wide:
        assert n_left > 0  # some shots left their lanes (to the wide round)
    ref = oracle.run(circ, circ.n, noise, circ.cap, 9, 0, n_shots, threads=8)
    assert compare_records(circ, noise, 9, 0, rec, st, ref, precision) <= 2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["w42", "w42_rerun_chunks", "w42_mid32", "tiny6", "random40", "random40_mid32",
                                  "w97"])
def test_lane_per_shot_matches_oracle(soft, precision, case):
    """One shot per lane, 32 per warp, event-aligned: records, statuses and
    tallies against the oracle (and the tallies of the warp-per-shot kernel).
    Shots whose maps outgrow a lane go through the middle pass (a warp, up to
    first_cap entries) and the pass at the circuit's cap."""
    S = soft
    kw = {}
    n_shots = 3000
    if case.startswith("w42"):
        circ, noise = C.workload("w42")
        if case == "w42_rerun_chunks":
            kw = {"first_cap": 8, "chunk_shots": 1000}
        elif case == "w42_mid32":
            kw = {"first_cap": 32, "chunk_shots": 1000}
    elif case == "w97":
        circ, noise = C.workload("w97")
        n_shots = 800
    elif case == "tiny6":
        circ, noise = C.workload("tiny6")
        noise = C.Noise.uniform(0.02)
    else:
        circ = _random40()
        noise = C.Noise(0.005, 0.005, 0.005, 0.005)
        if case == "random40_mid32":
            kw = {"first_cap": 32}
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, n_shots, 0, 9, precision=precision, record_mode=S.REC_ALL, time_passes=True, **kw)
    rec, st = S.soft_get_records(r, n_shots)
    tal = S.soft_tally(r)
    assert S.soft_run_diagnostics(r)[0] == 0
    if case.startswith("w42"):
        assert S.soft_run_pass_timing(r)[2] > 0  # some shots left their lane
    ref = oracle.run(circ, circ.n, noise, circ.cap, 9, 0, n_shots, threads=8)
    assert compare_records(circ, noise, 9, 0, rec, st, ref, precision) <= 2
    t2 = S.soft_tally(S.soft_run_shots(c, n_shots, 0, 9, precision=precision, lanes=False, **kw))
    assert abs(tal["kept"] - t2["kept"]) <= 2 and tal["shots"] == t2["shots"] == n_shots


def _lane_case(case):
    """(circuit, noise, run keywords) of the lane-kernel state-parity cases."""
    if case.startswith("w42"):
        circ, noise = C.workload("w42")
        if case == "w42_p3e-3":
            noise = C.Noise.uniform(3e-3)
        return circ, noise, ({"first_cap": 32} if case == "w42_mid32" else {})
    if case == "random40_mpp":
        circ = _random40()
        return circ, C.Noise(0.005, 0.005, 0.005, 0.005), {}
    if case == "win5":  # 5-qubit windows: noiseless maps of 32 entries, a 32-entry first-pass lane
        circ, noise = C.windowed(12, n_data=36, n_anc=4, blocks=3, w=5, p=3e-3)
        return circ, noise, {}
    if case == "w97":  # 6-qubit windows, two key words: 64-entry first-pass lanes (FP32), warps (FP64)
        circ, noise = C.workload("w97")
        return circ, noise, {}
    n_data, n_anc = {"win76": (72, 4), "win128": (120, 8)}[case]
    circ, noise = C.windowed(11, n_data=n_data, n_anc=n_anc, blocks=4, p=4e-3)
    return circ, noise, {}


@pytest.mark.parametrize("precision,wide", [("fp64", False), ("fp64", True), ("fp32", False), ("fp32", True)])
@pytest.mark.parametrize("case", ["w42", "w42_p3e-3", "w42_mid32", "random40_mpp", "win76", "win128", "win5", "w97"])
def test_lane_kernel_states_match_oracle(soft, precision, wide, case):
    """State capture keeps lane-per-shot scheduling: each captured shot's final
    signs, keys and values are written from wherever it ends (a first-round
    lane, an eviction round, the wide round's lanes, the middle warp pass after
    a hand-over, the pass at the circuit's cap), and equal the oracle's within
    1e-12 (FP64) / 1e-5 (FP32) for kept and discarded shots, with and without
    the wide round in either precision; also for circuits whose noiseless maps
    need a 32-entry (win5) or, in FP32, a 64-entry (w97) first-pass lane, which
    never hand over (a shot that outgrows it runs again in a warp). Theorem 1
    (update rules) in the GS representation of Sec. II-C."""
    S = soft
    if wide and case in ("win5", "w97"):
        pytest.skip("the wide round follows 16-entry lanes only")
    circ, noise, kw = _lane_case(case)
    k = 512
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(c, k, 0, 17, precision=precision, record_mode=S.REC_ALL, capture_k=k, time_passes=True,
                         wide=wide, **kw)
    rec, st = S.soft_get_records(r, k)
    assert S.soft_run_diagnostics(r)[0] == 0
    ms, _, n_left = S.soft_run_pass_timing(r)
    if not (case == "w97" and precision == "fp64"):  # (64-entry lanes are FP32 only)
        assert ms[0] > 0.0  # the lane pre-pass ran: lane-per-shot scheduling was kept
    ref = oracle.run(circ, circ.n, noise, circ.cap, 17, 0, k, threads=8)
    assert compare_records(circ, noise, 17, 0, rec, st, ref, precision) <= 2
    compared, left = compare_states(S, c, r, circ, noise, 17, 0, k, precision, statuses=(0, 1), rec=rec, st=st)
    assert compared >= 64, compared
    if case.startswith("w42"):
        assert n_left > 0 and left > 0, (n_left, left)  # the sample holds shots that left their lane


def test_lane_overflow_rule_below_lane_capacity(soft):
    """A circuit whose cap (8) is below a lane's map (16 entries): four T gates
    on |+> states make 16 entries, above the cap, so every shot overflows
    (nonzero count after pruning above the cap), in lanes as in the oracle."""
    S = soft
    c = C.Circuit(6, cap=8)
    for q in range(4):
        c.gate(C.H, q)
        c.gate(C.T, q)
    c.measure(5)
    for precision in ("fp64", "fp32"):
        _, r, rec, st, tal, ref = run_both(S, c, C.Noise(), 64, 0, precision)
        assert list(ref["status"]) == [2] * 64
        assert list(st) == [2] * 64 and tal["overflow"] == 64
