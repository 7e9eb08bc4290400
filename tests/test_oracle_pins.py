"""Pins of the FP64 oracle against things other than itself.

Every check here is CPU only. Sources of truth: published Philox vectors,
dense matrices, an independent Aaronson-Gottesman sampler, closed forms and
the invariants of Theorem 1 / the coset bound of arxiv 2512.23037.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2512_23037_gb300 import circuits as C
from tests import ag_ref, dense_ref

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ RNG
def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert oracle.philox(w[0:4], w[4:6]) == w[6:10]


def test_gap_threshold_closed_form():
    # p = 1/2: 1 - (1/2)^(g+1) is exact in binary
    for g in range(8):
        assert oracle.gap_threshold(0.5, g) == (1 << 64) - (1 << (63 - g))
    # small g: 2^64 * (1 - (1-p)^(g+1)) to double precision
    p = 1e-3
    for g in (0, 1, 10, 1000):
        want = (1.0 - (1.0 - p) ** (g + 1)) * 2.0 ** 64
        assert abs(oracle.gap_threshold(p, g) / want - 1) < 1e-12
    t = [oracle.gap_threshold(1e-3, g) for g in range(2000)]
    assert all(a <= b for a, b in zip(t, t[1:]))


def test_uniform53_is_exact_and_in_range():
    for j in range(200):
        u = oracle.uniform53(7, 11, j)
        assert 0.0 <= u < 1.0
        assert float(u * 2 ** 53).is_integer()


def test_noise_rate_matches_p():
    """Error counts of the geometric-gap stream: mean p * sites."""
    c = C.Circuit(2)
    for _ in range(500):
        c.gate(C.H, 0)
    nz = C.Noise(p1=0.02)
    r = oracle.run(c, 2, nz, 16, 3, 0, 4000, threads=4)
    per_shot = r["counts"]["errors"] / 4000
    assert abs(per_shot - 10.0) < 0.3  # 500 * 0.02 = 10, sd/sqrt(N) ~ 0.05


# ------------------------------------------------------------------ Clifford rules vs matrices
def _dense_unitary(circ):
    n = circ.n
    dim = 1 << n
    U = np.zeros((dim, dim), complex)
    for j in range(dim):
        v = np.zeros(dim, complex)
        v[j] = 1
        for o in circ.ops:
            if o[0] in C.ONE_Q:
                v = dense_ref.apply_1q(v, n, o[2], dense_ref.one_q_matrix(o[0], o[5]))
            else:
                v = dense_ref.apply_2q(v, n, o[0], o[2], o[3])
        U[:, j] = v
    return U


def _row_matrix(n, x, z, r):
    dim = 1 << n
    M = np.zeros((dim, dim), complex)
    for j in range(dim):
        e = np.zeros(dim, complex)
        e[j] = 1
        M[:, j] = dense_ref.pauli_row_apply(e, n, x, z, r)
    return M


@pytest.mark.parametrize("seed", range(6))
def test_clifford_conjugation_matches_dense(seed):
    rng = np.random.default_rng(seed)
    n = 3
    c = C.Circuit(n)
    for _ in range(40):
        if rng.random() < 0.4:
            a, b = (int(v) for v in rng.choice(n, 2, replace=False))
            c.gate(C.CX if rng.random() < 0.5 else C.CZ, a, b)
        else:
            c.gate(C.CLIFFORD_1Q[int(rng.integers(6))], int(rng.integers(n)))
    tr = oracle.trace(c, n, C.Noise(), 4, 0, 0)
    U = _dense_unitary(c)
    for i in range(2 * n):
        x = int(tr["rows_x"][i][0])
        z = int(tr["rows_z"][i][0])
        r = int(tr["rows_r"][i])
        P0 = _row_matrix(n, (1 << i) if i < n else 0, (1 << (i - n)) if i >= n else 0, 0)
        assert np.allclose(U @ P0 @ U.conj().T, _row_matrix(n, x, z, r))


# ------------------------------------------------------------------ dense statevector replay
def _check_replay(circ, noise, shot, seed, stop_after=None):
    tr = oracle.trace(circ, circ.n, noise, circ.cap, seed, shot, stop_after=stop_after)
    rep = dense_ref.replay(circ, noise, tr["events"], stop_after=stop_after)
    assert rep["mismatches"] == 0
    assert rep["p_err"] < 1e-10
    assert rep["status"] == tr["status"]
    if tr["status"] == 0:
        gs = dense_ref.gs_to_dense(circ.n, tr["rows_x"], tr["rows_z"], tr["rows_r"], tr["keys"], tr["vals"])
        fid = abs(np.vdot(rep["psi"], gs))
        assert abs(fid - 1) < 1e-10, fid
        nrec = len(rep["records"])
        bits = [(int(tr["records"][r // 64]) >> (r % 64)) & 1 for r in range(nrec)]
        assert bits == rep["records"]
        assert rep["logical"] == tr["logical"]
    return tr


@pytest.mark.parametrize("seed", range(12))
def test_dense_replay_random_circuits(seed):
    n = 2 + seed % 5
    circ = C.random_circuit(seed, n, 60 + 10 * n, detectors=(seed % 3 == 0))
    noise = C.Noise(0.03, 0.03, 0.02, 0.02)
    for shot in range(6):
        _check_replay(circ, noise, shot, seed=100 + seed)


@pytest.mark.parametrize("seed", range(4))
def test_dense_replay_prefixes(seed):
    """State equality at intermediate steps: the GS state after every 7th op."""
    circ = C.random_circuit(50 + seed, 4, 50)
    noise = C.Noise(0.05, 0.05, 0.0, 0.05)
    for k in range(1, len(circ.ops), 7):
        _check_replay(circ, noise, 1, seed=seed, stop_after=k)


def test_dense_replay_tiny_workload():
    circ, noise = C.workload("tiny6")
    noise = C.Noise.uniform(0.02)  # enough errors to exercise every path
    for shot in range(25):
        _check_replay(circ, noise, shot, seed=0)


def test_dense_replay_windowed_small():
    circ, noise = C.windowed(5, n_data=7, n_anc=2, blocks=3, w=3, n_cliff=12, checks=2, p=0.01)
    for shot in range(12):
        _check_replay(circ, noise, shot, seed=1)


# ------------------------------------------------------------------ Aaronson-Gottesman
def _oracle_stabilizers(tr, n):
    alpha = int(tr["keys"][0][0]) | (int(tr["keys"][0][1]) << 64)
    rows = []
    for i in range(n):
        x = int(tr["rows_x"][n + i][0]) | (int(tr["rows_x"][n + i][1]) << 64)
        z = int(tr["rows_z"][n + i][0]) | (int(tr["rows_z"][n + i][1]) << 64)
        r = int(tr["rows_r"][n + i]) ^ ((alpha >> i) & 1)  # d_a s_i d_a = (-1)^{a_i} s_i
        rows.append((x, z, r))
    return rows


@pytest.mark.parametrize("seed", range(10))
def test_clifford_only_against_aaronson_gottesman(seed):
    n = 3 + seed % 6
    circ = C.random_circuit(200 + seed, n, 120, t_frac=0.0, meas_frac=0.15, rz=False, feedback=False)
    noise = C.Noise(0.05, 0.05, 0.05, 0.05)
    for shot in range(5):
        tr = oracle.trace(circ, n, noise, circ.cap, seed, shot)
        assert tr["status"] == 0 and len(tr["keys"]) == 1
        t, recs = ag_ref.run(circ, noise, tr["events"])
        bits = [(int(tr["records"][r // 64]) >> (r % 64)) & 1 for r in range(len(recs))]
        assert bits == recs
        assert ag_ref.canonical(n, _oracle_stabilizers(tr, n)) == ag_ref.canonical(n, t.stabilizers())


# ------------------------------------------------------------------ closed forms
def _meas_events(tr):
    return [e for e in tr["events"] if e["kind"] == 3]


def test_hth_closed_form():
    c = C.Circuit(1)
    c.gate(C.H, 0); c.gate(C.T, 0); c.gate(C.H, 0); c.measure(0)
    e = _meas_events(oracle.trace(c, 1, C.Noise(), 16, 0, 0))[0]
    assert abs(e["p_plus"] - (2 + np.sqrt(2)) / 4) < 1e-14


def test_t_on_zero_is_deterministic():
    c = C.Circuit(1)
    c.gate(C.T, 0); c.measure(0)
    tr = oracle.trace(c, 1, C.Noise(), 16, 0, 0)
    e = _meas_events(tr)[0]
    assert e["det"] == 1 and e["outcome"] == 1
    assert len(tr["keys"]) == 1


@pytest.mark.parametrize("theta", [0.1, 0.7, 1.3, 2.9, -2.2])
def test_rz_closed_form(theta):
    c = C.Circuit(1)
    c.gate(C.H, 0); c.gate(C.RZ, 0, angle=theta); c.gate(C.H, 0); c.measure(0)
    e = _meas_events(oracle.trace(c, 1, C.Noise(), 16, 0, 0))[0]
    assert abs(e["p_plus"] - np.cos(theta / 2) ** 2) < 1e-14


def test_bell_t_closed_form():
    """(|00>+|11>)/sqrt2, T on qubit 0, H x H, measure: P(00)=P(11)=(1+1/sqrt2)/4."""
    c = C.Circuit(2)
    c.gate(C.H, 0); c.gate(C.CX, 0, 1); c.gate(C.T, 0); c.gate(C.H, 0); c.gate(C.H, 1)
    c.measure(0); c.measure(1)
    for shot in range(8):
        ev = _meas_events(oracle.trace(c, 2, C.Noise(), 16, 5, shot))
        assert abs(ev[0]["p_plus"] - 0.5) < 1e-14
        x = 0 if ev[0]["outcome"] == 1 else 1
        p_same = (1 + 1 / np.sqrt(2)) / 2  # P(y = x | x)
        want = p_same if x == 0 else 1 - p_same
        assert abs(ev[1]["p_plus"] - want) < 1e-14


def _gs_dense(tr, n):
    return dense_ref.gs_to_dense(n, tr["rows_x"], tr["rows_z"], tr["rows_r"], tr["keys"], tr["vals"])


def test_t_tdag_is_identity():
    base = C.random_circuit(9, 4, 40, t_frac=0.3, meas_frac=0.0, rz=False, resets=False)
    base.ops = base.ops[:40]
    c = C.Circuit(4, list(base.ops))
    tr0 = oracle.trace(c, 4, C.Noise(), 1 << 12, 0, 0)
    c.gate(C.T, 2); c.gate(C.T_DAG, 2)
    tr1 = oracle.trace(c, 4, C.Noise(), 1 << 12, 0, 0)
    assert np.array_equal(tr0["keys"], tr1["keys"])
    assert np.allclose(tr0["vals"], tr1["vals"], atol=1e-15)


def test_t_squared_is_s_and_t8_is_identity():
    base = C.random_circuit(11, 3, 30, t_frac=0.2, meas_frac=0.0, rz=False, resets=False)
    base.ops = base.ops[:30]
    a = C.Circuit(3, list(base.ops)); a.gate(C.T, 1); a.gate(C.T, 1)
    b = C.Circuit(3, list(base.ops)); b.gate(C.S, 1)
    ta, tb = oracle.trace(a, 3, C.Noise(), 1 << 12, 0, 0), oracle.trace(b, 3, C.Noise(), 1 << 12, 0, 0)
    assert abs(abs(np.vdot(_gs_dense(ta, 3), _gs_dense(tb, 3))) - 1) < 1e-12
    c8 = C.Circuit(3, list(base.ops))
    t0 = oracle.trace(c8, 3, C.Noise(), 1 << 12, 0, 0)
    for _ in range(8):
        c8.gate(C.T, 0)
    t8 = oracle.trace(c8, 3, C.Noise(), 1 << 12, 0, 0)
    assert np.array_equal(t0["keys"], t8["keys"])
    assert np.allclose(t0["vals"], t8["vals"], atol=1e-14)


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("seed", range(5))
def test_norm_and_growth_bounds(seed):
    circ = C.random_circuit(300 + seed, 6, 150)
    noise = C.Noise.uniform(0.02)
    for shot in range(4):
        tr = oracle.trace(circ, 6, noise, circ.cap, seed, shot)
        prev = 1
        for e in tr["events"]:
            assert abs(e["norm"] - 1) < 1e-12
            assert e["nnz_before"] == prev  # Clifford gates and noise keep |v|
            if e["kind"] == 2:
                assert e["nnz_after"] <= 2 * e["nnz_before"]
            if e["kind"] == 3:
                assert e["nnz_after"] <= e["nnz_before"]
            prev = e["nnz_after"]


def test_windowed_noiseless_coset_bound_and_detectors():
    """Noiseless: every detector 0, no logical error, |v| <= 2^w (coset bound)."""
    for name in ("w42",):
        circ, _ = C.workload(name)
        w = 4
        for shot in range(3):
            tr = oracle.trace(circ, circ.n, C.Noise(), circ.cap, 0, shot)
            assert tr["status"] == 0 and tr["logical"] == 0
            assert int(tr["events"]["nnz_after"].max()) <= 2 ** w
            assert len(tr["keys"]) == 1
        r = oracle.run(circ, circ.n, C.Noise(), circ.cap, 0, 0, 16, threads=4)
        assert r["tally"] == [16, 0, 0, 16, 0]


def test_xz_words_are_shot_invariant():
    """The X/Z part of the tableau is the same in every shot (only signs and
    coefficients depend on noise and outcomes)."""
    circ = C.random_circuit(77, 5, 120)
    noise = C.Noise.uniform(0.05)
    trs = [oracle.trace(circ, 5, noise, circ.cap, 3, s) for s in range(10)]
    for tr in trs[1:]:
        assert np.array_equal(tr["rows_x"], trs[0]["rows_x"])
        assert np.array_equal(tr["rows_z"], trs[0]["rows_z"])
    assert len({tuple(t["rows_r"]) for t in trs}) > 1


# ------------------------------------------------------------------ exact distribution
def test_tiny_record_distribution_chi2():
    circ, noise = C.workload("tiny6")
    dist = dense_ref.record_distribution(circ, noise)
    assert abs(sum(dist.values()) - 1) < 1e-9
    N = 10000
    r = oracle.run(circ, circ.n, noise, circ.cap, 0, 0, N, threads=4)
    nrec = 9
    counts = {}
    for w in r["records"][:, 0]:
        bits = tuple((int(w) >> j) & 1 for j in range(nrec))
        counts[bits] = counts.get(bits, 0) + 1
    keys = sorted(dist, key=lambda k: -dist[k])
    big = [k for k in keys if dist[k] * N >= 5]
    obs = [counts.get(k, 0) for k in big] + [N - sum(counts.get(k, 0) for k in big)]
    exp = [dist[k] * N for k in big] + [N * (1 - sum(dist[k] for k in big))]
    if exp[-1] < 5:
        obs[-2] += obs[-1]; exp[-2] += exp[-1]; obs.pop(); exp.pop()
    chi2 = sum((o - e) ** 2 / e for o, e in zip(obs, exp))
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, len(obs) - 1) > 1e-4
    # none of the observed records is impossible
    assert all(k in dist for k in counts)


# ------------------------------------------------------------------ error paths
def test_overflow_status():
    c = C.Circuit(4)
    for q in range(4):
        c.gate(C.H, q); c.gate(C.T, q)
    r = oracle.run(c, 4, C.Noise(), 8, 0, 0, 3)
    assert list(r["status"]) == [oracle.ST_OVERFLOW] * 3
    r = oracle.run(c, 4, C.Noise(), 16, 0, 0, 3)
    assert list(r["status"]) == [oracle.ST_OK] * 3


def test_malformed_inputs_rejected():
    c = C.Circuit(2)
    c.gate(C.H, 5)
    with pytest.raises(RuntimeError):
        oracle.run(c, 2, C.Noise(), 16, 0, 0, 1)
    c = C.Circuit(2)
    c.detector([0])
    with pytest.raises(RuntimeError):
        oracle.run(c, 2, C.Noise(), 16, 0, 0, 1)


# ------------------------------------------------------------------ post-prefix work counters
def _counts(circ, noise, shots=300, seed=0):
    return oracle.run(circ, circ.n, noise, circ.cap, seed, 0, shots, threads=4, records=False)["counts"]


def test_post_prefix_counts_bounded_by_full():
    circ, noise = C.windowed(3, n_data=10, n_anc=2, blocks=4, w=3, n_cliff=16, checks=2, p=0.01)
    k = _counts(circ, noise)
    for a, b in (("post_t_out", "t_out_entries"), ("post_t_diag", "t_diag_entries"),
                 ("post_meas", "meas_entries"), ("post_noise", "noise_entries")):
        assert 0 < k[a] <= k[b]


def test_post_prefix_noiseless_counts_only_the_observed_chain_in_fidelity_mode():
    """Noiselessly every outcome of the windowed circuit is decided and the map
    stays <= 16: a sampled shot never leaves the prefix; in fidelity mode the
    final observed measurements are past it."""
    circ, _ = C.windowed(3, n_data=10, n_anc=2, blocks=4, w=3, n_cliff=16, checks=2, p=0.0)
    k = _counts(circ, C.Noise(), shots=20)
    assert k["post_t_out"] == k["post_t_diag"] == k["post_meas"] == k["post_noise"] == 0
    kf = oracle.run(circ, circ.n, C.Noise(), circ.cap, 0, 0, 20, threads=4, records=False, fidelity=True)["counts"]
    assert kf["post_t_out"] == 0 and kf["post_t_diag"] == 0 and kf["post_noise"] == 0
    n_final = 10  # one measurement per data qubit, one entry each
    assert kf["post_meas"] == 20 * n_final


def test_post_prefix_undecided_first_outcome_counts_everything():
    c = C.Circuit(3)
    c.gate(C.H, 0)
    c.measure(0)  # p_+ = 1/2: every shot differs from here on
    for q in range(3):
        c.gate(C.H, q)
        c.gate(C.T, q)
    c.measure(1)
    k = _counts(c, C.Noise(), shots=50)
    assert k["post_t_out"] == k["t_out_entries"] > 0 and k["post_meas"] == k["meas_entries"]
