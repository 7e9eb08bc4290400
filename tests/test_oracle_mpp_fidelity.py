"""Pins of the oracle's Pauli-product measurement (MPP), measurement/reset
flip sites and exact-fidelity mode, against dense statevectors, exact
density-matrix distributions, closed forms and the sampled logical-error rate.

Fidelity mode: every measurement whose record an OBSERVABLE reads is
projected onto +1; F = product of their conditional probabilities p_+ equals
|<0..0| phi>|^2 on the observed qubits (the Born rule chained over the final
measurements), so E[1 - F | kept] is the logical-error rate of the sampled
mode (the variance reduction for rare logical errors of Sec. V).
"""
import numpy as np
import pytest

import oracle
from paper_2512_23037_gb300 import circuits as C
from tests import dense_ref


def _bits(r, nrec):
    return np.array([[(int(w[j // 64]) >> (j % 64)) & 1 for j in range(nrec)] for w in r["records"]])


# ------------------------------------------------------------------ flip sites
def test_measurement_flip_is_x():
    """p_meas = 0.3 before M on |0>: P(record 1) = 0.3 for an X flip (a
    uniformly drawn X/Y/Z would give 0.2)."""
    c = C.Circuit(1)
    c.measure(0)
    N = 40000
    r = oracle.run(c, 1, C.Noise(p_meas=0.3), 4, 5, 0, N, threads=4)
    f = _bits(r, 1)[:, 0].mean()
    assert abs(f - 0.3) < 5 * np.sqrt(0.21 / N), f


def test_reset_flip_is_x():
    c = C.Circuit(1)
    c.gate(C.H, 0)
    c.reset(0)
    c.measure(0)
    N = 40000
    r = oracle.run(c, 1, C.Noise(p_reset=0.25), 4, 6, 0, N, threads=4)
    f = _bits(r, 1)[:, 0].mean()
    assert abs(f - 0.25) < 5 * np.sqrt(0.1875 / N), f


@pytest.mark.parametrize("first", [1, 2, 3])
def test_mpp_flip_anticommutes_with_first_factor(first):
    """The flip before an MPP chain flips its outcome: on the +1 eigenstate of
    P = (first)_0 Z_1, P(record 1) = p_meas."""
    c = C.Circuit(2)
    if first == 1:
        c.gate(C.H, 0)  # |+>
    elif first == 2:
        c.gate(C.H, 0)
        c.gate(C.S, 0)  # |+i>
    c.mpp([(first, 0), (3, 1)])
    N = 40000
    r = oracle.run(c, 2, C.Noise(p_meas=0.2), 4, 7, 0, N, threads=4)
    f = _bits(r, 1)[:, 0].mean()
    assert abs(f - 0.2) < 5 * np.sqrt(0.16 / N), f


# ------------------------------------------------------------------ MPP closed forms
def _single_record(c, seed=0, shots=64):
    r = oracle.run(c, c.n, C.Noise(), 16, seed, 0, shots)
    return _bits(r, c.n_records)


def test_mpp_bell_and_ghz_eigenvalues():
    c = C.Circuit(3)
    c.gate(C.H, 0)
    c.gate(C.CX, 0, 1)
    rx = c.mpp([(1, 0), (1, 1)])   # XX |Phi+> = +|Phi+>
    rz = c.mpp([(3, 0), (3, 1)])   # ZZ = +1
    ry = c.mpp([(2, 0), (2, 1)])   # YY = -1
    c.gate(C.CX, 1, 2)              # GHZ on 3
    rg = c.mpp([(1, 0), (1, 1), (1, 2)])  # XXX = +1
    ryy = c.mpp([(2, 0), (2, 1), (1, 2)])  # YYX = -1
    b = _single_record(c)
    assert (b[:, rx] == 0).all() and (b[:, rz] == 0).all() and (b[:, ry] == 1).all()
    assert (b[:, rg] == 0).all() and (b[:, ryy] == 1).all()


def test_mpp_single_z_equals_m():
    """A one-factor Z product is the Z measurement: identical records and final state."""
    base = C.random_circuit(3, 4, 50)
    alt = C.Circuit(base.n, cap=base.cap)
    for o in base.ops:
        if o[0] == C.M:
            alt.mpp([(3, o[2])])
        else:
            alt.ops.append(o)
            if C.records_outcome(o):
                alt.n_records += 1
    nz = C.Noise(0.02, 0.02, 0.0, 0.02)
    for shot in range(8):
        a = oracle.trace(base, 4, nz, base.cap, 9, shot)
        b = oracle.trace(alt, 4, nz, alt.cap, 9, shot)
        assert np.array_equal(a["records"], b["records"])
        assert np.array_equal(a["rows_x"], b["rows_x"]) and np.array_equal(a["rows_r"], b["rows_r"])
        assert np.array_equal(a["keys"], b["keys"]) and np.allclose(a["vals"], b["vals"], atol=1e-15)


def test_mpp_x_on_zero_is_fair():
    c = C.Circuit(1)
    c.mpp([(1, 0)])
    N = 20000
    r = oracle.run(c, 1, C.Noise(), 4, 3, 0, N, threads=4)
    f = _bits(r, 1)[:, 0].mean()
    assert abs(f - 0.5) < 5 * np.sqrt(0.25 / N)


# ------------------------------------------------------------------ MPP vs dense
@pytest.mark.parametrize("seed", range(10))
def test_mpp_dense_replay_random_circuits(seed):
    n = 3 + seed % 4
    circ = C.random_circuit(300 + seed, n, 50 + 10 * n, mpp_frac=0.12, detectors=(seed % 2 == 0))
    noise = C.Noise(0.03, 0.03, 0.03, 0.02)
    for shot in range(6):
        tr = oracle.trace(circ, n, noise, circ.cap, 40 + seed, shot)
        rep = dense_ref.replay(circ, noise, tr["events"])
        assert rep["mismatches"] == 0
        assert rep["p_err"] < 1e-10
        assert rep["status"] == tr["status"]
        if tr["status"] == 0:
            gs = dense_ref.gs_to_dense(n, tr["rows_x"], tr["rows_z"], tr["rows_r"], tr["keys"], tr["vals"])
            assert abs(abs(np.vdot(rep["psi"], gs)) - 1) < 1e-10
            bits = [(int(tr["records"][r // 64]) >> (r % 64)) & 1 for r in range(len(rep["records"]))]
            assert bits == rep["records"]


def test_mpp_record_distribution_chi2():
    """Exact record distribution (density matrix, exact channels incl. the MPP flip) vs sampled."""
    rng = np.random.default_rng(4)
    c = C.Circuit(4)
    for layer in range(5):
        for q in range(4):
            c.gate([C.H, C.S, C.T, C.T_DAG][int(rng.integers(4))], q)
        c.gate(C.CX, layer % 4, (layer + 1) % 4)
        c.mpp([(int(rng.integers(1, 4)), q) for q in rng.choice(4, size=2 + layer % 2, replace=False)])
    c.measure(0)
    noise = C.Noise(0.02, 0.02, 0.05, 0.0)
    dist = dense_ref.record_distribution(c, noise)
    assert abs(sum(dist.values()) - 1) < 1e-9
    N = 20000
    r = oracle.run(c, 4, noise, 64, 11, 0, N, threads=4)
    b = _bits(r, c.n_records)
    counts = {}
    for row in b:
        counts[tuple(int(v) for v in row)] = counts.get(tuple(int(v) for v in row), 0) + 1
    big = [k for k in dist if dist[k] * N >= 5]
    obs = [counts.get(k, 0) for k in big] + [N - sum(counts.get(k, 0) for k in big)]
    exp = [dist[k] * N for k in big] + [N * (1 - sum(dist[k] for k in big))]
    if exp[-1] < 5:
        obs[-2] += obs[-1]; exp[-2] += exp[-1]; obs.pop(); exp.pop()
    chi2 = sum((o - e) ** 2 / e for o, e in zip(obs, exp))
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, len(obs) - 1) > 1e-4
    assert all(k in dist for k in counts)


def test_mpp_malformed_chains_rejected():
    c = C.Circuit(3)
    c.mpp([(1, 0), (3, 0)])  # repeated qubit
    with pytest.raises(RuntimeError):
        oracle.run(c, 3, C.Noise(), 8, 0, 0, 1)
    c = C.Circuit(3)
    c.mpp([(1, 0), (3, 1), (2, 2)])
    c.ops[-1] = (C.MPP, c.ops[-1][1] | C.MPP_MORE) + tuple(c.ops[-1][2:])  # chain left open
    with pytest.raises(RuntimeError):
        oracle.run(c, 3, C.Noise(), 8, 0, 0, 1)


# ------------------------------------------------------------------ fidelity mode
def _hth(n_q, ops_per_q):
    c = C.Circuit(n_q)
    for q, (op, ang) in enumerate(ops_per_q):
        c.gate(C.H, q)
        c.gate(op, q, angle=ang)
        c.gate(C.H, q)
    recs = [c.measure(q) for q in range(n_q)]
    for r in recs:
        c.observable([r])
    return c


@pytest.mark.parametrize("theta", [0.3, 1.1, -2.0])
def test_fidelity_closed_forms(theta):
    c = _hth(1, [(C.T, 0.0)])
    r = oracle.run(c, 1, C.Noise(), 8, 0, 0, 16, fidelity=True)
    assert np.allclose(r["fid"], np.cos(np.pi / 8) ** 2, atol=1e-14, rtol=0)
    c = _hth(2, [(C.RZ, theta), (C.T_DAG, 0.0)])
    r = oracle.run(c, 2, C.Noise(), 8, 0, 0, 16, fidelity=True)
    want = np.cos(theta / 2) ** 2 * np.cos(np.pi / 8) ** 2
    assert np.allclose(r["fid"], want, atol=1e-14, rtol=0)
    assert r["tally"][4] == 0 and r["fsum"][1] == 16


def test_fidelity_zero_branch():
    """X then M then OBSERVABLE: the +1 outcome is impossible, F = 0."""
    c = C.Circuit(1)
    c.gate(C.X, 0)
    c.observable([c.measure(0)])
    r = oracle.run(c, 1, C.Noise(), 8, 0, 0, 4, fidelity=True)
    assert np.all(r["fid"] == 0.0) and r["tally"][3] == 4


def test_fidelity_noiseless_windowed_is_one():
    circ, _ = C.windowed(2, n_data=8, n_anc=2, blocks=3, w=3, n_cliff=14, checks=2, p=0.0)
    r = oracle.run(circ, circ.n, C.Noise(), circ.cap, 0, 0, 50, fidelity=True)
    assert r["tally"][3] == 50 and np.all(r["fid"] == 1.0)


def _first_observed_op(circ):
    obs = set()
    for o in circ.ops:
        if o[0] == C.OBSERVABLE:
            obs.update(r for r in o[6] if r >= 0)
    rec = 0
    for i, o in enumerate(circ.ops):
        if C.records_outcome(o):
            if rec in obs:
                return i, obs
            rec += 1
    return None, obs


@pytest.mark.parametrize("seed", range(3))
def test_fidelity_matches_dense_overlap(seed):
    """F per kept shot = sum over basis states with every observed qubit 0 of
    |psi|^2, psi the dense state just before the (noiseless Z) final chain."""
    circ, noise = C.windowed(10 + seed, n_data=7, n_anc=2, blocks=3, w=3, n_cliff=12, checks=2, p=0.004)
    k, _ = _first_observed_op(circ)
    data_q = [o[2] for o in circ.ops[k:] if o[0] == C.M]
    N = 40
    r = oracle.run(circ, circ.n, noise, circ.cap, 3, 0, N, fidelity=True)
    idx = np.arange(1 << circ.n)
    mask = np.ones(1 << circ.n, bool)
    for q in data_q:
        mask &= ((idx >> q) & 1) == 0
    checked = nontrivial = 0
    for shot in range(N):
        if r["status"][shot] != 0:
            continue
        tr = oracle.trace(circ, circ.n, noise, circ.cap, 3, shot, stop_after=k)
        rep = dense_ref.replay(circ, noise, tr["events"], stop_after=k)
        psi = rep["psi"] / np.linalg.norm(rep["psi"])
        f_dense = float(np.sum(np.abs(psi[mask]) ** 2))
        assert abs(r["fid"][shot] - f_dense) < 1e-10, (shot, r["fid"][shot], f_dense)
        checked += 1
        nontrivial += f_dense < 1 - 1e-6
    assert checked >= 10 and nontrivial >= 1


def test_fidelity_estimator_matches_sampled_ler():
    """Same shots in both modes: identical statuses; 1 - mean F within the
    binomial interval of the sampled logical-error rate."""
    circ, noise = C.windowed(5, n_data=10, n_anc=2, blocks=4, w=3, n_cliff=16, checks=2, p=0.01)
    N = 6000
    a = oracle.run(circ, circ.n, noise, circ.cap, 8, 0, N, threads=8)
    b = oracle.run(circ, circ.n, noise, circ.cap, 8, 0, N, threads=8, fidelity=True)
    assert np.array_equal(a["status"], b["status"])
    kept = a["tally"][3]
    assert b["fsum"][1] == kept and kept > 1000
    ler = a["tally"][4] / kept
    est = 1 - b["fsum"][0] / kept
    sd = np.sqrt(max(ler * (1 - ler), 1e-4) / kept)
    assert abs(ler - est) < 5 * sd, (ler, est)
    assert est > 0


def test_fidelity_rejects_detector_after_chain():
    c = C.Circuit(2)
    r0 = c.measure(0)
    c.observable([r0])
    c.detector([c.measure(1)])
    with pytest.raises(RuntimeError):
        oracle.run(c, 2, C.Noise(), 8, 0, 0, 2, fidelity=True)
    oracle.run(c, 2, C.Noise(), 8, 0, 0, 2)  # sampling mode accepts it
