"""Pins of the oracle's noise stream and measurement uniforms (CPU only).

The stream (Philox4x32-10, counter (shot_lo, shot_hi, stream, index), key =
seed) decides which noise sites of a shot carry an error. Its sequencing is
pinned here against probability theory and against the stream's published
definition evaluated independently:

  - every site's error marginal equals its own p (binomial, 5 sigma), also on
    mixed-p circuits where sites below the largest p are thinned;
  - the joint of two sites (adjacent ones included) equals p_a p_b: errors at
    distinct sites are independent;
  - depolarizing Pauli choices are uniform over 3 (one qubit) and 15 (two
    qubits) (chi^2), and flip sites apply their one Pauli;
  - the full error list of a few shots equals one computed here from Philox
    blocks with the inverse CDF of the geometric gap (a closed form, not the
    threshold table the oracle searches);
  - the measurement uniform u = ((w0 << 21) xor (w1 >> 11)) 2^-53 of one
    (seed, shot, j), from its Philox block (the generator is pinned by the
    published known-answer vectors in tests/golden).

A mis-sequenced stream (the next site one too far, the two words of U
swapped, the thinning or Pauli words exchanged) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_23037_gb300 import circuits as C

N_SHOTS = 40000


def _mixed_circuit(n_rounds=20):
    """Each round: H on q0 (one-qubit depolarizing site), CX q0 q1 (two-qubit
    site), M q1 (a flip site before the measurement): 3 sites per round, in
    op order (the flip site of M comes before it, gate sites after the gate)."""
    c = C.Circuit(2)
    for _ in range(n_rounds):
        c.gate(C.H, 0)
        c.gate(C.CX, 0, 1)
        c.measure(1)
    return c


def _site_probs(noise, n_rounds):
    return np.array([noise.p1, noise.p2, noise.p_meas] * n_rounds)


def _error_matrix(circ, noise, seed, n_shots):
    """(n_shots, n_sites) 0/1 error indicators and the per-error codes by site."""
    ns, _ = oracle.count_sites(circ, circ.n, noise)
    hits = np.zeros((n_shots, ns), dtype=np.uint8)
    codes = [[] for _ in range(ns)]
    for s in range(n_shots):
        sites, cds = oracle.errors(circ, circ.n, noise, seed, s)
        for st, cd in zip(sites, cds):
            hits[s, st] = 1
            codes[st].append(int(cd))
    return hits, codes


@pytest.fixture(scope="module")
def mixed():
    circ = _mixed_circuit(20)
    noise = C.Noise(p1=0.2, p2=0.12, p_meas=0.05)
    hits, codes = _error_matrix(circ, noise, 11, N_SHOTS)
    return circ, noise, hits, codes


def test_site_count_and_order(mixed):
    circ, noise, hits, _ = mixed
    assert hits.shape[1] == 60 == len(_site_probs(noise, 20))


def test_every_site_marginal_equals_its_p(mixed):
    """Per site: P(error) = p_s within 5 binomial sigma, for the largest p
    (no thinning) and the two thinned rates."""
    _, noise, hits, _ = mixed
    p = _site_probs(noise, 20)
    freq = hits.mean(axis=0)
    sig = np.sqrt(p * (1 - p) / N_SHOTS)
    assert np.all(np.abs(freq - p) <= 5 * sig), np.max(np.abs(freq - p) / sig)


def test_pairwise_joints_are_products(mixed):
    """Errors at two sites are independent: P(both) = p_a p_b, for adjacent
    sites (a next site one too far makes adjacent pairs impossible), sites two
    apart and distant ones."""
    _, noise, hits, _ = mixed
    p = _site_probs(noise, 20)
    for a, b in [(0, 1), (1, 2), (2, 3), (3, 4), (9, 10), (0, 2), (12, 14), (5, 40), (0, 59)]:
        both = np.mean(hits[:, a] & hits[:, b])
        want = p[a] * p[b]
        sig = math.sqrt(want * (1 - want) / N_SHOTS)
        assert abs(both - want) <= 5 * sig, (a, b, both, want)


def _chi2_uniform(counts):
    counts = np.asarray(counts, dtype=float)
    exp = counts.sum() / len(counts)
    return float(np.sum((counts - exp) ** 2 / exp))


def test_pauli_choices_uniform(mixed):
    """DEPOL1 sites: codes 1..3 (X, Y, Z) uniform; DEPOL2: codes 1..15
    uniform; flip sites before M: always X (code 1)."""
    _, _, _, codes = mixed
    c1 = [c for s in range(0, 60, 3) for c in codes[s]]
    c2 = [c for s in range(1, 60, 3) for c in codes[s]]
    cf = [c for s in range(2, 60, 3) for c in codes[s]]
    h1 = np.bincount(c1, minlength=4)[1:4]
    h2 = np.bincount(c2, minlength=16)[1:16]
    assert len(c1) == h1.sum() and len(c2) == h2.sum()
    # chi^2 critical values at 1e-4: 18.42 (2 dof), 42.58 (14 dof)
    assert _chi2_uniform(h1) < 18.42, h1
    assert _chi2_uniform(h2) < 42.58, h2
    assert set(cf) == {1}


def _expected_errors(seed, shot, site_p):
    """The error list of one shot from the stream's definition: block k of
    stream 0 gives U = w0 + 2^32 w1; the gap to the next error is the smallest
    g with U < floor(2^64 (1 - (1 - p_max)^(g+1))), here by the inverse CDF
    g = floor(log(1 - U 2^-64) / log(1 - p_max)); a site with p_s < p_max keeps
    the error iff w3 < floor(2^32 p_s / p_max); the Pauli choice is
    floor(w2 K / 2^32) + 1 with K = 3 (one qubit) or 15 (two qubits)."""
    pmax = max(site_p)
    n = len(site_p)
    cur, k, out = 0, 0, []
    while cur < n:
        w = oracle.philox([shot & 0xFFFFFFFF, shot >> 32, 0, k], [seed & 0xFFFFFFFF, seed >> 32])
        k += 1
        U = w[0] + (w[1] << 32)
        x = math.log1p(-U / 2.0 ** 64) / math.log1p(-pmax)
        g = math.floor(x)
        if cur + g >= n:
            break
        s = cur + g
        cur = s + 1
        if site_p[s] < pmax and not (w[3] < math.floor(site_p[s] / pmax * 2.0 ** 32)):
            continue
        out.append((s, w[2]))
    return out


@pytest.mark.parametrize("shot", [0, 1, 7, 123456, (1 << 40) + 3])
def test_error_list_matches_stream_definition(shot):
    circ = _mixed_circuit(20)
    noise = C.Noise(p1=0.2, p2=0.12, p_meas=0.05)
    site_p = list(_site_probs(noise, 20))
    seed = 0x0123456789ABCDEF
    sites, codes = oracle.errors(circ, circ.n, noise, seed, shot)
    want = _expected_errors(seed, shot, site_p)
    assert [int(s) for s in sites] == [s for s, _ in want]
    for (s, w2), code in zip(want, codes):
        kind = s % 3
        if kind == 0:
            assert code == ((w2 * 3) >> 32) + 1
        elif kind == 1:
            assert code == ((w2 * 15) >> 32) + 1
        else:
            assert code == 1


def test_uniform53_fixed_value():
    """u of (seed, shot, j) from its Philox block of stream 1."""
    seed, shot, j = 0xDEADBEEF12345678, (1 << 33) + 5, 17
    w = oracle.philox([shot & 0xFFFFFFFF, shot >> 32, 1, j], [seed & 0xFFFFFFFF, seed >> 32])
    m = ((w[0] << 21) ^ (w[1] >> 11)) & ((1 << 53) - 1)
    assert oracle.uniform53(seed, shot, j) == m / 2.0 ** 53
    # the two words enter in this order: swapping them gives another value
    m_sw = ((w[1] << 21) ^ (w[0] >> 11)) & ((1 << 53) - 1)
    assert m_sw != m
