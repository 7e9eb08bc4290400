"""Seeded synthetic circuits and the circuit interchange format.

This module is the one input source shared by the CUDA path, the oracle and
the tests. It holds no step of the simulation method: it only writes op
lists. To build parity checks that are deterministic when noiseless it
propagates Pauli strings through Clifford gates with lookup tables derived
here from explicit 2x2 / 4x4 matrices (U P U^dagger), not from tableau rules.

Op record (32 bytes, little endian), shared with the C ABI:
  op u16, flags u16, q0 u32, q1 u32, param u32, angle f64, rec i32[2]
A parameterised RZ carries param = k + 1 and flags bit 0 = 1 for the angle
-theta_k (0 for +theta_k); its `angle` field holds the current value used by
plain runs, and gradient runs substitute the parameter vector.

Noise model (uniform depolarizing, Sec. III of arxiv 2512.23037): DEPOL1(p1)
after every one-qubit gate (T/T^dagger/Rz included), DEPOL2(p2) after every
two-qubit gate, an X flip with p_meas before every M/MR and with p_reset
after every R/MR; before an MPP chain the flip is the Pauli on the chain's
first qubit that anticommutes with its first factor (Z for X, X for Y and Z).
Ops between NOISELESS_BEGIN and NOISELESS_END carry none. Idle noise is not modelled (p_idle must be 0).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------- op codes
H, S, S_DAG, X, Y, Z, CX, CZ, T, T_DAG, RZ, M, R, MR, CPAULI, DETECTOR, OBSERVABLE, \
    NOISELESS_BEGIN, NOISELESS_END, MPP = range(20)
OP_NAMES = ["H", "S", "S_DAG", "X", "Y", "Z", "CX", "CZ", "T", "T_DAG", "RZ", "M", "R", "MR",
            "CPAULI", "DETECTOR", "OBSERVABLE", "NOISELESS_BEGIN", "NOISELESS_END", "MPP"]
FLAG_INVERT = 1
FLAG_CHAIN = 2
# MPP: flags bits 0-1 Pauli on q0 (1 X, 2 Y, 3 Z), bits 2-3 Pauli on q1 (0 none),
# MPP_MORE = the product continues in the next op; the chain's last op records.
MPP_MORE = 16
ONE_Q = (H, S, S_DAG, X, Y, Z, T, T_DAG, RZ)
TWO_Q = (CX, CZ)
CLIFFORD_1Q = (H, S, S_DAG, X, Y, Z)

OP_DTYPE = np.dtype([("op", "<u2"), ("flags", "<u2"), ("q0", "<u4"), ("q1", "<u4"),
                     ("pad", "<u4"), ("angle", "<f8"), ("rec", "<i4", (2,))])
assert OP_DTYPE.itemsize == 32


@dataclass
class Noise:
    p1: float = 0.0
    p2: float = 0.0
    p_meas: float = 0.0
    p_reset: float = 0.0
    p_idle: float = 0.0

    @staticmethod
    def uniform(p: float) -> "Noise":
        return Noise(p, p, p, p, 0.0)

    def as_tuple(self):
        return (float(self.p1), float(self.p2), float(self.p_meas), float(self.p_reset), float(self.p_idle))


@dataclass
class Circuit:
    """An op list under construction. `n` is the qubit count."""
    n: int
    ops: list = field(default_factory=list)
    n_records: int = 0
    cap: int = 256
    name: str = ""

    def _add(self, op, q0=0, q1=0, flags=0, angle=0.0, rec=(-1, -1)):
        self.ops.append((op, flags, q0, q1, 0, angle, (int(rec[0]), int(rec[1]))))

    def gate(self, op, *qs, angle=0.0, param=None, negate=False):
        if op in TWO_Q:
            self._add(op, qs[0], qs[1])
        elif param is not None:
            self.ops.append((op, 1 if negate else 0, qs[0], 0, int(param) + 1, float(angle), (-1, -1)))
        else:
            self._add(op, qs[0], angle=angle)

    def measure(self, q, reset=False) -> int:
        self._add(MR if reset else M, q)
        r = self.n_records
        self.n_records += 1
        return r

    def mpp(self, terms) -> int:
        """Measure the Pauli product of `terms` = [(pauli_code, qubit), ...]
        (codes 1 X, 2 Y, 3 Z; distinct qubits) as one record."""
        terms = list(terms)
        assert terms, "empty Pauli product"
        pairs = [terms[i:i + 2] for i in range(0, len(terms), 2)]
        for i, pr in enumerate(pairs):
            (pa, qa) = pr[0]
            pb, qb = pr[1] if len(pr) > 1 else (0, 0)
            fl = (pa & 3) | ((pb & 3) << 2) | (MPP_MORE if i < len(pairs) - 1 else 0)
            self._add(MPP, qa, qb, flags=fl)
        r = self.n_records
        self.n_records += 1
        return r

    def reset(self, q):
        self._add(R, q)

    def cpauli(self, q, pauli_code, recs):
        recs = list(recs) + [-1, -1]
        self._add(CPAULI, q, flags=pauli_code, rec=recs[:2])

    def parity_op(self, op, recs, invert=False):
        """DETECTOR / OBSERVABLE over any number of records (chained in pairs)."""
        recs = list(recs)
        if not recs:
            recs = [-1]
        chunks = [recs[i:i + 2] for i in range(0, len(recs), 2)]
        for i, ch in enumerate(chunks):
            last = i == len(chunks) - 1
            fl = (FLAG_INVERT if (invert and last) else 0) | (0 if last else FLAG_CHAIN)
            ch = ch + [-1] * (2 - len(ch))
            self._add(op, flags=fl, rec=ch)

    def detector(self, recs, invert=False):
        self.parity_op(DETECTOR, recs, invert)

    def observable(self, recs, invert=False):
        self.parity_op(OBSERVABLE, recs, invert)

    def noiseless(self, on: bool):
        self._add(NOISELESS_BEGIN if on else NOISELESS_END)

    def array(self) -> np.ndarray:
        a = np.zeros(len(self.ops), dtype=OP_DTYPE)
        for i, (op, fl, q0, q1, pad, ang, rec) in enumerate(self.ops):
            a[i] = (op, fl, q0, q1, pad, ang, rec)
        return a

    def prefix(self, k: int) -> "Circuit":
        c = Circuit(self.n, list(self.ops[:k]), 0, self.cap, self.name)
        c.n_records = sum(1 for o in c.ops if records_outcome(o))
        return c


def records_outcome(o) -> bool:
    """True for an op tuple that appends a record: M, MR, the last op of an MPP chain."""
    return o[0] in (M, MR) or (o[0] == MPP and not (o[1] & MPP_MORE))


def mpp_chain_terms(ops, i):
    """[(pauli_code, qubit), ...] of the MPP chain whose last op is ops[i]."""
    j = i
    while j > 0 and ops[j - 1][0] == MPP and (ops[j - 1][1] & MPP_MORE):
        j -= 1
    out = []
    for o in ops[j:i + 1]:
        out.append((o[1] & 3, o[2]))
        if (o[1] >> 2) & 3:
            out.append(((o[1] >> 2) & 3, o[3]))
    return out


# ------------------------------------------------ Pauli strings (generator only)
_PM = [np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], complex),
       np.array([[0, -1j], [1j, 0]], complex), np.array([[1, 0], [0, -1]], complex)]
_U1 = {H: np.array([[1, 1], [1, -1]], complex) / np.sqrt(2),
       S: np.diag([1, 1j]), S_DAG: np.diag([1, -1j]),
       X: _PM[1], Y: _PM[2], Z: _PM[3]}
_CXm = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex)  # control = first factor
_CZm = np.diag([1, 1, 1, -1]).astype(complex)
_PHASES = [1, 1j, -1, -1j]


def _match(mat, cands):
    for key, cm in cands:
        for e, ph in enumerate(_PHASES):
            if np.allclose(mat, ph * cm):
                return e, key
    raise AssertionError("not a Pauli")


_CONJ1 = {}
for _g, _u in _U1.items():
    for _p in range(4):
        _CONJ1[(_g, _p)] = _match(_u @ _PM[_p] @ _u.conj().T, [(k, _PM[k]) for k in range(4)])
_CONJ2 = {}
_two = [((a, b), np.kron(_PM[a], _PM[b])) for a in range(4) for b in range(4)]
for _g, _u in ((CX, _CXm), (CZ, _CZm)):
    for a in range(4):
        for b in range(4):
            _CONJ2[(_g, a, b)] = _match(_u @ np.kron(_PM[a], _PM[b]) @ _u.conj().T, _two)
_MUL = {}
for a in range(4):
    for b in range(4):
        _MUL[(a, b)] = _match(_PM[a] @ _PM[b], [(k, _PM[k]) for k in range(4)])


class PauliString:
    """i^e * tensor of per-qubit codes (0 I, 1 X, 2 Y, 3 Z)."""

    def __init__(self, codes, e=0):
        self.c = np.array(codes, dtype=np.int8)
        self.e = e % 4

    def copy(self):
        return PauliString(self.c.copy(), self.e)

    def conj_gate(self, op, q0, q1=None):
        """self <- U self U^dagger for one Clifford gate."""
        if op in TWO_Q:
            e, (a, b) = _CONJ2[(op, int(self.c[q0]), int(self.c[q1]))]
            self.c[q0], self.c[q1] = a, b
            self.e = (self.e + e) % 4
        elif op in _U1:
            e, p = _CONJ1[(op, int(self.c[q0]))]
            self.c[q0] = p
            self.e = (self.e + e) % 4
        else:
            raise ValueError(op)

    def mul(self, other):
        out = PauliString(np.zeros_like(self.c), self.e + other.e)
        for q in range(len(self.c)):
            e, p = _MUL[(int(self.c[q]), int(other.c[q]))]
            out.c[q] = p
            out.e = (out.e + e) % 4
        return out

    def sign(self):
        assert self.e in (0, 2), "not Hermitian"
        return 1 if self.e == 0 else -1


def _nullspace_gf2(mat: np.ndarray) -> list:
    """Basis of {x : mat @ x = 0 mod 2} for a (rows x cols) 0/1 matrix."""
    m = mat.copy().astype(np.uint8) % 2
    rows, cols = m.shape
    piv_cols, r = [], 0
    for c in range(cols):
        p = next((i for i in range(r, rows) if m[i, c]), None)
        if p is None:
            continue
        m[[r, p]] = m[[p, r]]
        for i in range(rows):
            if i != r and m[i, c]:
                m[i] ^= m[r]
        piv_cols.append(c)
        r += 1
        if r == rows:
            break
    free = [c for c in range(cols) if c not in piv_cols]
    basis = []
    for f in free:
        x = np.zeros(cols, dtype=np.uint8)
        x[f] = 1
        for i, pc in enumerate(piv_cols):
            x[pc] = m[i, f]
        basis.append(x)
    return basis


def _rank_gf2(vs) -> int:
    m = np.array(vs, dtype=np.uint8) % 2
    rank = 0
    rows, cols = m.shape
    for c in range(cols):
        p = next((i for i in range(rank, rows) if m[i, c]), None)
        if p is None:
            continue
        m[[rank, p]] = m[[p, rank]]
        for i in range(rows):
            if i != rank and m[i, c]:
                m[i] ^= m[rank]
        rank += 1
    return rank


def _inverse_op(op):
    return {S: S_DAG, S_DAG: S}.get(op, op)


# ---------------------------------------------------------------- generators
def random_layers(seed: int, n: int = 6, depth: int = 20, n_t: int = 4, n_mid: int = 3,
                  p: float = 1e-3) -> tuple:
    """Small random Clifford+T circuit (6-qubit tiny workload).

    Each of `depth` layers shuffles the qubits and pairs them; a pair gets CX
    or CZ with probability 1/2 (random orientation), otherwise each of its
    qubits gets H or S. `n_t` T/T^dagger (fair coin) sit at uniform random
    (layer, qubit) positions after that layer's gates; `n_mid` non-resetting
    Z measurements sit at random layer boundaries on random qubits; the
    circuit ends with M on every qubit.
    """
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"random_layers(n={n},depth={depth},seed={seed})", cap=256)
    tpos = set()
    while len(tpos) < n_t:
        tpos.add((int(rng.integers(depth)), int(rng.integers(n))))
    tkind = {pos: (T if rng.integers(2) == 0 else T_DAG) for pos in sorted(tpos)}
    mids = sorted((int(rng.integers(1, depth)), int(rng.integers(n))) for _ in range(n_mid))
    for layer in range(depth):
        for (lb, q) in mids:
            if lb == layer:
                c.measure(q)
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            a, b = int(perm[i]), int(perm[i + 1])
            if rng.random() < 0.5:
                c.gate(CX if rng.random() < 0.5 else CZ, a, b)
            else:
                c.gate(H if rng.random() < 0.5 else S, a)
                c.gate(H if rng.random() < 0.5 else S, b)
        if n % 2:
            q = int(perm[-1])
            c.gate(H if rng.random() < 0.5 else S, q)
        for q in range(n):
            if (layer, q) in tkind:
                c.gate(tkind[(layer, q)], q)
    for q in range(n):
        c.measure(q)
    return c, Noise.uniform(p)


def random_prep(rng, data: list, layers: int) -> list:
    """Gate list of a seeded random Clifford V on `data` (H/S layers + CX pairs)."""
    gates = []
    for _ in range(layers):
        for q in data:
            k = int(rng.integers(4))
            if k == 1:
                gates.append((H, q))
            elif k == 2:
                gates.append((S, q))
            elif k == 3:
                gates.append((H, q))
                gates.append((S, q))
        perm = rng.permutation(data)
        for i in range(0, len(perm) - 1, 2):
            gates.append((CX, int(perm[i]), int(perm[i + 1])))
    return gates


def windowed(seed: int, n_data: int = 38, n_anc: int = 4, blocks: int = 18, w: int = 4,
             n_cliff: int = 60, checks: int = 4, p: float = 1e-3, prep_layers: int = 2,
             check_terms: int = 2,
             cliff_two_q_frac: float = 2.0 / 3.0, cap: int | None = None,
             rz_angles=None) -> tuple:
    """Windowed Clifford+T workload (42-qubit / 97-qubit throughput circuits).

    psi0 = V|0> for a seeded random Clifford V (noiseless). Each block: T on a
    random w-subset W of the data; a random Clifford C of `n_cliff` gates from
    {CX, CZ, H}; `checks` ancilla-mediated measurements of P_k = C g_k C^dag
    with g_k random independent elements of Stab(psi0) having only I/Z on W
    (so they commute with the T layer and are +1 when noiseless), each with a
    DETECTOR; then C^-1 and T^dagger on W. Each g_k is the product of 1 to
    `check_terms` random vectors of a basis of that subgroup (a sparse random
    element, so checks stay low weight like colour-code checks). Finally V^-1 and Z measurement of
    every data qubit (noiseless), one OBSERVABLE per data qubit. Noiseless the
    circuit is the identity on the data and every detector reads 0.

    rz_angles: optional list of `blocks*w` angles; the T / T^dagger pair of
    position i becomes Rz(+theta_i) / Rz(-theta_i).
    """
    rng = np.random.default_rng(seed)
    n = n_data + n_anc
    if cap is None:
        cap = 4 ** w
    c = Circuit(n, name=f"windowed(n={n},blocks={blocks},w={w},seed={seed})", cap=cap)
    data = list(range(n_data))
    V = random_prep(rng, data, prep_layers)
    c.noiseless(True)
    for g in V:
        c.gate(*g)
    c.noiseless(False)
    # generators of Stab(psi0): V Z_i V^dag
    gens = []
    for i in data:
        ps = PauliString([0] * n)
        ps.c[i] = 3
        for g in V:
            ps.conj_gate(g[0], *g[1:])
        gens.append(ps)
    pos = 0
    for blk in range(blocks):
        W = sorted(int(q) for q in rng.choice(n_data, size=w, replace=False))
        angs = None
        if rz_angles is not None:
            angs = [float(rz_angles[pos + j]) for j in range(w)]
        pos += w
        for j, q in enumerate(W):
            if angs is None:
                c.gate(T, q)
            else:
                c.gate(RZ, q, angle=angs[j], param=pos - w + j)
        # random Clifford C from {CX, CZ, H}
        C = []
        for _ in range(n_cliff):
            if rng.random() < cliff_two_q_frac:
                a, b = (int(v) for v in rng.choice(n_data, size=2, replace=False))
                C.append((CX if rng.random() < 0.5 else CZ, a, b))
            else:
                C.append((H, int(rng.integers(n_data))))
        for g in C:
            c.gate(*g)
        # checks: combos of generators with no X/Y on the window
        xw = np.array([[1 if g.c[q] in (1, 2) else 0 for q in W] for g in gens], dtype=np.uint8)
        null = _nullspace_gf2(xw.T)  # combos x with sum_i x_i * xw[i] = 0
        chosen = []
        while len(chosen) < checks:
            pick = rng.choice(len(null), size=int(rng.integers(1, check_terms + 1)), replace=False)
            combo = np.zeros(len(gens), dtype=np.uint8)
            for k in pick:
                combo ^= null[int(k)]
            if _rank_gf2(chosen + [combo]) == len(chosen) + 1:
                chosen.append(combo)
        for k, combo in enumerate(chosen):
            gk = PauliString([0] * n)
            for i, b in enumerate(combo):
                if b:
                    gk = gk.mul(gens[i])
            assert all(gk.c[q] in (0, 3) for q in W)
            Pk = gk.copy()
            for g in C:
                Pk.conj_gate(g[0], *g[1:])
            anc = n_data + (k % n_anc)
            c.reset(anc)
            c.gate(H, anc)
            for q in range(n_data):
                code = int(Pk.c[q])
                if code == 1:
                    c.gate(CX, anc, q)
                elif code == 3:
                    c.gate(CZ, anc, q)
                elif code == 2:
                    c.gate(S_DAG, q)
                    c.gate(CX, anc, q)
                    c.gate(S, q)
            c.gate(H, anc)
            r = c.measure(anc)
            c.detector([r], invert=(Pk.sign() == -1))
        for g in reversed(C):
            c.gate(_inverse_op(g[0]), *g[1:])
        for j, q in enumerate(W):
            if angs is None:
                c.gate(T_DAG, q)
            else:
                c.gate(RZ, q, angle=-angs[j], param=pos - w + j, negate=True)
    c.noiseless(True)
    for g in reversed(V):
        c.gate(_inverse_op(g[0]), *g[1:])
    recs = [c.measure(q) for q in data]
    c.noiseless(False)
    for r in recs:
        c.observable([r])
    return c, Noise.uniform(p)


def rz_thetas(seed: int = 1, n: int = 72, sigma: float = 0.01):
    """theta_i = pi/4 + N(0, sigma) (the angles of the differentiation workload)."""
    rng = np.random.default_rng(seed)
    return np.pi / 4 + rng.normal(0.0, sigma, size=n)


def workload(name: str) -> tuple:
    """Named seeded workloads: 'tiny6' (6 qubits, 4 T, 3 mid-circuit M),
    'w42' (42 qubits, 18 windows of 4, cap 2^8, p=1e-3), 'w97' (97 qubits,
    24 windows of 6, cap 2^12, p=5e-4)."""
    if name == "tiny6":
        return random_layers(0)
    if name == "w42":
        return windowed(1)
    if name == "w42rz":  # every T / T^dag pair of w42 becomes Rz(+theta_i) / Rz(-theta_i)
        return windowed(1, rz_angles=rz_thetas(1, 72))
    if name == "w97":
        return windowed(4, n_data=89, n_anc=8, blocks=24, w=6, n_cliff=160, checks=8, p=5e-4,
                        cliff_two_q_frac=0.75)
    raise KeyError(name)


def batch_of_windowed(seed: int = 2, n_circuits: int = 64, mean_shots: float = 1e6):
    """Many windowed circuits for one batched launch (multi-circuit workload).

    Per circuit: qubits uniform in 17..49 (4 ancillas, the rest data), window
    w uniform in 2..6 (cap 4^w: 2^4..2^12), blocks uniform in 6..24, noise p
    log-uniform in [1e-4, 3e-3], shot count geometric with the given mean.
    Returns a list of (circuit, noise, n_shots)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_circuits):
        n = int(rng.integers(17, 50))
        w = int(rng.integers(2, 7))
        blocks = int(rng.integers(6, 25))
        p = float(np.exp(rng.uniform(np.log(1e-4), np.log(3e-3))))
        shots = int(rng.geometric(1.0 / mean_shots)) if mean_shots > 1 else 1
        circ, noise = windowed(1000 + k, n_data=n - 4, n_anc=4, blocks=blocks, w=w, n_cliff=max(20, 2 * (n - 4)),
                               checks=4, p=p)
        out.append((circ, noise, shots))
    return out


def random_param_circuit(seed: int, n: int, n_ops: int, n_params: int, n_checks: int = 3, p: float = 0.02):
    """Random circuit whose post-selected fidelity depends on every parameter:
    H on all qubits, then a mix of Clifford gates and parameterised Rz gates
    (random parameter, random sign), non-resetting mid-circuit Z measurements
    each with a detector (random expected parity), and finally Z measurement of
    every qubit with one observable each (the fidelity measurements)."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"random_param_circuit(n={n},ops={n_ops},seed={seed})", cap=256)
    for q in range(n):
        c.gate(H, q)
    checks_at = set(int(v) for v in rng.choice(np.arange(n_ops // 3, n_ops), size=n_checks, replace=False))
    for i in range(n_ops):
        if i in checks_at:
            r = c.measure(int(rng.integers(n)))
            c.detector([r], invert=bool(rng.integers(2)))
        u = rng.random()
        if u < 0.35:
            k = int(rng.integers(n_params))
            neg = bool(rng.integers(2))
            c.gate(RZ, int(rng.integers(n)), angle=0.0, param=k, negate=neg)
        elif u < 0.65 and n >= 2:
            a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
            c.gate(CX if rng.random() < 0.5 else CZ, a, b)
        else:
            c.gate(CLIFFORD_1Q[int(rng.integers(6))], int(rng.integers(n)))
    for q in range(n):
        c.gate(H, q)
    c.noiseless(True)
    recs = [c.measure(q) for q in range(n)]
    c.noiseless(False)
    for r in recs:
        c.observable([r])
    return c, Noise.uniform(p)


def random_circuit(seed: int, n: int, n_ops: int, t_frac=0.15, meas_frac=0.1, rz=True,
                   resets=True, feedback=True, detectors=False, mpp_frac=0.0) -> Circuit:
    """Random op mix over every op kind, for differential tests on small n.
    mpp_frac > 0 adds Pauli-product measurements of weight 1..4."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"random_circuit(n={n},ops={n_ops},seed={seed})", cap=1 << 16)
    for _ in range(n_ops):
        u = rng.random()
        if u < t_frac:
            k = int(rng.integers(3 if rz else 2))
            q = int(rng.integers(n))
            if k == 0:
                c.gate(T, q)
            elif k == 1:
                c.gate(T_DAG, q)
            else:
                c.gate(RZ, q, angle=float(rng.uniform(-np.pi, np.pi)))
        elif u < t_frac + meas_frac:
            q = int(rng.integers(n))
            k = int(rng.integers(3 if resets else 1))
            if k == 0:
                c.measure(q)
            elif k == 1:
                c.reset(q)
            else:
                c.measure(q, reset=True)
        elif u < t_frac + meas_frac + mpp_frac:
            w = int(rng.integers(1, min(4, n) + 1))
            qs = [int(v) for v in rng.choice(n, size=w, replace=False)]
            c.mpp([(int(rng.integers(1, 4)), q) for q in qs])
        elif feedback and u < t_frac + meas_frac + mpp_frac + 0.03 and c.n_records > 0:
            recs = [int(rng.integers(c.n_records))]
            if rng.random() < 0.5:
                recs.append(int(rng.integers(c.n_records)))
            c.cpauli(int(rng.integers(n)), int(rng.integers(1, 4)), recs)
        elif detectors and u < t_frac + meas_frac + mpp_frac + 0.05 and c.n_records > 0:
            recs = [int(rng.integers(c.n_records)) for _ in range(int(rng.integers(1, 4)))]
            c.observable(recs, invert=bool(rng.integers(2)))
        else:
            if n >= 2 and rng.random() < 0.4:
                a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
                c.gate(CX if rng.random() < 0.5 else CZ, a, b)
            else:
                c.gate(CLIFFORD_1Q[int(rng.integers(6))], int(rng.integers(n)))
    for q in range(n):
        c.measure(q)
    return c


def all_combos(n):
    return list(itertools.product(range(4), repeat=n))
