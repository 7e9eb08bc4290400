"""Independent Aaronson-Gottesman (CHP-style) tableau sampler.

Used only to pin the oracle on Clifford-only circuits. Written from the
Aaronson-Gottesman algorithm (Phys. Rev. A 70, 052328): only H, S and CNOT
act on the tableau directly; every other Clifford is built from them
(S^dag = S S S, Z = S S, X = H Z H, Y = X Z, CZ = H_b CX H_b); products of
rows use the g-function phase rule; Z measurement follows the CHP procedure
(rowsum of every other row with x_a = 1 into the pivot, or a scratch row for
deterministic outcomes). Rows are Python ints.
"""
from __future__ import annotations

from paper_2512_23037_gb300 import circuits as C


def _g(x1, z1, x2, z2):
    if not x1 and not z1:
        return 0
    if x1 and z1:
        return z2 - x2
    if x1 and not z1:
        return z2 * (2 * x2 - 1)
    return x2 * (1 - 2 * z2)


class AG:
    def __init__(self, n):
        self.n = n
        # rows 0..n-1 destabilizers, n..2n-1 stabilizers, 2n scratch
        self.x = [0] * (2 * n + 1)
        self.z = [0] * (2 * n + 1)
        self.r = [0] * (2 * n + 1)
        for i in range(n):
            self.x[i] = 1 << i
            self.z[n + i] = 1 << i

    def _bit(self, v, q):
        return (v >> q) & 1

    def h(self, a):
        for i in range(2 * self.n):
            xa, za = self._bit(self.x[i], a), self._bit(self.z[i], a)
            self.r[i] ^= xa & za
            if xa != za:
                self.x[i] ^= 1 << a
                self.z[i] ^= 1 << a

    def s(self, a):
        for i in range(2 * self.n):
            xa, za = self._bit(self.x[i], a), self._bit(self.z[i], a)
            self.r[i] ^= xa & za
            if xa:
                self.z[i] ^= 1 << a

    def cx(self, a, b):
        for i in range(2 * self.n):
            xa, za = self._bit(self.x[i], a), self._bit(self.z[i], a)
            xb, zb = self._bit(self.x[i], b), self._bit(self.z[i], b)
            self.r[i] ^= xa & zb & (xb ^ za ^ 1)
            if xa:
                self.x[i] ^= 1 << b
            if zb:
                self.z[i] ^= 1 << a

    def gate(self, op, a, b=None):
        if op == C.H:
            self.h(a)
        elif op == C.S:
            self.s(a)
        elif op == C.S_DAG:
            self.s(a); self.s(a); self.s(a)
        elif op == C.Z:
            self.s(a); self.s(a)
        elif op == C.X:
            self.h(a); self.s(a); self.s(a); self.h(a)
        elif op == C.Y:
            self.gate(C.X, a); self.gate(C.Z, a)
        elif op == C.CX:
            self.cx(a, b)
        elif op == C.CZ:
            self.h(b); self.cx(a, b); self.h(b)
        else:
            raise ValueError(op)

    def pauli(self, code, a):
        """Conjugate by a Pauli: flip the sign of every row that anticommutes."""
        px = 1 if code in (1, 2) else 0
        pz = 1 if code in (2, 3) else 0
        for i in range(2 * self.n):
            xa, za = self._bit(self.x[i], a), self._bit(self.z[i], a)
            if (xa & pz) ^ (za & px):
                self.r[i] ^= 1

    def rowsum(self, h, i):
        tot = 2 * self.r[h] + 2 * self.r[i]
        for j in range(self.n):
            tot += _g(self._bit(self.x[i], j), self._bit(self.z[i], j), self._bit(self.x[h], j),
                      self._bit(self.z[h], j))
        tot %= 4
        assert tot in (0, 2)
        self.r[h] = 0 if tot == 0 else 1
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    def measure(self, a, u):
        """Z measurement; a random outcome is +1 iff u < 1/2. Returns (m, random?)."""
        n = self.n
        p = next((i for i in range(n, 2 * n) if self._bit(self.x[i], a)), None)
        if p is not None:
            for i in range(2 * n):
                # row p - n (the partner destabilizer) is overwritten just below
                if i != p and i != p - n and self._bit(self.x[i], a):
                    self.rowsum(i, p)
            self.x[p - n], self.z[p - n], self.r[p - n] = self.x[p], self.z[p], self.r[p]
            m = 1 if u < 0.5 else -1
            self.x[p], self.z[p], self.r[p] = 0, 1 << a, (0 if m == 1 else 1)
            return m, True
        s = 2 * n
        self.x[s], self.z[s], self.r[s] = 0, 0, 0
        for i in range(n):
            if self._bit(self.x[i], a):
                self.rowsum(s, i + n)
        return (1 if self.r[s] == 0 else -1), False

    def stabilizers(self):
        n = self.n
        return [(self.x[n + i], self.z[n + i], self.r[n + i]) for i in range(n)]


def _mul_rows(n, a, b):
    """Hermitian product of two commuting rows with the g-function rule."""
    (x1, z1, r1), (x2, z2, r2) = a, b
    tot = 2 * r1 + 2 * r2
    for j in range(n):
        tot += _g((x1 >> j) & 1, (z1 >> j) & 1, (x2 >> j) & 1, (z2 >> j) & 1)
    tot %= 4
    assert tot in (0, 2)
    return (x1 ^ x2, z1 ^ z2, 0 if tot == 0 else 1)


def canonical(n, rows):
    """Reduced row echelon form of a stabilizer generator list over the
    2n-bit (x|z) vectors, with signs carried by row products. Two lists
    generate the same signed group iff their canonical forms are equal."""
    rows = list(rows)
    out = []
    for col in range(2 * n):
        def bit(rw):
            return ((rw[0] >> col) & 1) if col < n else ((rw[1] >> (col - n)) & 1)
        p = next((i for i, rw in enumerate(rows) if bit(rw)), None)
        if p is None:
            continue
        piv = rows.pop(p)
        rows = [_mul_rows(n, rw, piv) if bit(rw) else rw for rw in rows]
        out = [_mul_rows(n, rw, piv) if bit(rw) else rw for rw in out]
        out.append(piv)
    assert not rows or all(rw[0] == 0 and rw[1] == 0 for rw in rows)
    return sorted(out)


def run(circ: C.Circuit, noise: C.Noise, events):
    """Replay a Clifford-only circuit with the oracle's error and u inputs."""
    from tests.dense_ref import site_layout
    layout = site_layout(circ.ops, noise)
    errs, us = {}, {}
    for e in events:
        if e["kind"] == 1:
            i, where = layout[int(e["a"])]
            errs[(i, where)] = int(e["b"])
        elif e["kind"] == 3:
            us[int(e["op_index"])] = float(e["u"])
    t = AG(circ.n)
    recs = []

    def err(i, where, o):
        code = errs.get((i, where))
        if code is None:
            return
        if o[0] in C.TWO_Q and where == "post":
            if code >> 2:
                t.pauli(code >> 2, o[2])
            if code & 3:
                t.pauli(code & 3, o[3])
        else:
            t.pauli(code, o[2])

    for i, o in enumerate(circ.ops):
        op, fl, q0, q1 = o[0], o[1], o[2], o[3]
        err(i, "pre", o)
        if op in C.CLIFFORD_1Q:
            t.gate(op, q0)
        elif op in C.TWO_Q:
            t.gate(op, q0, q1)
        elif op in (C.M, C.R, C.MR):
            m, _ = t.measure(q0, us[i])
            if op != C.R:
                recs.append(0 if m == 1 else 1)
            if op in (C.R, C.MR) and m == -1:
                t.pauli(1, q0)
        err(i, "post", o)
    return t, recs
