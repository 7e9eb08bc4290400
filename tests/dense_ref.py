"""Dense statevector / density-matrix references used to pin the oracle.

Written from the definitions only: gates are explicit matrices acting on a
2^n vector (qubit q = bit q of the basis index), Pauli errors are applied as
matrices, measurements project with (I +- Z_q)/2 and renormalise. Random
inputs (which error hit which site, the uniform u of every measurement) are
taken from the oracle's event log, so the two runs see the same randomness;
the arithmetic is this file's own.
"""
from __future__ import annotations

import numpy as np

from paper_2512_23037_gb300 import circuits as C

SQ = 1 / np.sqrt(2)
_M1 = {C.H: np.array([[SQ, SQ], [SQ, -SQ]], complex), C.S: np.diag([1, 1j]), C.S_DAG: np.diag([1, -1j]),
       C.X: np.array([[0, 1], [1, 0]], complex), C.Y: np.array([[0, -1j], [1j, 0]], complex),
       C.Z: np.diag([1, -1]).astype(complex), C.T: np.diag([1, np.exp(1j * np.pi / 4)]),
       C.T_DAG: np.diag([1, np.exp(-1j * np.pi / 4)])}
PAULI = [np.eye(2, dtype=complex), _M1[C.X], _M1[C.Y], _M1[C.Z]]


def one_q_matrix(op, angle=0.0):
    if op == C.RZ:
        return np.diag([np.exp(-0.5j * angle), np.exp(0.5j * angle)])
    return _M1[op]


def apply_1q(psi, n, q, U):
    t = psi.reshape([2] * n)  # axis k <-> qubit n-1-k
    ax = n - 1 - q
    t = np.moveaxis(np.tensordot(U, t, axes=([1], [ax])), 0, ax)
    return t.reshape(-1)


def apply_2q(psi, n, op, a, b):
    idx = np.arange(1 << n)
    ba = (idx >> a) & 1
    bb = (idx >> b) & 1
    out = psi.copy()
    if op == C.CX:
        src = idx ^ (ba << b)
        out = psi[src]
    elif op == C.CZ:
        out = psi * np.where((ba & bb) == 1, -1, 1)
    return out


def apply_pauli_code(psi, n, code, q):
    if code == 0:
        return psi
    return apply_1q(psi, n, q, PAULI[code])


def apply_pauli_terms(psi, n, terms):
    """prod of single-qubit Paulis [(code, qubit), ...] on distinct qubits."""
    for code, q in terms:
        psi = apply_1q(psi, n, q, PAULI[code])
    return psi


def mpp_first(circ_ops, i):
    o = circ_ops[i]
    if o[0] != C.MPP:
        return False
    return i == 0 or not (circ_ops[i - 1][0] == C.MPP and (circ_ops[i - 1][1] & C.MPP_MORE))


def site_layout(circ_ops, noise):
    """Noise sites of the uniform depolarizing model, numbered in op order:
    the flip before M/MR (and before the first op of an MPP chain), then the
    site after the op (depolarizing after a gate, flip after R/MR).
    Returns {site: (op_index, 'pre'|'post')}."""
    out = {}
    ns = 0
    noiseless = False
    p1, p2, pm, pr, _ = noise.as_tuple()
    for i, o in enumerate(circ_ops):
        op = o[0]
        if op == C.NOISELESS_BEGIN:
            noiseless = True
        elif op == C.NOISELESS_END:
            noiseless = False
        if noiseless:
            continue
        if (op in (C.M, C.MR) or mpp_first(circ_ops, i)) and pm > 0:
            out[ns] = (i, "pre")
            ns += 1
        if op in C.ONE_Q and p1 > 0:
            out[ns] = (i, "post")
            ns += 1
        elif op in C.TWO_Q and p2 > 0:
            out[ns] = (i, "post")
            ns += 1
        elif op in (C.R, C.MR) and pr > 0:
            out[ns] = (i, "post")
            ns += 1
    return out


def replay(circ: C.Circuit, noise: C.Noise, events, stop_after=None, band=1e-9):
    """Replay one shot densely with the oracle's random inputs.

    Returns dict(psi, records, status, logical, mismatches, p_err) where
    mismatches counts outcomes that differ while |p - u| > band and p_err is
    the largest |p_dense - p_oracle| seen."""
    n = circ.n
    ops = circ.ops if stop_after is None else circ.ops[:stop_after]
    layout = site_layout(circ.ops, noise)
    errs = {}
    meas = {}
    for e in events:
        if e["kind"] == 1:
            i, where = layout[int(e["a"])]
            assert i == int(e["op_index"])
            errs[(i, where)] = int(e["b"])
        elif e["kind"] == 3:
            meas[int(e["op_index"])] = (float(e["u"]), int(e["outcome"]), float(e["p_plus"]))
    psi = np.zeros(1 << n, complex)
    psi[0] = 1
    recs = []
    chain = 0
    status, logical, mism, p_err = 0, 0, 0, 0.0

    def err(i, where, o):
        nonlocal psi
        code = errs.get((i, where))
        if code is None:
            return
        if o[0] in C.TWO_Q and where == "post":
            psi = apply_pauli_code(psi, n, code >> 2, o[2])
            psi = apply_pauli_code(psi, n, code & 3, o[3])
        else:
            psi = apply_pauli_code(psi, n, code, o[2])

    for i, o in enumerate(ops):
        op, fl, q0, q1, _, ang, rec = o
        err(i, "pre", o)
        if op in C.ONE_Q:
            psi = apply_1q(psi, n, q0, one_q_matrix(op, ang))
        elif op in C.TWO_Q:
            psi = apply_2q(psi, n, op, q0, q1)
        elif op in (C.M, C.R, C.MR):
            idx = np.arange(1 << n)
            one = ((idx >> q0) & 1) == 1
            p1 = float(np.sum(np.abs(psi[one]) ** 2))
            tot = float(np.sum(np.abs(psi) ** 2))
            pp = (tot - p1) / tot
            if pp < 1e-12:
                pp = 0.0
            if pp > 1 - 1e-12:
                pp = 1.0
            u, m_or, p_or = meas[i]
            p_err = max(p_err, abs(pp - p_or))
            m = 1 if u < pp else -1
            if m != m_or:
                if abs(pp - u) > band:
                    mism += 1
                m = m_or  # follow the oracle's branch to keep comparing
            keep = ~one if m == 1 else one
            psi = np.where(keep, psi, 0)
            psi = psi / np.linalg.norm(psi)
            if op in (C.M, C.MR):
                recs.append(0 if m == 1 else 1)
            if op in (C.R, C.MR) and m == -1:
                psi = apply_1q(psi, n, q0, PAULI[1])
        elif op == C.MPP:
            if fl & C.MPP_MORE:
                err(i, "post", o)
                continue
            ppsi = apply_pauli_terms(psi, n, C.mpp_chain_terms(circ.ops, i))
            tot = float(np.sum(np.abs(psi) ** 2))
            pp = 0.5 * (1.0 + float(np.real(np.vdot(psi, ppsi))) / tot)
            if pp < 1e-12:
                pp = 0.0
            if pp > 1 - 1e-12:
                pp = 1.0
            u, m_or, p_or = meas[i]
            p_err = max(p_err, abs(pp - p_or))
            m = 1 if u < pp else -1
            if m != m_or:
                if abs(pp - u) > band:
                    mism += 1
                m = m_or
            psi = (psi + m * ppsi) / 2
            psi = psi / np.linalg.norm(psi)
            recs.append(0 if m == 1 else 1)
        elif op == C.CPAULI:
            par = 0
            for r in rec:
                if r >= 0:
                    par ^= recs[r]
            if par and (fl & 3):
                psi = apply_1q(psi, n, q0, PAULI[fl & 3])
        elif op in (C.DETECTOR, C.OBSERVABLE):
            par = chain
            for r in rec:
                if r >= 0:
                    par ^= recs[r]
            par ^= fl & C.FLAG_INVERT
            if fl & C.FLAG_CHAIN:
                chain = par
            else:
                chain = 0
                if op == C.DETECTOR and par:
                    status = 1
                    break
                if op == C.OBSERVABLE and par:
                    logical = 1
        err(i, "post", o)
    return {"psi": psi, "records": recs, "status": status, "logical": logical, "mismatches": mism,
            "p_err": p_err}


def pauli_row_apply(vec, n, x, z, r):
    """(-1)^r prod_k i^{x_k z_k} X^{x_k} Z^{z_k} applied to vec (x, z ints)."""
    idx = np.arange(1 << n)
    ph = ((-1) ** r) * (1j ** bin(x & z).count("1"))
    zs = np.array([(-1) ** bin(z & j).count("1") for j in range(1 << n)])
    out = np.zeros_like(vec)
    out[idx ^ x] = ph * zs * vec
    return out


def gs_to_dense(n, rows_x, rows_z, rows_r, keys, vals):
    """Expand (v, B(S, D)) to a dense vector: |psi_S> from prod (I + s_i)/2,
    then sum_a v_a d_a |psi_S>."""
    def word(a, i):
        return int(a[i][0]) | (int(a[i][1]) << 64)
    for j in range(1 << n):
        v = np.zeros(1 << n, complex)
        v[j] = 1
        for i in range(n):
            si = pauli_row_apply(v, n, word(rows_x, n + i), word(rows_z, n + i), int(rows_r[n + i]))
            v = (v + si) / 2
        if np.linalg.norm(v) > 1e-6:
            break
    psi_s = v / np.linalg.norm(v)
    out = np.zeros(1 << n, complex)
    for k, val in zip(keys, vals):
        alpha = int(k[0]) | (int(k[1]) << 64)
        b = psi_s.copy()
        for i in range(n):
            if (alpha >> i) & 1:
                b = pauli_row_apply(b, n, word(rows_x, i), word(rows_z, i), int(rows_r[i]))
        out += val * b
    return out


# ------------------------------------------------------------- density matrix
def _kraus_apply(rho, n, mats_and_weights):
    out = np.zeros_like(rho)
    for w, U in mats_and_weights:
        out += w * (U @ rho @ U.conj().T)
    return out


def _full_1q(n, q, U):
    out = np.array([[1]], complex)
    for k in reversed(range(n)):
        out = np.kron(out, U if k == q else np.eye(2))
    return out


def _full_2q(n, op, a, b):
    dim = 1 << n
    M = np.zeros((dim, dim), complex)
    e = np.eye(dim, dtype=complex)
    for j in range(dim):
        M[:, j] = apply_2q(e[:, j], n, op, a, b)
    return M


def record_distribution(circ: C.Circuit, noise: C.Noise):
    """Exact distribution of the record bits (dict bits-tuple -> prob) by a
    branching density-matrix run with exact noise channels. No detectors."""
    n = circ.n
    p1, p2, pm, pr, _ = noise.as_tuple()
    P1 = [_full_1q(n, 0, PAULI[0])]  # placeholder for shapes
    del P1
    branches = [((), np.zeros((1 << n, 1 << n), complex))]
    branches[0][1][0, 0] = 1
    noiseless = False
    for oi, o in enumerate(circ.ops):
        op, fl, q0, q1, _, ang, rec = o
        if op == C.NOISELESS_BEGIN:
            noiseless = True
            continue
        if op == C.NOISELESS_END:
            noiseless = False
            continue
        nb = []
        for bits, rho in branches:
            if op in (C.M, C.MR) and pm > 0 and not noiseless:
                Xq = _full_1q(n, q0, PAULI[1])
                rho = _kraus_apply(rho, n, [(1 - pm, np.eye(1 << n)), (pm, Xq)])
            if op == C.MPP and pm > 0 and not noiseless and mpp_first(circ.ops, oi):
                # the flip anticommutes with the chain's first factor
                Fq = _full_1q(n, q0, PAULI[3 if (fl & 3) == 1 else 1])
                rho = _kraus_apply(rho, n, [(1 - pm, np.eye(1 << n)), (pm, Fq)])
            if op in C.ONE_Q:
                U = _full_1q(n, q0, one_q_matrix(op, ang))
                rho = U @ rho @ U.conj().T
                if p1 > 0 and not noiseless:
                    ks = [(1 - p1, np.eye(1 << n))] + [(p1 / 3, _full_1q(n, q0, PAULI[k])) for k in (1, 2, 3)]
                    rho = _kraus_apply(rho, n, ks)
                nb.append((bits, rho))
            elif op in C.TWO_Q:
                U = _full_2q(n, op, q0, q1)
                rho = U @ rho @ U.conj().T
                if p2 > 0 and not noiseless:
                    ks = [(1 - p2, np.eye(1 << n))]
                    for a in range(4):
                        for b in range(4):
                            if a or b:
                                ks.append((p2 / 15, _full_1q(n, q0, PAULI[a]) @ _full_1q(n, q1, PAULI[b])))
                    rho = _kraus_apply(rho, n, ks)
                nb.append((bits, rho))
            elif op == C.M:
                idx = np.arange(1 << n)
                for m in (0, 1):
                    Pm = np.diag(((idx >> q0) & 1) == m).astype(complex)
                    r2 = Pm @ rho @ Pm
                    if np.real(np.trace(r2)) > 1e-15:
                        nb.append((bits + (m,), r2))
            elif op == C.MPP:
                if fl & C.MPP_MORE:
                    nb.append((bits, rho))
                    continue
                Pf = np.eye(1 << n, dtype=complex)
                for code, q in C.mpp_chain_terms(circ.ops, oi):
                    Pf = _full_1q(n, q, PAULI[code]) @ Pf
                for m in (0, 1):
                    Pm = (np.eye(1 << n) + (1 - 2 * m) * Pf) / 2
                    r2 = Pm @ rho @ Pm
                    if np.real(np.trace(r2)) > 1e-15:
                        nb.append((bits + (m,), r2))
            else:
                raise ValueError("record_distribution handles gates, M and MPP only")
        branches = nb
    return {bits: float(np.real(np.trace(rho))) for bits, rho in branches}


def project_pattern(circ: C.Circuit, noise: C.Noise, sites, codes, theta=None):
    """Dense projection run of one error pattern: detector measurements are
    projected onto their passing outcome, observable measurements onto 0,
    nothing is renormalised. Returns (n_acc, n_fid) or None when a reset is
    not deterministic."""
    n = circ.n
    layout = site_layout(circ.ops, noise)
    errs = {layout[int(s)]: int(k) for s, k in zip(sites, codes)}
    role, target = {}, {}
    chain = 0
    for o in circ.ops:
        op, fl, rec = o[0], o[1], o[6]
        if op == C.DETECTOR:
            single = rec[0] >= 0 and rec[1] < 0 and not (fl & C.FLAG_CHAIN) and not chain
            for r in rec:
                if r >= 0:
                    role[r] = 1 if single else 3
                    target[r] = fl & C.FLAG_INVERT
            chain = fl & C.FLAG_CHAIN
        elif op == C.OBSERVABLE:
            for r in rec:
                if r >= 0 and r not in role:
                    role[r] = 2
            chain = fl & C.FLAG_CHAIN
    psi = np.zeros(1 << n, complex)
    psi[0] = 1
    n_acc = None
    rec_i = 0
    bits = {}

    def err(i, where, o):
        nonlocal psi
        code = errs.get((i, where))
        if code is None:
            return
        if o[0] in C.TWO_Q and where == "post":
            psi = apply_pauli_code(psi, n, code >> 2, o[2])
            psi = apply_pauli_code(psi, n, code & 3, o[3])
        else:
            psi = apply_pauli_code(psi, n, code, o[2])

    idx = np.arange(1 << n)
    for i, o in enumerate(circ.ops):
        op, fl, q0, q1, prm, ang, rec = o
        err(i, "pre", o)
        if op in C.ONE_Q:
            if op == C.RZ and theta is not None and prm > 0:
                ang = (-1.0 if fl & 1 else 1.0) * theta[prm - 1]
            psi = apply_1q(psi, n, q0, one_q_matrix(op, ang))
        elif op in C.TWO_Q:
            psi = apply_2q(psi, n, op, q0, q1)
        elif op in (C.M, C.R, C.MR):
            one = ((idx >> q0) & 1) == 1
            if op == C.R:
                p1 = np.sum(np.abs(psi[one]) ** 2) / np.sum(np.abs(psi) ** 2)
                if 1e-12 < p1 < 1 - 1e-12:
                    return None
                bit = 1 if p1 > 0.5 else 0
            else:
                rl = role.get(rec_i, 0)
                if rl == 1:
                    bit = target[rec_i]
                elif rl == 2:
                    if n_acc is None:
                        n_acc = float(np.sum(np.abs(psi) ** 2))
                    bit = 0
                else:
                    return None
                psi = np.where(one if bit else ~one, psi, 0)
                bits[rec_i] = bit
                rec_i += 1
            if op in (C.R, C.MR) and bit == 1:
                psi = apply_1q(psi, n, q0, PAULI[1])
        elif op == C.MPP and not (fl & C.MPP_MORE):
            rl = role.get(rec_i, 0)
            if rl == 1:
                bit = target[rec_i]
            elif rl == 2:
                if n_acc is None:
                    n_acc = float(np.sum(np.abs(psi) ** 2))
                bit = 0
            else:
                return None
            ppsi = apply_pauli_terms(psi, n, C.mpp_chain_terms(circ.ops, i))
            psi = (psi + (1 - 2 * bit) * ppsi) / 2
            bits[rec_i] = bit
            rec_i += 1
        elif op == C.CPAULI:
            par = 0
            for r in rec:
                if r >= 0:
                    par ^= bits[r]
            if par and (fl & 3):
                psi = apply_1q(psi, n, q0, PAULI[fl & 3])
        err(i, "post", o)
    n_fid = float(np.sum(np.abs(psi) ** 2))
    return (n_fid if n_acc is None else n_acc), n_fid
