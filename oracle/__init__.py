"""FP64 CPU oracle of the generalized-stabilizer shot simulator (ctypes binding).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may use it; the product path never does. It
shares no code with the CUDA path; circuits arrive as arrays of 32-byte op
records (the public interchange format).

Pins (tests/test_oracle_*.py): Philox known-answer vectors; Clifford rules
against dense 2x2/4x4 conjugation; shot-by-shot dense statevector replay of
random Clifford+T+measurement circuits (<= 8 qubits); Clifford-only circuits
against an independent Aaronson-Gottesman sampler; closed-form outcome
probabilities of single-T circuits; T.T^dag = I, T^2 = S, T^8 = I;
normalisation and the |v| bounds of Theorem 1; exact record distribution
of the 6-qubit workload from a density-matrix run; the noise stream's
sequencing (per-site marginals, pairwise joints, Pauli-choice frequencies,
thinning, and error lists recomputed from Philox blocks by the geometric
gap's inverse CDF) and the measurement uniform's construction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "soft_oracle.c")
_HDR = os.path.join(_HERE, "soft_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "libsoft_oracle.so")
_lock = threading.Lock()
_lib = None

ST_OK, ST_DISCARDED, ST_OVERFLOW, ST_ERROR = 0, 1, 2, 3
EV_ERROR, EV_ROT, EV_MEAS = 1, 2, 3

EVENT_DTYPE = np.dtype([("kind", "<i4"), ("op_index", "<i4"), ("a", "<i4"), ("b", "<i4"),
                        ("p_plus", "<f8"), ("u", "<f8"), ("outcome", "<i4"), ("det", "<i4"),
                        ("caseb", "<i4"), ("nnz_before", "<i4"), ("nnz_after", "<i4"),
                        ("pad", "<i4"), ("norm", "<f8")])
assert EVENT_DTYPE.itemsize == 64


class _Counts(ctypes.Structure):
    _fields_ = [("shots", ctypes.c_uint64), ("t_out_entries", ctypes.c_uint64),
                ("t_diag_entries", ctypes.c_uint64), ("meas_entries", ctypes.c_uint64),
                ("noise_entries", ctypes.c_uint64), ("errors", ctypes.c_uint64),
                ("post_t_out", ctypes.c_uint64), ("post_t_diag", ctypes.c_uint64),
                ("post_meas", ctypes.c_uint64), ("post_noise", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C11, -O2) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < newest:
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.or_uniform53.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
            L.or_uniform53.restype = ctypes.c_double
            L.or_gap_threshold.argtypes = [ctypes.c_double, ctypes.c_uint64]
            L.or_gap_threshold.restype = ctypes.c_uint64
            L.or_run.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p,
                                 ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, u64p,
                                 ctypes.POINTER(_Counts)]
            L.or_run_ex.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                    u64p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Counts)]
            L.or_trace.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p,
                                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_size_t,
                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]
            L.or_count_sites.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_uint32)]
            L.or_count_sites.restype = ctypes.c_uint32
            L.or_errors.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p,
                                    ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32]
            L.or_project.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p,
                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                     ctypes.c_uint32, ctypes.c_int64, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            _lib = L
        return _lib


def _ops_array(ops) -> np.ndarray:
    a = ops.array() if hasattr(ops, "array") else ops
    a = np.ascontiguousarray(a)
    if a.dtype.itemsize != 32:
        raise TypeError("ops must be 32-byte op records")
    return a


def _noise_arr(noise) -> np.ndarray:
    t = noise.as_tuple() if hasattr(noise, "as_tuple") else tuple(noise)
    return np.array(t, dtype=np.float64)


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform53(seed, shot, j):
    return float(lib().or_uniform53(seed, shot, j))


def gap_threshold(p, g):
    return int(lib().or_gap_threshold(p, g))


def count_sites(ops, n_qubits, noise):
    a = _ops_array(ops)
    nz = _noise_arr(noise)
    nrec = ctypes.c_uint32(0)
    ns = lib().or_count_sites(a.ctypes.data, len(a), n_qubits, nz.ctypes.data, ctypes.byref(nrec))
    return int(ns), int(nrec.value)


RUN_FIDELITY = 1


def run(ops, n_qubits, noise, cap, seed, first_shot, n_shots, threads=1, records=True, fidelity=False):
    """Run shots [first_shot, first_shot + n_shots). Returns a dict with
    status (u8 per shot), records (u64 words per shot, bit j = 1 for outcome
    -1 of record j), tally [shots, discarded, overflow, kept, logical_errors]
    and the work counters. With fidelity=True every measurement an OBSERVABLE
    reads is projected onto +1: `fid` holds each shot's F (product of those
    conditional probabilities; 0 for shots not kept) and `fsum` = [sum of F
    over kept shots, kept shots]."""
    a = _ops_array(ops)
    nz = _noise_arr(noise)
    _, nrec = count_sites(a, n_qubits, noise)
    rw = max(1, (nrec + 63) // 64)
    status = np.zeros(n_shots, dtype=np.uint8)
    recs = np.zeros((n_shots, rw), dtype=np.uint64) if records else None
    tally = (ctypes.c_uint64 * 5)()
    fsum = np.zeros(2, dtype=np.float64)
    fid = np.zeros(n_shots, dtype=np.float64) if fidelity else None
    cnt = _Counts()
    rc = lib().or_run_ex(a.ctypes.data, len(a), n_qubits, nz.ctypes.data, cap, seed, first_shot, n_shots,
                         threads, RUN_FIDELITY if fidelity else 0, status.ctypes.data,
                         recs.ctypes.data if recs is not None else None, rw, tally, fsum.ctypes.data,
                         fid.ctypes.data if fid is not None else None, ctypes.byref(cnt))
    if rc != 0:
        raise RuntimeError(f"oracle run failed: {rc}")
    return {"status": status, "records": recs, "tally": [int(v) for v in tally],
            "counts": {f: int(getattr(cnt, f)) for f, _ in _Counts._fields_}, "rw": rw, "n_records": nrec,
            "fid": fid, "fsum": fsum}


def trace(ops, n_qubits, noise, cap, seed, shot, stop_after=None, max_events=1 << 16, max_keys=1 << 16):
    """One shot with its event log and final GS state.

    rows_x / rows_z: (2n, 2) words, rows d_0..d_{n-1} then s_0..s_{n-1};
    rows_r: sign bits; keys: (nnz, 2) words sorted; vals: complex128."""
    a = _ops_array(ops)
    nz = _noise_arr(noise)
    _, nrec = count_sites(a, n_qubits, noise)
    rw = max(1, (nrec + 63) // 64)
    n = n_qubits
    ev = np.zeros(max_events, dtype=EVENT_DTYPE)
    nev = ctypes.c_size_t(0)
    rx = np.zeros((2 * n, 2), dtype=np.uint64)
    rz = np.zeros((2 * n, 2), dtype=np.uint64)
    rr = np.zeros(2 * n, dtype=np.uint8)
    keys = np.zeros((max_keys, 2), dtype=np.uint64)
    vals = np.zeros(2 * max_keys, dtype=np.float64)
    nk = ctypes.c_size_t(0)
    rec = np.zeros(rw, dtype=np.uint64)
    st = ctypes.c_int(0)
    lg = ctypes.c_int(0)
    sa = len(a) if stop_after is None else int(stop_after)
    rc = lib().or_trace(a.ctypes.data, len(a), n, nz.ctypes.data, cap, seed, shot, sa, ev.ctypes.data,
                        max_events, ctypes.byref(nev), rx.ctypes.data, rz.ctypes.data, rr.ctypes.data,
                        keys.ctypes.data, vals.ctypes.data, max_keys, ctypes.byref(nk), rec.ctypes.data, rw,
                        ctypes.byref(st), ctypes.byref(lg))
    if rc != 0:
        raise RuntimeError(f"oracle trace failed: {rc}")
    k = int(nk.value)
    return {"events": ev[:min(int(nev.value), max_events)], "rows_x": rx, "rows_z": rz, "rows_r": rr,
            "keys": keys[:k].copy(), "vals": (vals[0:2 * k:2] + 1j * vals[1:2 * k:2]).copy(),
            "status": int(st.value), "logical": int(lg.value), "records": rec}


PROJ_OK, PROJ_OVERFLOW, PROJ_ERROR, PROJ_ZERO = 0, 2, 3, 4


def project(ops, n_qubits, noise, cap, seed, pattern, theta=None, shift_op=-1, shift=0.0):
    """Projection run of the fixed error pattern of shot `pattern`: detector
    measurements forced to their passing outcome, observable measurements to
    0, unnormalised. Returns (status, n_acc, n_fid); the post-selected output
    fidelity is F = n_fid / n_acc."""
    a = _ops_array(ops)
    nz = _noise_arr(noise)
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    na, nf = ctypes.c_double(0), ctypes.c_double(0)
    st = lib().or_project(a.ctypes.data, len(a), n_qubits, nz.ctypes.data, cap, seed, pattern,
                          th.ctypes.data if th is not None else None, 0 if th is None else len(th), int(shift_op),
                          float(shift), ctypes.byref(na), ctypes.byref(nf))
    return int(st), float(na.value), float(nf.value)


def fidelity_grad(ops, n_qubits, noise, cap, seed, pattern, theta):
    """F and dF/dtheta of one pattern by the parameter-shift rule: the squared
    norms are trigonometric polynomials of degree 1 in each Rz angle, so
    d/dx = [N(x + pi/2) - N(x - pi/2)] / 2 per gate occurrence, summed with the
    occurrence's sign (+theta_k or -theta_k)."""
    a = _ops_array(ops)
    st, na, nf = project(a, n_qubits, noise, cap, seed, pattern, theta)
    if st != PROJ_OK:
        return st, na, nf, None
    F = nf / na
    grad = np.zeros(len(theta))
    for i in np.nonzero((a["op"] == 10) & (a["pad"] > 0))[0]:
        k = int(a["pad"][i]) - 1
        sgn = -1.0 if (a["flags"][i] & 1) else 1.0
        _, ap, fp = project(a, n_qubits, noise, cap, seed, pattern, theta, int(i), np.pi / 2)
        _, am, fm = project(a, n_qubits, noise, cap, seed, pattern, theta, int(i), -np.pi / 2)
        dna, dnf = (ap - am) / 2, (fp - fm) / 2
        grad[k] += sgn * (dnf - F * dna) / na
    return st, na, nf, grad


def errors(ops, n_qubits, noise, seed, pattern, max_out=4096):
    """(sites, codes) of every error of shot `pattern`'s noise stream."""
    a = _ops_array(ops)
    nz = _noise_arr(noise)
    sites = np.zeros(max_out, dtype=np.uint32)
    codes = np.zeros(max_out, dtype=np.uint32)
    k = lib().or_errors(a.ctypes.data, len(a), n_qubits, nz.ctypes.data, seed, pattern, sites.ctypes.data,
                        codes.ctypes.data, max_out)
    if k < 0:
        raise RuntimeError("bad circuit")
    return sites[:k].copy(), codes[:k].copy()
