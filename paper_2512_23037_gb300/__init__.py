"""GB300 generalized-stabilizer shot simulator (arxiv 2512.23037, shot-parallel hot path).

Thin ctypes binding over the C ABI of include/soft.h; every step of the
simulation runs in libsoft.so (sm_103a). The binding only marshals
arguments. There is no CPU fallback: if the shared library cannot be built
or loaded, every call raises.

    from paper_2512_23037_gb300 import circuits, soft_compile_circuit, soft_run_shots, soft_tally
    circ, noise = circuits.workload("w42")
    c = soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = soft_run_shots(c, 1 << 20, 0, seed=0, precision="fp32")
    print(soft_tally(r))
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import circuits  # noqa: F401  (input format + seeded generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

SOFT_OK = 0
FP64, FP32 = 0, 1
REC_NONE, REC_FIRST_K, REC_ALL = 0, 1, 2
SHOT_KEPT, SHOT_DISCARDED, SHOT_OVERFLOW, SHOT_ERROR = 0, 1, 2, 3
RUN_GRAPH, RUN_FIDELITY, RUN_NO_PREFIX, RUN_NO_LANES, RUN_TIME_PASSES, RUN_NO_WIDE_LANES, RUN_WIDE_LANES = \
    1, 2, 4, 8, 16, 32, 64


class SoftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"soft error {code}: {msg}")
        self.code = code


class _Noise(ctypes.Structure):
    _fields_ = [("p1", ctypes.c_double), ("p2", ctypes.c_double), ("p_meas", ctypes.c_double),
                ("p_reset", ctypes.c_double), ("p_idle", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_uint32), ("n_records", ctypes.c_uint32), ("record_words", ctypes.c_uint32),
                ("n_sites", ctypes.c_uint32), ("n_events", ctypes.c_uint32), ("coeff_cap", ctypes.c_uint32),
                ("program_bytes", ctypes.c_uint64)]


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("record_mode", ctypes.c_int32), ("record_k", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("group_size", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("chunk_shots", ctypes.c_uint64), ("first_cap", ctypes.c_uint32), ("capture_k", ctypes.c_uint32),
                ("d_records", ctypes.c_void_p), ("d_status", ctypes.c_void_p),
                ("groups_per_block", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class _Tally(ctypes.Structure):
    _fields_ = [("shots", ctypes.c_uint64), ("discarded", ctypes.c_uint64), ("overflow", ctypes.c_uint64),
                ("kept", ctypes.c_uint64), ("logical_errors", ctypes.c_uint64), ("sum_fidelity", ctypes.c_double),
                ("sum_weight", ctypes.c_double)]


EXPORTED = ["soft_compile_circuit", "soft_circuit_info", "soft_circuit_tableau", "soft_circuit_free",
            "soft_run_shots", "soft_tally", "soft_get_records", "soft_get_state", "soft_run_timing", "soft_run_pass_timing", "soft_release_workspace",
            "soft_run_free", "soft_run_shots_noalloc", "soft_run_diagnostics", "soft_run_batch",
            "soft_tally_batch", "soft_fidelity_grad", "soft_last_error", "soft_peak_pipe_rate"]
PEAK_FP64_FMA, PEAK_FP32_FMA, PEAK_INT32_LOGIC = 0, 1, 2


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "libsoft.so")


def load(build_if_missing: bool = True):
    """Load libsoft.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from .build import build
            build()
        L = ctypes.CDLL(lib_path())
        vp, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
        L.soft_compile_circuit.argtypes = [vp, sz, u32, ctypes.POINTER(_Noise), u32, ctypes.POINTER(vp)]
        L.soft_circuit_info.argtypes = [vp, ctypes.POINTER(_Info)]
        L.soft_circuit_tableau.argtypes = [vp, vp, vp]
        L.soft_circuit_free.argtypes = [vp]
        L.soft_circuit_free.restype = None
        L.soft_run_shots.argtypes = [vp, u64, u64, u64, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
        L.soft_tally.argtypes = [vp, ctypes.POINTER(_Tally)]
        L.soft_get_records.argtypes = [vp, vp, sz, vp, sz]
        L.soft_get_state.argtypes = [vp, u64, vp, vp, vp, sz, ctypes.POINTER(sz)]
        L.soft_run_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32)]
        L.soft_run_pass_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32), ctypes.POINTER(u64)]
        L.soft_run_free.argtypes = [vp]
        L.soft_run_free.restype = None
        L.soft_release_workspace.argtypes = []
        L.soft_run_shots_noalloc.argtypes = [vp, u64, u64, u64, ctypes.c_int32, vp, vp, vp, vp]
        L.soft_run_diagnostics.argtypes = [vp, vp]
        L.soft_run_batch.argtypes = [vp, vp, vp, u32, u64, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
        L.soft_tally_batch.argtypes = [vp, u32, ctypes.POINTER(_Tally)]
        L.soft_fidelity_grad.argtypes = [vp, vp, u32, u64, u64, u64, ctypes.c_int32, vp, vp, vp, vp, vp, vp]
        L.soft_peak_pipe_rate.argtypes = [ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.soft_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(rc):
    if rc != SOFT_OK:
        raise SoftError(rc, load().soft_last_error().decode())


class Circuit:
    """Compiled circuit handle (owns device memory)."""

    def __init__(self, handle, n_qubits):
        self.h = ctypes.c_void_p(handle)
        self.n = n_qubits
        info = _Info()
        _check(load().soft_circuit_info(self.h, ctypes.byref(info)))
        self.info = {f: int(getattr(info, f)) for f, _ in _Info._fields_}

    def tableau(self):
        """Final shot-invariant X/Z words, shape (2n, 2): rows d_0.. then s_0.."""
        x = np.zeros((2 * self.n, 2), dtype=np.uint64)
        z = np.zeros((2 * self.n, 2), dtype=np.uint64)
        _check(load().soft_circuit_tableau(self.h, x.ctypes.data, z.ctypes.data))
        return x, z

    def free(self):
        if self.h:
            load().soft_circuit_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Run:
    """Run handle: tallies, records, captured states, timing."""

    def __init__(self, handle, circuit, n_shots):
        self.h = ctypes.c_void_p(handle)
        self.circuit = circuit  # keep the program alive while the run is in flight
        self.n_shots = n_shots

    def free(self):
        if self.h:
            load().soft_run_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _noise(noise) -> _Noise:
    t = noise.as_tuple() if hasattr(noise, "as_tuple") else tuple(noise)
    return _Noise(*[float(v) for v in t])


def soft_compile_circuit(ops, n_qubits: int, noise, coeff_cap: int) -> Circuit:
    a = np.ascontiguousarray(ops.array() if hasattr(ops, "array") else ops)
    if a.dtype.itemsize != 32:
        raise TypeError("ops must be 32-byte op records")
    out = ctypes.c_void_p()
    nz = _noise(noise)
    _check(load().soft_compile_circuit(a.ctypes.data if len(a) else None, len(a), n_qubits, ctypes.byref(nz),
                                       int(coeff_cap), ctypes.byref(out)))
    return Circuit(out.value, n_qubits)


def _opts(precision="fp64", record_mode=REC_NONE, record_k=0, stream=None, group_size=0, blocks_per_sm=0,
          chunk_shots=0, first_cap=0, capture_k=0, d_records=None, d_status=None, groups_per_block=0,
          graph=False, fidelity=False, prefix=True, lanes=True, time_passes=False, wide=None) -> _Opts:
    o = _Opts()
    o.precision = FP32 if precision in ("fp32", FP32) else FP64
    o.record_mode = int(record_mode)
    o.record_k = int(record_k)
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream()
        except ImportError:
            stream = None
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    o.stream = ctypes.c_void_p(int(stream) if stream else 0)
    o.group_size = int(group_size)
    o.blocks_per_sm = int(blocks_per_sm)
    o.chunk_shots = int(chunk_shots)
    o.first_cap = int(first_cap)
    o.capture_k = int(capture_k)
    o.d_records = ctypes.c_void_p(int(d_records) if d_records else 0)
    o.d_status = ctypes.c_void_p(int(d_status) if d_status else 0)
    o.groups_per_block = int(groups_per_block)
    o.flags = ((RUN_GRAPH if graph else 0) | (RUN_FIDELITY if fidelity else 0) | (0 if prefix else RUN_NO_PREFIX)
               | (0 if lanes else RUN_NO_LANES) | (RUN_TIME_PASSES if time_passes else 0)
               | (0 if wide is None else (RUN_WIDE_LANES if wide else RUN_NO_WIDE_LANES)))
    return o


def soft_run_shots(circ: Circuit, n_shots: int, first_shot: int = 0, seed: int = 0, precision="fp64",
                   record_mode=REC_NONE, record_k: int = 0, stream=None, group_size: int = 0,
                   blocks_per_sm: int = 0, chunk_shots: int = 0, first_cap: int = 0, capture_k: int = 0,
                   d_records=None, d_status=None, groups_per_block: int = 0, graph: bool = False,
                   fidelity: bool = False, prefix: bool = True, lanes: bool = True,
                   time_passes: bool = False, wide=None) -> Run:
    """Launch shots asynchronously on `stream` (a torch.cuda.Stream, a raw
    cudaStream_t int, or None for torch's current stream when torch is
    imported, else the legacy default stream). fidelity=True projects the
    observed measurements onto +1 and sums their exact fidelity F per kept
    shot (tally sum_fidelity / sum_weight). prefix=False runs every shot from
    the first event instead of from the shared noiseless prefix, lanes=False a
    warp per shot instead of a lane per shot where that applies (same results).
    time_passes=True records events between passes for soft_run_pass_timing.
    wide: None runs the wide round (FP32 single-circuit runs) for chunks of at
    least 2^23 shots, True for any chunk, False never."""
    o = _opts(precision, record_mode, record_k, stream, group_size, blocks_per_sm, chunk_shots, first_cap,
              capture_k, d_records, d_status, groups_per_block, graph, fidelity, prefix, lanes, time_passes, wide)
    out = ctypes.c_void_p()
    _check(load().soft_run_shots(circ.h, int(n_shots), int(first_shot), int(seed) & (2 ** 64 - 1), ctypes.byref(o),
                                 ctypes.byref(out)))
    return Run(out.value, circ, n_shots)


def soft_run_batch(circs, n_shots, first_shots, seed: int = 0, **kw) -> Run:
    """One launch sequence over several compiled circuits; tallies per circuit
    with soft_tally_batch."""
    n = len(circs)
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in circs])
    ns = (ctypes.c_uint64 * n)(*[int(v) for v in n_shots])
    fs = (ctypes.c_uint64 * n)(*[int(v) for v in first_shots])
    o = _opts(**kw)
    out = ctypes.c_void_p()
    _check(load().soft_run_batch(hs, ns, fs, n, int(seed) & (2 ** 64 - 1), ctypes.byref(o), ctypes.byref(out)))
    r = Run(out.value, circs[0], sum(int(v) for v in n_shots))
    r.circuits = list(circs)
    return r


def soft_tally_batch(run: Run, index: int) -> dict:
    t = _Tally()
    _check(load().soft_tally_batch(run.h, int(index), ctypes.byref(t)))
    return {f: (float(getattr(t, f)) if f.startswith("sum") else int(getattr(t, f))) for f, _ in _Tally._fields_}


def soft_tally(run: Run) -> dict:
    t = _Tally()
    _check(load().soft_tally(run.h, ctypes.byref(t)))
    return {f: (float(getattr(t, f)) if f.startswith("sum") else int(getattr(t, f))) for f, _ in _Tally._fields_}


def soft_get_records(run: Run, n: int):
    """Records (n, record_words) uint64 and status bytes of the first n kept shots."""
    rw = run.circuit.info["record_words"]
    rec = np.zeros((n, rw), dtype=np.uint64)
    st = np.zeros(n, dtype=np.uint8)
    _check(load().soft_get_records(run.h, rec.ctypes.data, rec.size, st.ctypes.data, st.size))
    return rec, st


def soft_get_state(run: Run, shot_offset: int):
    """(signs[4], keys (nnz, 2) uint64, vals complex128) of a captured shot."""
    cap = run.circuit.info["coeff_cap"]
    signs = np.zeros(4, dtype=np.uint64)
    keys = np.zeros((cap, 2), dtype=np.uint64)
    vals = np.zeros(2 * cap, dtype=np.float64)
    nnz = ctypes.c_size_t(0)
    _check(load().soft_get_state(run.h, int(shot_offset), signs.ctypes.data, keys.ctypes.data, vals.ctypes.data,
                                 cap, ctypes.byref(nnz)))
    k = int(nnz.value)
    return signs, keys[:k].copy(), (vals[0:2 * k:2] + 1j * vals[1:2 * k:2]).copy()


def soft_run_diagnostics(run: Run):
    """[failed checks, code << 32 | event, shot, value] of the run's in-kernel bounds checks."""
    out = np.zeros(4, dtype=np.uint64)
    _check(load().soft_run_diagnostics(run.h, out.ctypes.data))
    return [int(v) for v in out]


def soft_run_timing(run: Run):
    ms = ctypes.c_double(0)
    nl = ctypes.c_uint32(0)
    _check(load().soft_run_timing(run.h, ctypes.byref(ms), ctypes.byref(nl)))
    return float(ms.value), int(nl.value)


def soft_release_workspace():
    """Free every device's cached run workspace (runs still alive keep theirs)."""
    _check(load().soft_release_workspace())


def soft_run_pass_timing(run: Run):
    """([pre-pass, first pass, rerun pass] ms summed over chunks, chunks, shots
    finished by the rerun pass) of a run launched with time_passes=True."""
    ms = (ctypes.c_double * 3)()
    nc = ctypes.c_uint32(0)
    nr = ctypes.c_uint64(0)
    _check(load().soft_run_pass_timing(run.h, ms, ctypes.byref(nc), ctypes.byref(nr)))
    return [float(v) for v in ms], int(nc.value), int(nr.value)


def soft_run_shots_noalloc(circ: Circuit, n_shots: int, first_shot: int, seed: int, precision, stream,
                           d_tally: int, d_status: int = 0, d_records: int = 0) -> None:
    """Allocation-free run (at most 2^20 shots per call) into caller device
    buffers given as raw pointers; see include/soft.h."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(load().soft_run_shots_noalloc(circ.h, int(n_shots), int(first_shot), int(seed) & (2 ** 64 - 1),
                                         FP32 if precision in ("fp32", FP32) else FP64,
                                         ctypes.c_void_p(int(stream) if stream else 0),
                                         ctypes.c_void_p(int(d_tally)), ctypes.c_void_p(int(d_status or 0)),
                                         ctypes.c_void_p(int(d_records or 0))))


def soft_fidelity_grad(circ: Circuit, theta, n_patterns: int, first_pattern: int = 0, seed: int = 0,
                       precision="fp64", stream=None, sums=False):
    """Post-selected fidelity F, acceptance N_acc, dF/dtheta and status of
    fixed error patterns (see include/soft.h). Returns torch tensors on the
    current CUDA device: F (n,), p_acc (n,), grad (n, n_params), status (n,),
    and with sums=True also (3,) = [sum N_acc, sum N_acc F, ok count] over ok
    patterns (the ratio estimator is sums[1] / sums[0])."""
    import torch
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    n = int(n_patterns)
    dev = torch.device("cuda", torch.cuda.current_device())
    fid = torch.zeros(n, dtype=torch.float64, device=dev)
    pacc = torch.zeros(n, dtype=torch.float64, device=dev)
    grad = torch.zeros((n, len(th)), dtype=torch.float64, device=dev)
    status = torch.zeros(n, dtype=torch.uint8, device=dev)
    s3 = torch.zeros(3, dtype=torch.float64, device=dev) if sums else None
    if stream is None:
        stream = torch.cuda.current_stream()
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(load().soft_fidelity_grad(circ.h, th.ctypes.data if len(th) else None, len(th), n, int(first_pattern),
                                     int(seed) & (2 ** 64 - 1), FP32 if precision in ("fp32", FP32) else FP64,
                                     ctypes.c_void_p(int(stream) if stream else 0), fid.data_ptr(),
                                     pacc.data_ptr(), grad.data_ptr() if len(th) else None, status.data_ptr(),
                                     s3.data_ptr() if s3 is not None else None))
    if sums:
        return fid, pacc, grad, status, s3
    return fid, pacc, grad, status


def soft_peak_pipe_rate(kind: int, stream=None):
    """(ops/s, ms per launch) of one arithmetic pipe on the current device:
    kind PEAK_FP64_FMA / PEAK_FP32_FMA (flops/s, an FMA = 2) or
    PEAK_INT32_LOGIC (ops/s); see include/soft_peak.h."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    r, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().soft_peak_pipe_rate(int(kind), ctypes.c_void_p(int(stream) if stream else 0), ctypes.byref(r),
                                      ctypes.byref(ms)))
    return float(r.value), float(ms.value)
