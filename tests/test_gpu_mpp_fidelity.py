"""GPU path (through the C ABI) against the oracle for Pauli-product
measurements (MPP), fixed-Pauli flip sites and the exact-fidelity mode.

Bars: records, statuses and tableau words bit-exact (outcomes with
|p - u| <= band excepted, counted); coefficients within 1e-12 (FP64) /
1e-5 (FP32); the fidelity sum over kept shots within kept * 1e-12 (FP64) /
kept * 1e-5 (FP32) of the oracle's, with identical kept counts.
"""
import numpy as np
import pytest

import oracle
from paper_2512_23037_gb300 import circuits as C
from tests.test_gpu_parity import compare_records, compare_states, run_both

pytestmark = pytest.mark.gpu

FSUM_TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def soft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_23037_gb300 as S
    S.load()
    return S


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(5))
def test_mpp_random_circuits(soft, precision, seed):
    n = [3, 6, 11, 40, 90][seed]
    circ = C.random_circuit(2000 + seed, n, 60 + 8 * n, t_frac=0.18, detectors=True, mpp_frac=0.1)
    circ.cap = 256
    noise = C.Noise(0.01, 0.01, 0.02, 0.01)
    c, r, rec, st, tal, ref = run_both(soft, circ, noise, 700, seed, precision, capture=40)
    assert compare_records(circ, noise, seed, 0, rec, st, ref, precision) <= 3
    compare_states(soft, c, r, circ, noise, seed, 0, 40, precision)


def test_mpp_closed_form_eigenvalues(soft):
    S = soft
    c = C.Circuit(3)
    c.gate(C.H, 0)
    c.gate(C.CX, 0, 1)
    c.gate(C.CX, 1, 2)
    rg = c.mpp([(1, 0), (1, 1), (1, 2)])
    ry = c.mpp([(2, 0), (2, 1), (1, 2)])
    h = S.soft_compile_circuit(c.array(), 3, C.Noise(), 16)
    r = S.soft_run_shots(h, 256, 0, 1, record_mode=S.REC_ALL)
    rec, st = S.soft_get_records(r, 256)
    assert np.all(st == 0)
    assert np.all((rec[:, 0] >> np.uint64(rg)) & np.uint64(1) == 0)
    assert np.all((rec[:, 0] >> np.uint64(ry)) & np.uint64(1) == 1)


def test_flip_sites_are_x(soft):
    """p_meas = 0.3 before M on |0>: record 1 with probability 0.3, shot for
    shot the oracle's draws."""
    S = soft
    c = C.Circuit(1)
    c.measure(0)
    noise = C.Noise(p_meas=0.3)
    h = S.soft_compile_circuit(c.array(), 1, noise, 4)
    r = S.soft_run_shots(h, 20000, 0, 5, record_mode=S.REC_ALL)
    rec, st = S.soft_get_records(r, 20000)
    ref = oracle.run(c, 1, noise, 4, 5, 0, 20000, threads=8)
    assert np.array_equal(rec[:, 0], ref["records"][:, 0])
    f = float(np.mean(rec[:, 0] & np.uint64(1)))
    assert abs(f - 0.3) < 5 * np.sqrt(0.21 / 20000)


def _fid_both(S, circ, noise, n_shots, seed, precision, first_shot=0, **kw):
    h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = S.soft_run_shots(h, n_shots, first_shot, seed, precision=precision, fidelity=True, **kw)
    tal = S.soft_tally(r)
    ref = oracle.run(circ, circ.n, noise, circ.cap, seed, first_shot, n_shots, threads=8, records=False,
                     fidelity=True)
    return tal, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fidelity_windowed(soft, precision):
    circ, noise = C.windowed(5, n_data=14, n_anc=2, blocks=5, w=3, n_cliff=20, checks=2, p=0.004)
    tal, ref = _fid_both(soft, circ, noise, 4000, 3, precision)
    assert tal["kept"] == ref["tally"][3] and tal["discarded"] == ref["tally"][1]
    assert tal["sum_weight"] == ref["fsum"][1]
    assert abs(tal["sum_fidelity"] - ref["fsum"][0]) <= FSUM_TOL[precision] * max(1, tal["kept"])
    assert tal["sum_fidelity"] < tal["kept"]  # some kept shots carry F < 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fidelity_w42_prefix_and_graph(soft, precision):
    """The 42-qubit workload in fidelity mode; graph replay of chunks gives the same sums."""
    circ, noise = C.workload("w42")
    tal, ref = _fid_both(soft, circ, noise, 3000, 7, precision)
    assert tal["kept"] == ref["tally"][3]
    assert abs(tal["sum_fidelity"] - ref["fsum"][0]) <= FSUM_TOL[precision] * max(1, tal["kept"])
    import torch
    s = torch.cuda.Stream()
    h = soft.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    r = soft.soft_run_shots(h, 3000, 0, 7, precision=precision, fidelity=True, graph=True, chunk_shots=1000,
                            stream=s)
    t2 = soft.soft_tally(r)
    assert t2["kept"] == tal["kept"]
    assert abs(t2["sum_fidelity"] - tal["sum_fidelity"]) <= 1e-9 * max(1, tal["kept"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fidelity_prefix_start_is_exact(soft, precision):
    """Fidelity mode stops the shared noiseless run at the first observed
    measurement: with and without the prefix start (a warp per shot on both
    sides; the lane kernel always starts from the prefix) the counters are
    identical and the fidelity sums equal up to the order of their FP64 atomic
    additions; the default lane-per-shot run gives the same counters and sum."""
    S = soft
    circ, noise = C.workload("w42")
    h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    a = S.soft_tally(S.soft_run_shots(h, 20000, 0, 4, precision=precision, fidelity=True, lanes=False))
    b = S.soft_tally(S.soft_run_shots(h, 20000, 0, 4, precision=precision, fidelity=True, prefix=False))
    c = S.soft_tally(S.soft_run_shots(h, 20000, 0, 4, precision=precision, fidelity=True))
    key = ("shots", "discarded", "overflow", "kept", "logical_errors", "sum_weight")
    assert [a[k] for k in key] == [b[k] for k in key] == [c[k] for k in key]
    assert abs(a["sum_fidelity"] - b["sum_fidelity"]) <= 1e-12 * a["kept"]
    tol = {"fp64": 1e-12, "fp32": 1e-5}[precision]
    assert abs(c["sum_fidelity"] - b["sum_fidelity"]) <= tol * a["kept"]


def test_fidelity_estimator_vs_sampling_on_gpu(soft):
    """Same shots sampled and in fidelity mode: identical kept counts; the
    sampled logical-error rate within 5 sigma of 1 - mean F."""
    S = soft
    circ, noise = C.windowed(5, n_data=10, n_anc=2, blocks=4, w=3, n_cliff=16, checks=2, p=0.01)
    h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    N = 200000
    a = S.soft_tally(S.soft_run_shots(h, N, 0, 8, precision="fp32"))
    b = S.soft_tally(S.soft_run_shots(h, N, 0, 8, precision="fp32", fidelity=True))
    assert a["kept"] == b["kept"] and a["discarded"] == b["discarded"]
    ler = a["logical_errors"] / a["kept"]
    est = 1 - b["sum_fidelity"] / b["sum_weight"]
    assert abs(ler - est) < 5 * np.sqrt(max(ler * (1 - ler), 1e-6) / a["kept"]), (ler, est)


def test_fidelity_rejects_detector_after_chain(soft):
    S = soft
    c = C.Circuit(2)
    c.observable([c.measure(0)])
    c.detector([c.measure(1)])
    h = S.soft_compile_circuit(c.array(), 2, C.Noise(), 8)
    with pytest.raises(S.SoftError):
        S.soft_run_shots(h, 4, 0, 0, fidelity=True)
