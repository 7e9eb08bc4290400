"""C ABI library: builds, loads and exports every call include/*.h
declares; host-side validation errors need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2512_23037_gb300 import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(soft_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def S():
    import paper_2512_23037_gb300 as S
    S.load()
    return S


def test_every_declared_symbol_is_exported(S):
    names = _declared()
    assert "soft_compile_circuit" in names and "soft_run_shots" in names and "soft_tally" in names
    lib = ctypes.CDLL(S.lib_path())
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(S.EXPORTED)


def _expect(S, code, circ, n, noise, cap=16):
    with pytest.raises(S.SoftError) as ei:
        S.soft_compile_circuit(circ.array(), n, noise, cap)
    assert ei.value.code == code


def test_host_validation_errors(S):
    c = C.Circuit(2)
    c.gate(C.H, 2)
    _expect(S, -2, c, 2, C.Noise())
    c = C.Circuit(2)
    c.gate(C.CX, 1, 1)
    _expect(S, -2, c, 2, C.Noise())
    c = C.Circuit(2)
    c.detector([0])
    _expect(S, -3, c, 2, C.Noise())
    c = C.Circuit(2)
    c.measure(0)
    c.cpauli(1, 1, [1])
    _expect(S, -3, c, 2, C.Noise())
    c = C.Circuit(2)
    c.gate(C.H, 0)
    _expect(S, -4, c, 2, C.Noise(p_idle=1e-3))
    _expect(S, -1, c, 2, C.Noise(p1=1.5))
    _expect(S, -1, c, 2, C.Noise(), cap=0)
    _expect(S, -2, c, 0, C.Noise())
    _expect(S, -2, C.Circuit(200), 200, C.Noise())
    bad = c.array()
    bad["op"][0] = 99
    with pytest.raises(S.SoftError) as ei:
        S.soft_compile_circuit(bad, 2, C.Noise(), 16)
    assert ei.value.code == -4


def test_peak_rejects_bad_kind(S):
    with pytest.raises(S.SoftError) as ei:
        S.soft_peak_pipe_rate(7)
    assert ei.value.code == -1
