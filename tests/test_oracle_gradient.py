"""Pins of the oracle's projection mode and gradient (CPU only).

Projection mode runs one fixed error pattern (the noise draws of a shot)
with every detector measurement projected onto its passing outcome and
every observable measurement onto 0, unnormalised; F = n_fid / n_acc is the
post-selected output fidelity. The oracle's gradient uses the exact
parameter-shift rule. Sources of truth: a dense-statevector projection, a
closed form, and central finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_2512_23037_gb300 import circuits as C
from tests import dense_ref


def test_closed_form_single_rz():
    """H Rz(theta) H |0>, fidelity measurement on qubit 0: F = cos^2(theta/2)."""
    for th in (0.3, 1.1, 2.5, -0.7):
        c = C.Circuit(1)
        c.gate(C.H, 0)
        c.gate(C.RZ, 0, angle=0.0, param=0)
        c.gate(C.H, 0)
        c.observable([c.measure(0)])
        st, na, nf, g = oracle.fidelity_grad(c, 1, C.Noise(), 16, 0, 0, np.array([th]))
        assert st == 0 and abs(na - 1) < 1e-14
        assert abs(nf - np.cos(th / 2) ** 2) < 1e-14
        assert abs(g[0] + 0.5 * np.sin(th)) < 1e-13


@pytest.mark.parametrize("seed", range(6))
def test_projection_matches_dense(seed):
    n = 3 + seed % 4
    c, nz = C.random_param_circuit(seed, n, 40 + 5 * n, n_params=4, p=0.03)
    th = C.rz_thetas(seed, 4, sigma=0.4)
    seen = 0
    for pat in range(12):
        st, na, nf = oracle.project(c, n, nz, c.cap, 9, pat, th)
        s, k = oracle.errors(c, n, nz, 9, pat)
        d = dense_ref.project_pattern(c, nz, s, k, th)
        assert d is not None
        if st == oracle.PROJ_OK:
            seen += 1
            assert abs(na - d[0]) < 1e-12 * max(1, d[0]) and abs(nf - d[1]) < 1e-12 * max(1, d[1])
        else:
            assert st == oracle.PROJ_ZERO and d[0] < 1e-20
    assert seen > 0


@pytest.mark.parametrize("seed", range(4))
def test_parameter_shift_matches_finite_differences(seed):
    n = 4
    c, nz = C.random_param_circuit(100 + seed, n, 60, n_params=5, p=0.02)
    th = C.rz_thetas(seed, 5, sigma=0.5)
    h = 1e-6
    checked = 0
    for pat in range(6):
        st, na, nf, g = oracle.fidelity_grad(c, n, nz, c.cap, 3, pat, th)
        if st != oracle.PROJ_OK:
            continue
        for k in range(len(th)):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            _, a1, f1 = oracle.project(c, n, nz, c.cap, 3, pat, tp)
            _, a2, f2 = oracle.project(c, n, nz, c.cap, 3, pat, tm)
            fd = (f1 / a1 - f2 / a2) / (2 * h)
            assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(g[k])), (pat, k, fd, g[k])
        checked += 1
        assert np.abs(g).max() > 1e-3  # the fidelity really depends on the angles
    assert checked > 0
