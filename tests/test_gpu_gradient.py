"""GPU fidelity gradient (adjoint kernel, through the C ABI) against the
oracle's projection runs and parameter-shift gradient, against central
finite differences of the GPU's own F, and through torch.autograd.

Bars: statuses equal; F and p_acc within 1e-10 (FP64) / 1e-5 (FP32) of the
oracle; dF/dtheta within 1e-8 (FP64) / 1e-5 (FP32) absolute of the oracle's
exact parameter-shift gradient. The FP32 bars are about 6x the largest errors
observed on these cases on GB300 (F 1.1e-6, gradient 1.7e-6, both on the
6-qubit case with 64-entry maps; 1e-7 to 3e-7 on the others): FP32
coefficients carry ~1e-6 relative error through ~200 updates, and the
gradient differences two such sums.
"""
import numpy as np
import pytest

import oracle
from paper_2512_23037_gb300 import circuits as C

pytestmark = pytest.mark.gpu

FTOL = {"fp64": 1e-10, "fp32": 1e-5}
GTOL = {"fp64": 1e-8, "fp32": 1e-5}


@pytest.fixture(scope="module")
def soft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_23037_gb300 as S
    S.load()
    return S


def _compare(S, circ, noise, theta, n_pat, seed, precision, first=0):
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    fid, pacc, grad, status = S.soft_fidelity_grad(c, theta, n_pat, first, seed, precision)
    fid, pacc, grad, status = fid.cpu().numpy(), pacc.cpu().numpy(), grad.cpu().numpy(), status.cpu().numpy()
    ok = 0
    for i in range(n_pat):
        st, na, nf, g = oracle.fidelity_grad(circ, circ.n, noise, circ.cap, seed, first + i, theta)
        if status[i] == 2:  # GPU register map limit: skipped, counted
            continue
        want = {oracle.PROJ_OK: 0, oracle.PROJ_ZERO: 1}.get(st, 3)
        assert status[i] == want, (i, status[i], st)
        if st != oracle.PROJ_OK:
            continue
        ok += 1
        assert abs(pacc[i] - na) <= FTOL[precision] * max(1.0, na), (i, pacc[i], na)
        assert abs(fid[i] - nf / na) <= FTOL[precision], (i, fid[i], nf / na)
        assert np.max(np.abs(grad[i] - g)) <= GTOL[precision], (i, grad[i], g)
    return ok, status


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(5))
def test_random_param_circuits(soft, precision, seed):
    # n <= 5 keeps the coefficient map within the kernel's 32 register entries
    n = 3 + seed % 3
    circ, noise = C.random_param_circuit(700 + seed, n, 50 + 6 * n + 7 * seed, n_params=6, p=0.02)
    theta = C.rz_thetas(seed, 6, sigma=0.5)
    ok, _ = _compare(soft, circ, noise, theta, 60, 5 + seed, precision)
    assert ok >= 3


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [6, 7])
def test_wide_maps_match_oracle(soft, n, precision):
    """Random Rz angles on 6 and 7 qubits fill 64 and 128 map entries, beyond
    the 32-entry register maps: the shared-memory rerun must give every
    accepted pattern, matching the oracle."""
    circ, noise = C.random_param_circuit(700 + n - 3, n, 50 + 6 * n, n_params=6, p=0.02)
    theta = C.rz_thetas(n - 3, 6, sigma=0.5)
    ok, status = _compare(soft, circ, noise, theta, 24, n + 2, precision)
    n_ok = sum(1 for i in range(24)
               if oracle.fidelity_grad(circ, circ.n, noise, circ.cap, n + 2, i, theta)[0] == oracle.PROJ_OK)
    assert ok == n_ok and ok >= 3 and not np.any(status == 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_w42_rz_patterns(soft, precision):
    """The 42-qubit workload with every T/T^dag pair as Rz(+-theta_i), 72 angles."""
    circ, noise = C.workload("w42rz")
    theta = C.rz_thetas(1, 72)
    ok, status = _compare(soft, circ, noise, theta, 300, 0, precision)
    assert ok > 5 and np.sum(status == 1) > 100
    # ratio estimator sum N_acc F / sum N_acc over the ok patterns, reduced on the device
    c = soft.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    _, _, _, st, sums = soft.soft_fidelity_grad(c, theta, 300, 0, 0, precision, sums=True)
    st, sums = st.cpu().numpy(), sums.cpu().numpy()
    na = nf = 0.0
    for i in np.nonzero(st == 0)[0]:
        _, a, f, _ = oracle.fidelity_grad(circ, circ.n, noise, circ.cap, 0, int(i), theta)
        na += a
        nf += f
    assert sums[2] == np.sum(st == 0)
    assert abs(sums[0] - na) <= FTOL[precision] * max(1.0, na)
    assert abs(sums[1] / sums[0] - nf / na) <= FTOL[precision]


def test_gpu_gradient_matches_finite_differences(soft):
    S = soft
    circ, noise = C.random_param_circuit(901, 5, 80, n_params=4, p=0.02)
    theta = C.rz_thetas(3, 4, sigma=0.5)
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    fid, pacc, grad, status = S.soft_fidelity_grad(c, theta, 30, 0, 2, "fp64")
    fid, grad, status = fid.cpu().numpy(), grad.cpu().numpy(), status.cpu().numpy()
    h = 1e-6
    for k in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fp = S.soft_fidelity_grad(c, tp, 30, 0, 2, "fp64")[0].cpu().numpy()
        fm = S.soft_fidelity_grad(c, tm, 30, 0, 2, "fp64")[0].cpu().numpy()
        sel = status == 0
        fd = (fp - fm) / (2 * h)
        assert np.max(np.abs(fd[sel] - grad[sel, k])) < 1e-6
    assert np.abs(grad[status == 0]).max() > 1e-3


def test_w42rz_gradient_matches_finite_differences(soft):
    """The differentiation workload itself (w42rz: 72 angles): the adjoint
    gradient equals central differences of the GPU's own F, h = 1e-6, for all
    72 angles (FP64; the central difference's truncation and rounding error is
    ~1e-10 here), on every accepted pattern of the range, of which at least 20
    have a nonzero gradient. (Most accepted patterns have F = 1 for any angles:
    without an effective error each Rz(theta) meets its Rz(-theta); the range
    grows until it holds 20 that do not.)"""
    S = soft
    circ, noise = C.workload("w42rz")
    theta = C.rz_thetas(1, 72)
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    for n in (20000, 100000, 400000):
        fid, pacc, grad, status = [t.cpu().numpy() for t in S.soft_fidelity_grad(c, theta, n, 0, 0, "fp64")]
        sel = status == 0
        live = sel & (np.abs(grad).max(axis=1) > 1e-6)
        if live.sum() >= 20:
            break
    assert live.sum() >= 20, (n, sel.sum(), live.sum())
    h = 1e-6
    worst = 0.0
    for k in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fp, _, _, sp = [t.cpu().numpy() for t in S.soft_fidelity_grad(c, tp, n, 0, 0, "fp64")]
        fm, _, _, sm = [t.cpu().numpy() for t in S.soft_fidelity_grad(c, tm, n, 0, 0, "fp64")]
        assert np.array_equal(sp, status) and np.array_equal(sm, status)
        fd = (fp - fm) / (2 * h)
        worst = max(worst, float(np.max(np.abs(fd[sel] - grad[sel, k]))))
    assert worst < 1e-7, worst
    assert np.abs(grad[sel]).max() > 1e-3


def test_autograd_function(soft):
    import torch
    from paper_2512_23037_gb300.grad import PostSelectedFidelity
    S = soft
    circ, noise = C.random_param_circuit(902, 4, 70, n_params=5, p=0.02)
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    theta = torch.tensor(C.rz_thetas(4, 5, sigma=0.5), dtype=torch.float64, requires_grad=True)
    fid, pacc, status = PostSelectedFidelity.apply(theta, c, 25, 0, 8, "fp64")
    w = torch.linspace(0.5, 1.5, 25, dtype=torch.float64, device=fid.device)
    loss = (w * fid).sum()
    loss.backward()
    _, _, grad, _ = S.soft_fidelity_grad(c, theta.detach().numpy(), 25, 0, 8, "fp64")
    want = (w.unsqueeze(1) * grad).sum(0).cpu()
    assert torch.allclose(theta.grad, want, atol=1e-12)
