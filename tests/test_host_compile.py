"""Host logic of the circuit compiler, on the CPU: the gap-search index that the
noise stream's site search uses (bounded search = plain binary search for every
uniform, at bucket edges, at every threshold and with any number of remaining
sites), on the seeded workloads."""
import os
import shutil
import subprocess

import pytest

from paper_2512_23037_gb300 import circuits as C

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("host") / "gap_index_check")
    csrc = os.path.join(ROOT, "paper_2512_23037_gb300", "csrc")
    cmd = [gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
           os.path.join(HERE, "host", "gap_index_check.cpp"), os.path.join(csrc, "compile.cpp"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


@pytest.mark.parametrize("case", ["w42", "w97", "tiny6", "random40"])
def test_gap_index_matches_plain_search(checker, tmp_path, case):
    if case == "random40":
        circ = C.random_circuit(4040, 40, 400, t_frac=0.2, detectors=True, mpp_frac=0.05)
        p = 0.05
    else:
        circ, noise = C.workload(case)
        p = noise.p1
    ops = tmp_path / "ops.bin"
    ops.write_bytes(circ.array().tobytes())
    r = subprocess.run([checker, str(ops), str(circ.n), repr(p)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
