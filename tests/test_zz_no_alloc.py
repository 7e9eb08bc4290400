"""The allocation-free run entry point against the regular one.

soft_run_shots_noalloc serves callers that cannot call cudaMalloc (device
memory owned by another allocator, or loops that cannot afford cudaMalloc's
implicit synchronisation). Its outputs must equal those of soft_run_shots
for the same shots: tallies, status bytes and records are integer results,
compared exactly (the tolerance of the other parity tests for integer
work). Two calls in a row check that the shared static scratch, which keeps
the previous call's contents, is cleared correctly. This file is named to
run last.
"""
import numpy as np
import pytest

from paper_2512_23037_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_23037_gb300 as S
    S.load()
    return torch, S


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_regular_entry_point(env, precision):
    torch, S = env
    circ, noise = C.workload("w42")
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    n, first, seed = 200_000, 12345, 9
    r = S.soft_run_shots(c, n, first, seed, precision=precision, record_mode=S.REC_ALL)
    rec_ref, st_ref = S.soft_get_records(r, n)
    t = S.soft_tally(r)
    tally_ref = [t["shots"], t["discarded"], t["overflow"], t["kept"], t["logical_errors"]]
    rw = c.info["record_words"]
    stream = torch.cuda.current_stream()
    for call in range(2):
        tally = torch.full((5,), -1, dtype=torch.int64, device="cuda")
        status = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        records = torch.full((n, rw), -1, dtype=torch.int64, device="cuda")
        S.soft_run_shots_noalloc(c, n, first, seed, precision, stream, tally.data_ptr(), status.data_ptr(),
                                 records.data_ptr())
        torch.cuda.synchronize()
        assert tally.cpu().tolist() == tally_ref, f"call {call}"
        assert np.array_equal(status.cpu().numpy(), st_ref), f"call {call}"
        assert np.array_equal(records.cpu().numpy().view(np.uint64), rec_ref), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, S = env
    circ, noise = C.workload("tiny6")
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    tally = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(S.SoftError) as ei:
        S.soft_run_shots_noalloc(c, (1 << 20) + 1, 0, 0, "fp64", None, tally.data_ptr())
    assert ei.value.code == -1 and "limit" in str(ei.value)
