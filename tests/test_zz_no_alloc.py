"""The allocation-free run entry point against the regular one.

soft_run_shots_noalloc serves callers that cannot call cudaMalloc (device
memory owned by another allocator, or loops that cannot afford cudaMalloc's
implicit synchronisation). Its outputs must equal those of soft_run_shots
for the same shots: tallies, status bytes and records are integer results,
compared exactly (the tolerance of the other parity tests for integer
work). Calls in a row check that the shared static scratch, which keeps
the previous call's contents, is cleared correctly, and that after the first
call the device's free memory does not change across a call. A CPU test checks
that the entry point's source names no allocating routine. This file is named
to run last.
"""
import numpy as np
import pytest

from paper_2512_23037_gb300 import circuits as C



@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_23037_gb300 as S
    S.load()
    return torch, S


@pytest.mark.gpu
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
    # output buffers allocated once, refilled before every call
    tally = torch.empty((5,), dtype=torch.int64, device="cuda")
    status = torch.empty((n,), dtype=torch.uint8, device="cuda")
    records = torch.empty((n, rw), dtype=torch.int64, device="cuda")
    free_after = []
    for call in range(3):
        tally.fill_(-1)
        status.fill_(255)
        records.fill_(-1)
        torch.cuda.synchronize()
        S.soft_run_shots_noalloc(c, n, first, seed, precision, stream, tally.data_ptr(), status.data_ptr(),
                                 records.data_ptr())
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
        assert tally.cpu().tolist() == tally_ref, f"call {call}"
        assert np.array_equal(status.cpu().numpy(), st_ref), f"call {call}"
        assert np.array_equal(records.cpu().numpy().view(np.uint64), rec_ref), f"call {call}"
    # after the first call (which may load kernel code), calls take no device memory
    assert free_after[1] == free_after[2], free_after


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, S = env
    circ, noise = C.workload("tiny6")
    c = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    tally = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(S.SoftError) as ei:
        S.soft_run_shots_noalloc(c, (1 << 20) + 1, 0, 0, "fp64", None, tally.data_ptr())
    assert ei.value.code == -1 and "limit" in str(ei.value)


ALLOC = r"\b(cudaMalloc\w*|cudaFree\w*|cudaHostAlloc|cuMemAlloc\w*|cudaMemPool\w*)\b"


def _function(src, signature):
    """Text of the function that starts at `signature` (up to its closing brace
    at the start of a line)."""
    body = src[src.index(signature):]
    return body[:body.index("\n}\n")]


def test_noalloc_source_names_no_allocating_call():
    """The entry point's file, and the launch helpers it calls, name no device
    or pinned-host allocation routine: a regression that adds one fails here,
    without a GPU."""
    import os
    import re
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2512_23037_gb300",
                        "csrc")
    src = open(os.path.join(csrc, "noalloc.cu")).read()
    code = "\n".join(line.split("//", 1)[0] for line in src.splitlines())
    assert not re.findall(ALLOC, code)
    kern = open(os.path.join(csrc, "kernels.cu")).read()
    for sig in ("cudaError_t launch_shots(", "cudaError_t prepare_shots(", "cudaError_t launch_prepared("):
        assert not re.findall(ALLOC, _function(kern, sig)), sig
