"""Multi-rank path on CPU: two gloo ranks each run their contiguous part of one
job of N shots and sum the tallies with the all-reduce the bench uses; the
result must equal one process running the whole job (results depend only on
the shot index, Sec. IV-B). The worker is the oracle here (no GPU in this
test); what is tested is the partition and the reduction."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2512_23037_gb300 import circuits as C
from paper_2512_23037_gb300.sharding import all_reduce_tally, reduce_tallies, shot_range

N_JOB = 601  # odd: the two ranks get 300 and 301 shots
FIRST = 12345


def _tally_dict(r):
    t = r["tally"]
    return {"shots": t[0], "discarded": t[1], "overflow": t[2], "kept": t[3], "logical_errors": t[4],
            "sum_fidelity": float(r["fsum"][0]), "sum_weight": float(r["fsum"][1])}


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    circ, noise = C.workload("w42")
    first, n = shot_range(rank, world, N_JOB, FIRST)
    r = oracle.run(circ, circ.n, noise, circ.cap, 5, first, n, threads=1, records=False, fidelity=True)
    job = all_reduce_tally(_tally_dict(r), dist)
    if rank == 0:
        out.put(job)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_match_single_process():
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    circ, noise = C.workload("w42")
    whole = oracle.run(circ, circ.n, noise, circ.cap, 5, FIRST, N_JOB, threads=2, records=False, fidelity=True)
    want = _tally_dict(whole)
    for k in ("shots", "discarded", "overflow", "kept", "logical_errors"):
        assert got[k] == want[k], k
    assert got["shots"] == N_JOB
    # the FP64 sums agree up to the order of the additions
    assert abs(got["sum_fidelity"] - want["sum_fidelity"]) <= 1e-9 * max(1.0, want["sum_fidelity"])
    assert got["sum_weight"] == want["sum_weight"]


def test_shot_range_is_a_contiguous_partition():
    for world in (1, 2, 3, 8):
        for n in (0, 1, 7, 1000, (1 << 40) + 3):
            parts = [shot_range(r, world, n, 100) for r in range(world)]
            assert parts[0][0] == 100
            for (f0, c0), (f1, _) in zip(parts, parts[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in parts) == n
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        shot_range(4, 4, 10)


def test_reduce_tallies_lists_and_dicts():
    assert reduce_tallies([[1, 2, 3, 4, 5], [10, 20, 30, 40, 50]]) == [11, 22, 33, 44, 55]
    a = {"shots": 3, "discarded": 1, "overflow": 0, "kept": 2, "logical_errors": 1, "sum_fidelity": 1.5,
         "sum_weight": 2.0}
    s = reduce_tallies([a, a])
    assert s["shots"] == 6 and s["kept"] == 4 and s["sum_fidelity"] == 3.0
