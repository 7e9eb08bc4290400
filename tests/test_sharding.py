"""Multi-rank path on CPU: two gloo ranks each run their own shot range and
sum the tallies with one all-reduce; the result must equal one process
running both ranges (results depend only on the shot index)."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2512_23037_gb300 import circuits as C
from paper_2512_23037_gb300.sharding import reduce_tallies, shot_range

N_PER_RANK = 300


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    circ, noise = C.workload("w42")
    first, n = shot_range(rank, world, N_PER_RANK)
    r = oracle.run(circ, circ.n, noise, circ.cap, 5, first, n, threads=1, records=False)
    t = torch.tensor(r["tally"], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        out.put(t.tolist())
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
    parts = []
    for r in range(2):
        first, n = shot_range(r, 2, N_PER_RANK)
        parts.append(oracle.run(circ, circ.n, noise, circ.cap, 5, first, n, threads=2, records=False)["tally"])
    assert got == reduce_tallies(parts)
    assert got[0] == 2 * N_PER_RANK


def test_shot_range_validation():
    assert shot_range(1, 4, 10) == (1 << 40, 10)
    with pytest.raises(ValueError):
        shot_range(4, 4, 10)
