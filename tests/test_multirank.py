"""Host logic of multi-process runs, on CPU with the gloo backend (world size 2):
the job's time is its slowest rank's, its work is the sum of the ranks' work,
and the ranks' problem slices are disjoint."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1911_10228_gb300 import multirank as MR


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        MR.barrier()
        out = {
            "active": MR.active(),
            "max": MR.all_max(1.5 + rank),
            "sum": MR.all_sum(10.0 * (rank + 1)),
            "seeds": MR.problem_seeds(64, rank),
        }
        MR.barrier()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_and_shard():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r]["active"]
        assert res[r]["max"] == 2.5            # slowest rank
        assert res[r]["sum"] == 30.0           # all ranks' work
    s0, s1 = set(res[0]["seeds"]), set(res[1]["seeds"])
    assert not (s0 & s1) and s0 | s1 == set(range(128))
    assert res[0]["seeds"] == list(range(64))  # rank 0 alone is the single-GPU batch


def test_single_process_is_the_identity():
    assert not MR.active()
    assert MR.all_max(3.25) == 3.25 and MR.all_sum(7.0) == 7.0
    MR.barrier()
    with pytest.raises(ValueError):
        MR.problem_seeds(-1, 0)
