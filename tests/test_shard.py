"""Sharding one solve by target blocks (host logic, CPU).

* The Morton partition: owners of contiguous Z-order chunks of nearly equal
  size; on a 4x4x4 box in 8 parts every part is one 2x2x2 octant (the defining
  property of the Z-order curve), and every block has exactly one owner.
* Two gloo ranks, each evaluating only its own targets from the replicated
  source, and one summation of the owned blocks give exactly the single-rank
  solve.  The per-rank evaluation here is the oracle's FLGF restricted to
  target blocks (the GPU counterpart, a block set wanting only the rank's
  blocks, is checked in tests/test_gpu_shard.py).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1911_10228_gb300 import multirank as MR
from paper_1911_10228_gb300.inputs import box_coords, config_plain_32, random_sparse_problem
from paper_1911_10228_gb300.shard import morton_keys, morton_partition, shard_masks


def test_morton_keys_interleave_bits():
    c = np.array([[0, 0, 0], [0, 0, 1], [0, 1, 0], [1, 0, 0], [1, 1, 1], [2, 0, 0], [0, 0, 2]])
    assert morton_keys(c).tolist() == [0, 1, 2, 4, 7, 32, 8]


def test_box_in_eight_parts_gives_octants():
    c = box_coords(4)
    owner = morton_partition(c, 8)
    for r in range(8):
        part = c[owner == r]
        assert len(part) == 8
        assert np.all(part.max(axis=0) - part.min(axis=0) == 1) and np.all(part.min(axis=0) % 2 == 0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16])
def test_partition_is_balanced_and_contiguous(n):
    c = random_sparse_problem(3, N=8, nblk_range=(200, 400)).coords[0]
    owner = morton_partition(c, n)
    counts = np.bincount(owner, minlength=n)
    assert counts.sum() == len(c) and counts.max() - counts.min() <= 1
    seq = owner[np.argsort(morton_keys(c), kind="stable")]
    assert np.all(np.diff(seq) >= 0)                      # each rank one Z-order chunk
    masks = shard_masks([c], 0, n)
    assert masks[0].sum() == counts[0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.flgf import FLGF
        from oracle.lgf import LGF
        p = config_plain_32()
        owned = shard_masks(p.coords, rank, world)[0]
        op = FLGF(LGF(), p.coords[0], p.N, 6)
        u = op.apply(p.f[0], h=p.h0, targets=np.nonzero(owned)[0])   # valid on owned blocks only
        whole = MR.assemble_owned(torch.as_tensor(u), owned).numpy()
        q.put((rank, int(owned.sum()), whole))
    finally:
        dist.destroy_process_group()


def test_two_ranks_sharded_solve_equals_single_rank_solve():
    from oracle.flgf import FLGF
    from oracle.lgf import LGF
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = dict((r, (n, u)) for r, n, u in (q.get(timeout=600) for _ in range(world)))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = config_plain_32()
    ref = FLGF(LGF(), p.coords[0], p.N, 6).apply(p.f[0], h=p.h0)
    assert res[0][0] + res[1][0] == len(p.coords[0]) and min(res[0][0], res[1][0]) > 0
    for r in range(world):
        assert np.max(np.abs(res[r][1] - ref)) <= 1e-15 * np.max(np.abs(ref))
