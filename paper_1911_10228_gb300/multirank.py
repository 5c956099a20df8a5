"""Host-side logic of multi-process runs (one process per GPU).

The solver itself needs no exchange between GPUs during a solve: the batched
form is a set of independent problems, so a job of ``world`` ranks gives each
rank its own disjoint slice of problems, and a single solve sharded by target
blocks (``shard.py``) has every rank compute its own targets from the
replicated source.  What the ranks share is bookkeeping -- a barrier around
the timed region, the maximum of the ranks' timings, the sum of the work they
did -- and, when one rank needs the whole field of a sharded solve, one
summation of the owned blocks after it.  These helpers work with any initialised
``torch.distributed`` backend (NCCL on GPUs, gloo on CPUs) and reduce to the
plain value in a single-process run.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def _reduce(x: float, op, device) -> float:
    if not active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def all_max(x: float, device="cpu") -> float:
    """Maximum over ranks (the job's time is its slowest rank's)."""
    return _reduce(x, dist.ReduceOp.MAX, device)


def all_sum(x: float, device="cpu") -> float:
    """Sum over ranks (the job's work is every rank's work)."""
    return _reduce(x, dist.ReduceOp.SUM, device)


def barrier(device=None):
    if active():
        if device is not None and torch.device(device).type == "cuda":
            dist.barrier(device_ids=[torch.device(device).index or 0])
        else:
            dist.barrier()


def problem_seeds(per_rank: int, rank: int) -> list[int]:
    """Seeds of this rank's problems in a job of per_rank problems per rank:
    rank r takes seeds [r * per_rank, (r + 1) * per_rank), so the ranks' slices
    are disjoint, and rank 0 alone reproduces the single-GPU batch."""
    if per_rank < 0 or rank < 0:
        raise ValueError("per_rank and rank must be non-negative")
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def assemble_owned(u: torch.Tensor, owned) -> torch.Tensor:
    """Whole field of a solve sharded by blocks: every rank passes its field
    (nb, ...) and the boolean mask (nb,) of the blocks it owns; the blocks are
    owned by exactly one rank each, so zeroing the others and summing over the
    ranks returns every block from its owner, on every rank."""
    m = torch.as_tensor(owned, dtype=torch.bool, device=u.device).reshape(-1, *([1] * (u.dim() - 1)))
    out = torch.where(m, u, torch.zeros_like(u))
    if active():
        dist.all_reduce(out, op=dist.ReduceOp.SUM)
    return out
