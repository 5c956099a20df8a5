"""Plan autotuner for the spectrum multiply-accumulate.

The launch lists of a block set fix two choices that decide how fast the
level interactions (Sec. 2.1) run on a given mesh:

* the dense tile, in parents, of the parent-group kernel (each thread owns the
  8 children of one parent; the tile's source region is staged in shared
  memory), and
* the useful-pair percentage below which a tile runs on the pair-list kernel
  instead (explicit (target, source) lists: no work on absent blocks, but two
  shared-memory reads per pair).

``autotune`` builds the block set under each candidate plan, times its solve
with CUDA events on the context's stream, and leaves the context on the
fastest plan (block sets created afterwards use it).  The plan changes the
order of floating-point sums only; every plan computes the same operator.
"""
from __future__ import annotations

import torch

from .flgf import BlockSet, Context, OPT_GRAPH

DEFAULT_CANDIDATES = [
    (30, (4, 4, 8)), (0, (4, 4, 8)), (15, (4, 4, 8)), (40, (4, 4, 8)), (50, (4, 4, 8)),
    (30, (4, 4, 4)), (50, (4, 4, 4)), (30, (2, 4, 8)),
]


def time_plan(ctx: Context, problems, h0, sources=None, reps: int = 3) -> float:
    """ms per solve of the block set under the context's current plan
    (graph-replayed after one warm-up solve)."""
    bs = BlockSet(ctx, problems, h0)
    try:
        if sources is not None:
            for p, levels in enumerate(sources):
                for l, f in enumerate(levels):
                    bs.load_source(p, l, f)
        else:
            for p, levels in enumerate(problems):
                for l in range(len(levels)):
                    bs.load_source(p, l, torch.zeros(bs._shape(p, l), dtype=ctx.dtype, device=ctx.device))
        bs.set_option(OPT_GRAPH, 1)
        bs.solve()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(ctx.device)
        e0.record(ctx.stream)
        for _ in range(reps):
            bs.solve()
        e1.record(ctx.stream)
        torch.cuda.synchronize(ctx.device)
        return e0.elapsed_time(e1) / reps
    finally:
        bs.close()


def autotune(ctx: Context, problems, h0, sources=None, candidates=None, reps: int = 3):
    """Time every candidate plan (list_pct, tile) on this mesh; set the fastest on
    ``ctx`` and return (best plan, {plan: ms per solve})."""
    cands = list(candidates or DEFAULT_CANDIDATES)
    table = {}
    for pct, tile in cands:
        ctx.set_plan(list_pct=pct, tile=tile)
        table[(pct, tuple(tile))] = time_plan(ctx, problems, h0, sources, reps)
    best = min(table, key=table.get)
    ctx.set_plan(list_pct=best[0], tile=best[1])
    return best, table
