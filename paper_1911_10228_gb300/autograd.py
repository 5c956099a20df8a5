"""torch.autograd integration: the FLGF solve as a differentiable function.

``solve(bs, sources)`` maps the source tensors of every (problem, level) of a
block set to the potentials; its backward pass is the library's adjoint solve
(``flgf_solve_adjoint``, its own launch sequence), so gradients of any loss of
the potentials flow back to the sources.  Source values on non-leaf blocks are
ignored by the solve and receive zero gradient.
"""
from __future__ import annotations

import torch

from .flgf import BlockSet


class FLGFSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, bs: BlockSet, *sources):
        keys = bs.keys()
        if len(sources) != len(keys):
            raise ValueError(f"expected {len(keys)} source tensors (one per problem and level)")
        for (p, l), f in zip(keys, sources):
            bs.load_source(p, l, f.detach())
        bs.solve()
        ctx.bs = bs
        ctx.dtypes = [f.dtype for f in sources]
        return tuple(bs.potential(p, l) for p, l in keys)

    @staticmethod
    def backward(ctx, *grads):
        bs = ctx.bs
        keys = bs.keys()
        for (p, l), g in zip(keys, grads):
            if g is None:
                g = torch.zeros(bs._shape(p, l), dtype=bs.ctx.dtype, device=bs.ctx.device)
            bs.load_adjoint(p, l, g)
        bs.solve_adjoint()
        out = [bs.gradient(p, l).to(dt) for (p, l), dt in zip(keys, ctx.dtypes)]
        return (None,) + tuple(out)


def solve(bs: BlockSet, sources):
    """Differentiable solve: sources in ``bs.keys()`` order -> potentials in the same order."""
    return FLGFSolve.apply(bs, *sources)
