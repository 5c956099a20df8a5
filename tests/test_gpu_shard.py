"""A solve sharded by target blocks, on one GPU: block sets that each want a
disjoint Morton chunk of the blocks (flgf_blockset_create_masked) reproduce,
on their own blocks, the unmasked solve -- uniform and refined meshes, FP64
and FP32 -- and split the spectrum products of the targets between them."""
import numpy as np
import pytest
import torch

from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import box_coords, config_plain_32, refine_mesh, torus
from paper_1911_10228_gb300.shard import shard_masks

pytestmark = pytest.mark.gpu


def _solve(ctx, p, want=None):
    bs = F.BlockSet(ctx, [p.coords], [p.h0], want=None if want is None else [want])
    for l, f in enumerate(p.f):
        bs.load_source(0, l, torch.as_tensor(f))
    bs.solve()
    u = [bs.potential(0, l).double().cpu().numpy() for l in range(p.n_levels)]
    pairs = bs.work_counts()["pairs"]
    bs.close()
    return u, pairs


def _mesh():
    return refine_mesh(lambda x: torus(x, (0.5, 0.5, 0.5), 0.22, 0.05), box_coords(4), 8, 1.0 / 32, 3, 0.3)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["uniform", "refined"])
def test_sharded_solve_matches_whole_solve(case, precision, world):
    p = config_plain_32() if case == "uniform" else _mesh()
    ctx = F.Context(N=8, n_interp=6, precision=precision)
    ref, full_pairs = _solve(ctx, p)
    scale = max(np.max(np.abs(r)) for r in ref)
    covered = [np.zeros(len(c), int) for c in p.coords]
    shard_pairs = 0
    for rank in range(world):
        want = shard_masks(p.coords, rank, world)
        u, pairs = _solve(ctx, p, want)
        shard_pairs += pairs
        for l in range(p.n_levels):
            covered[l] += want[l]
            d = np.abs(u[l][want[l]] - ref[l][want[l]])
            # the same launch lists restricted to fewer targets: equal up to the
            # order in which the MAC kernels' groups are formed
            assert d.size == 0 or np.max(d) <= (1e-13 if precision == "fp64" else 1e-6) * scale, (rank, l)
    assert all(np.all(c == 1) for c in covered)
    if case == "uniform":
        assert shard_pairs == full_pairs          # every interaction on exactly one rank
    ctx.close()


def test_masked_block_set_refuses_the_adjoint():
    p = config_plain_32()
    ctx = F.Context(N=8, n_interp=6, precision="fp64")
    bs = F.BlockSet(ctx, [p.coords], [p.h0], want=[shard_masks(p.coords, 0, 2)])
    with pytest.raises(F.FLGFError) as ei:
        bs.load_adjoint(0, 0, torch.zeros((len(p.coords[0]), 8, 8, 8), dtype=torch.float64))
    assert ei.value.code == F.FLGF_ESTATE
    bs.close()
    ctx.close()
