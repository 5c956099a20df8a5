"""On-device refinement of a level (flgf_refine_level, Sec. 3.1 Eq. ref_crit)
against the oracle, element by element: flags, children and buffer blocks in
Morton order, bit-exact (integer output; the criterion is compared in FP64 on
both sides)."""
import numpy as np
import pytest
import torch

from oracle.meshgen import refine_level as oracle_refine
from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import box_coords, cell_centres, config_vortex_ring, vortex_ring

pytestmark = pytest.mark.gpu


def _random_level(seed, n, N, spread=40):
    rng = np.random.default_rng(seed)
    side = int(np.ceil((3 * n) ** (1 / 3))) + 1
    box = box_coords(side) + rng.integers(-spread, spread, size=3)
    c = box[np.sort(rng.choice(len(box), size=n, replace=False))]
    f = rng.standard_normal((n, N, N, N)) * rng.uniform(0, 2, size=(n, 1, 1, 1)) ** 4
    empty = rng.random(n) < 0.2
    empty[0] = False               # some empty blocks, never all of them
    f[empty] = 0.0
    return c, f


def _check(ctx, c, f, rel):
    flags, ch, buf = ctx.refine_level(torch.as_tensor(f), c, rel)
    # the oracle sees the source in the context precision, as the device does
    fr = torch.as_tensor(f).to(ctx.dtype).double().numpy()
    of, och, obuf = oracle_refine(c, fr, rel)
    assert np.array_equal(flags.cpu().numpy(), of)
    assert np.array_equal(ch.cpu().numpy(), och)
    assert np.array_equal(buf.cpu().numpy(), obuf)
    return int(of.sum()), len(obuf)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("n,rel", [(1, 0.5), (7, 0.3), (300, 0.05), (5000, 0.2)])
def test_random_levels_match_oracle(precision, n, rel):
    ctx = F.Context(N=8, n_interp=6, precision=precision)
    c, f = _random_level(n, n, 8)
    nflag, nbuf = _check(ctx, c, f, rel)
    assert nflag >= 1
    ctx.close()


def test_vortex_ring_base_level_and_many_tiles():
    """The vortex ring's base level with Eq. ref_crit's alpha = 1/32 over three
    levels (rel = alpha^2), and a 16^3 level whose 26-neighbour candidates
    (about 10^5) span over a hundred scan tiles of 1024."""
    p, _ = config_vortex_ring(3, 8, 4, 0)
    ctx = F.Context(N=8, n_interp=6, precision="fp32")
    base = np.asarray(p.coords[0])
    f = vortex_ring(cell_centres(base, 8, p.h0))[1]
    nflag, _ = _check(ctx, base, f, (1.0 / 32) ** 2)
    assert nflag > 0
    big = box_coords(16) - 8
    fb = np.random.default_rng(1).standard_normal((len(big), 8, 8, 8))
    nflag, nbuf = _check(ctx, big, fb, 0.5)
    assert nflag > 3000 and nbuf > 0
    ctx.close()


def test_edge_cases():
    ctx = F.Context(N=8, n_interp=6, precision="fp32")
    c = box_coords(2)
    flags, ch, buf = ctx.refine_level(torch.zeros((8, 8, 8, 8)), c, 0.1)
    assert not flags.any() and ch.shape == (0, 3) and buf.shape == (0, 3)
    f = torch.zeros((8, 8, 8, 8))
    f[2, 1, 1, 1] = 3.0
    flags, _, _ = ctx.refine_level(f, c, 1.0)   # strict comparison: nothing exceeds the maximum itself
    assert not flags.any()
    with pytest.raises(F.FLGFError) as ei:   # children would not fit the Morton keys
        ctx.refine_level(torch.ones((1, 8, 8, 8)), [[1 << 19, 0, 0]], 0.5)
    assert ei.value.code == F.FLGF_EINVAL
    with pytest.raises(ValueError):
        ctx.refine_level(torch.ones((2, 8, 8, 8)), c, 0.5)   # shape mismatch
    # the context still works after a refused call
    flags, ch, _ = ctx.refine_level(f, c, 0.5)
    assert flags.sum() == 1 and ch.shape == (8, 3)
    ctx.close()
