"""Vector Poisson problem: the Cartesian components of the vortex ring's
streamfunction (Sec. 3.1) solved together as problems of one block set, each
equal to its own scalar solve and to the analytic field."""
import numpy as np
import pytest
import torch

from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import config_vortex_ring, vortex_ring_vector, cell_centres

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vortex_ring_vector_solve(precision):
    p, _ = config_vortex_ring(3, 8, 4, 0)
    N = p.N
    pw = [vortex_ring_vector(cell_centres(c, N, p.h0 / (1 << l))) for l, c in enumerate(p.coords)]
    comps = [[w[..., a] for _, w in pw] for a in range(3)]
    exact = [[ps[..., a] for ps, _ in pw] for a in range(3)]
    c = F.Context(N=N, n_interp=6, precision=precision)
    vec = F.solve_vector(c, p.coords, p.h0, comps)
    leaf = p.leaf_masks()
    scale = max(np.max(np.abs(e[l][leaf[l]])) for e in exact[:2] for l in range(p.n_levels))
    for a in range(3):
        one = F.solve_problem(c, type(p)(N=N, h0=p.h0, coords=p.coords, f=comps[a]))
        for l in range(p.n_levels):
            u = vec[a][l].cpu().numpy()
            assert np.array_equal(u, one[l].cpu().numpy())        # same launches, same sums
            err = np.max(np.abs(u[leaf[l]] - exact[a][l][leaf[l]])) / scale
            assert err < 1e-2, (a, l, err)                        # 9.1e-3 at this resolution
        if a == 2:
            assert all(float(x.abs().max()) == 0.0 for x in vec[a])  # zero source, zero field
    c.close()


def test_vector_block_set_matches_scalar_solves_n16():
    """FP32, 16^3 blocks: the three components through the component-sharing
    spectrum products equal three scalar solves bit for bit (the per-frequency
    sums are the same operations in the same order), with every problem
    layout the planner produces: dense tiles only, and dense tiles beside
    pair lists."""
    p, _ = config_vortex_ring(3, 16, 4, 0)
    N = p.N
    pw = [vortex_ring_vector(cell_centres(c, N, p.h0 / (1 << l))) for l, c in enumerate(p.coords)]
    rng = np.random.default_rng(3)
    # component 2 gets a random source so that no component is trivially zero
    comps = [[w[..., a] for _, w in pw] for a in range(2)] + [[rng.standard_normal(w.shape[:-1]) for _, w in pw]]
    c = F.Context(N=N, n_interp=6, precision="fp32")
    for pct in (0, 30):
        c.set_plan(list_pct=pct, tile=(4, 4, 8))
        vec = F.solve_vector(c, p.coords, p.h0, comps)
        for a in range(3):
            one = F.solve_problem(c, type(p)(N=N, h0=p.h0, coords=p.coords, f=comps[a]))
            for l in range(p.n_levels):
                assert torch.equal(vec[a][l], one[l]), (pct, a, l)
    with pytest.raises(ValueError):
        F.BlockSet(c, [p.coords, p.coords[:1]], [p.h0, p.h0], vector=True)
    c.close()
