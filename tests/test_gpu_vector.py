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
