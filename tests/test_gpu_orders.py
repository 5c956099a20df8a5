"""Parity of the N = 16 paths and of other Lagrange orders n_I with the oracle."""
import numpy as np
import pytest

from oracle.flgf import FLGF
from oracle.multires import multires_solve
from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import Problem, box_coords, cell_centres, gaussians

pytestmark = pytest.mark.gpu

_REF = {}


def rel(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def _gauss(coords, N, h0):
    x = cell_centres(coords, N, h0)
    ext = (coords.max(axis=0) + 1) * N * h0
    return gaussians(x, [0.5 * ext, 0.45 * ext], [0.12 * ext[0], 0.08 * ext[0]], [1.0, -0.6])


@pytest.mark.parametrize("N,nI", [(16, 10), (16, 8), (16, 4), (8, 3), (8, 8)])
def test_uniform_orders_match_oracle(G, N, nI):
    coords = box_coords(6 if N == 16 else 8)
    f = _gauss(coords, N, 1.0)
    key = (N, nI)
    if key not in _REF:
        _REF[key] = FLGF(G, coords, N, nI).apply(f)
    ctx = F.Context(N=N, n_interp=nI, precision="fp64")
    u = F.solve_problem(ctx, Problem(N=N, h0=1.0, coords=[coords], f=[f]))[0].cpu().numpy()
    ctx.close()
    assert rel(u, _REF[key]) < 1e-10


@pytest.mark.parametrize("nI", [6, 10])
def test_multires_n16_matches_oracle(G, nI):
    N = 16
    h0 = 1.0 / (4 * N)
    c0 = box_coords(4)
    ref = c0[np.all((c0 >= 1) & (c0 <= 2), axis=1)]
    c1 = np.concatenate([2 * ref + np.array(a) for a in np.ndindex(2, 2, 2)])
    c1 = c1[np.lexsort(c1.T[::-1])]
    src = lambda x: gaussians(x, [(0.52, 0.47, 0.5)], [0.06], [1.0])
    p = Problem(N=N, h0=h0, coords=[c0, c1], f=[src(cell_centres(c0, N, h0)), src(cell_centres(c1, N, h0 / 2))])
    ctx = F.Context(N=N, n_interp=nI, precision="fp64")
    u = [x.cpu().numpy() for x in F.solve_problem(ctx, p)]
    ctx.close()
    ref, leaf = multires_solve(G, p.coords, p.f, N, nI, h0)
    for l in range(2):
        assert rel(u[l][leaf[l]], ref[l][leaf[l]]) < 1e-10, l
