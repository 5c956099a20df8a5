"""Pins of the oracle's adjoint: dot-product identities and finite differences."""
import numpy as np

from oracle.adjoint import flgf_transpose, multires_adjoint
from oracle.flgf import FLGF
from oracle.multires import multires_solve
from paper_1911_10228_gb300.inputs import box_coords


def _sparse(n, keep, seed):
    rng = np.random.default_rng(seed)
    c = box_coords(n)
    return c[rng.random(len(c)) < keep]


def test_fmm_transpose_dot_product(G):
    coords = _sparse(7, 0.6, 1)
    op = FLGF(G, coords, 4, 4)
    assert op.tree.top >= 1
    rng = np.random.default_rng(2)
    f = rng.standard_normal((len(coords), 4, 4, 4))
    g = rng.standard_normal((len(coords), 4, 4, 4))
    a = np.sum(op.apply(f, h=0.3) * g)
    b = np.sum(f * flgf_transpose(op, g, h=0.3))
    assert abs(a - b) < 1e-12 * abs(a)


def _three_level(N=4):
    c0 = box_coords(6)
    r0 = c0[np.all((c0 >= 2) & (c0 <= 3), axis=1)]
    c1 = np.concatenate([2 * r0 + np.array(a) for a in np.ndindex(2, 2, 2)])
    # refine a 2x2x2 corner of level 1 that keeps its 26-neighbour buffer
    r1 = c1[np.all((c1 >= 5) & (c1 <= 6), axis=1)]
    c2 = np.concatenate([2 * r1 + np.array(a) for a in np.ndindex(2, 2, 2)])
    return [c0, c1, c2]


def test_multires_adjoint_dot_product(G):
    levels = _three_level()
    rng = np.random.default_rng(3)
    f = [rng.standard_normal((len(c), 4, 4, 4)) for c in levels]
    g = [rng.standard_normal((len(c), 4, 4, 4)) for c in levels]
    for corr in (True, False):
        u, leaf = multires_solve(G, levels, f, 4, 4, 0.25, correction=corr)
        fl = [np.where(m[:, None, None, None], x, 0.0) for x, m in zip(f, leaf)]
        a = sum(np.sum(x * y) for x, y in zip(u, g))
        gf = multires_adjoint(G, levels, g, 4, 4, 0.25, correction=corr)
        b = sum(np.sum(x * y) for x, y in zip(fl, gf))
        assert abs(a - b) < 1e-11 * abs(a), (corr, a, b)
        for x, m in zip(gf, leaf):
            assert np.all(x[~m] == 0.0)


def test_gradient_matches_finite_differences(G):
    """loss = 0.5 ||u_leaf - t||^2 is quadratic in f, so central differences are
    exact up to round-off."""
    levels = _three_level()
    rng = np.random.default_rng(4)
    f = [rng.standard_normal((len(c), 4, 4, 4)) for c in levels]
    t = [rng.standard_normal((len(c), 4, 4, 4)) for c in levels]
    u, leaf = multires_solve(G, levels, f, 4, 4, 0.25)
    lm = [m[:, None, None, None] for m in leaf]

    def loss(ff):
        uu, _ = multires_solve(G, levels, ff, 4, 4, 0.25)
        return 0.5 * sum(np.sum(np.where(m, x - y, 0.0) ** 2) for x, y, m in zip(uu, t, lm))

    g = [np.where(m, x - y, 0.0) for x, y, m in zip(u, t, lm)]
    grad = multires_adjoint(G, levels, g, 4, 4, 0.25)
    step = 1e-3
    for l, b, i, j, k in [(0, 5, 1, 2, 3), (1, 3, 0, 0, 0), (2, 7, 3, 1, 2), (1, 20, 2, 2, 1)]:
        if not leaf[l][b]:
            continue
        fp = [x.copy() for x in f]
        fm = [x.copy() for x in f]
        fp[l][b, i, j, k] += step
        fm[l][b, i, j, k] -= step
        fd = (loss(fp) - loss(fm)) / (2 * step)
        assert abs(fd - grad[l][b, i, j, k]) < 1e-7 * max(1.0, abs(fd)), (l, b, fd, grad[l][b, i, j, k])
