"""Pins of the uniform FLGF oracle (Sec. 2.1)."""
import numpy as np
import pytest

from oracle.conv import direct_sum, hockney
from oracle.flgf import FLGF, Octree, blocks_to_dense, dense_to_blocks, lagrange_J1
from paper_1911_10228_gb300.inputs import box_coords, config_plain_32


@pytest.mark.parametrize("N,nI", [(8, 6), (16, 6), (8, 4), (16, 10), (8, 5)])
def test_lagrange_reproduces_polynomials(N, nI):
    """Lagrange interpolation on n_I nodes is exact for degree < n_I
    (child nodes at j + 1/2, parent nodes at 2p + 1)."""
    J = lagrange_J1(N, nI)
    xc = np.arange(2 * N) + 0.5
    xp = 2.0 * np.arange(N) + 1.0
    for deg in range(nI):
        p = lambda x: ((x - 7.3) / N) ** deg
        assert np.max(np.abs(J @ p(xp) - p(xc))) < 1e-11 * max(1.0, np.max(np.abs(p(xc))))
    # mirror symmetry of the node layout: J[2N-1-j, N-1-p] = J[j, p]
    assert np.allclose(J[::-1, ::-1], J, rtol=0, atol=1e-14)
    # each child row uses n_I consecutive parent nodes
    assert np.all(np.count_nonzero(np.abs(J) > 0, axis=1) <= nI)


def test_lagrange_interior_weights_quarter_offset():
    """Interior child nodes sit a quarter parent spacing from the nearest parent
    node; the centred 6-point weights are the Lagrange basis at +1/4 on nodes
    at -5/2 .. 5/2 (units of the parent spacing), written out independently here."""
    J = lagrange_J1(16, 6)
    w = J[10, 2:8]  # child x = 10.5 between parent nodes 9 (p = 4) and 11 (p = 5)
    t = np.array([-2.5, -1.5, -0.5, 0.5, 1.5, 2.5]) * 2.0  # node offsets from x' = 10 (child units)
    xq = 0.5                                             # child at 10.5 relative to 10
    ref = [np.prod([(xq - t[q]) / (t[m] - t[q]) for q in range(6) if q != m]) for m in range(6)]
    assert np.allclose(w, ref, rtol=0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-15


def test_every_pair_handled_once():
    """Near list + influence lists on all levels partition all (target, source) pairs."""
    rng = np.random.default_rng(0)
    allc = box_coords(12)
    coords = allc[np.sort(rng.choice(len(allc), 300, replace=False))]
    tr = Octree(coords)
    nb = coords.shape[0]
    for t in rng.choice(nb, 25, replace=False):
        seen = np.zeros(nb, dtype=int)
        for j in tr.near(t):
            seen[j] += 1
        for k in range(tr.top + 1):
            anc = tuple(int(v) for v in coords[t] >> k)
            i = tr.index[k][anc]
            for j in tr.influence(k, i):
                key = tr.levels[k][j]
                desc = np.all((coords >> k) == key[None, :], axis=1)
                seen[desc] += 1
        assert np.all(seen == 1)


def test_single_level_tree_equals_direct_sum(G):
    """The 32^3 workload (4^3 blocks of 8^3) has top level = finest level: every
    interaction is an exact block convolution, so FLGF = Eq. discretConv."""
    p = config_plain_32()
    op = FLGF(G, p.coords[0], p.N, 6)
    assert op.tree.top == 0
    u = op.apply(p.f[0])
    dense, org = blocks_to_dense(p.coords[0], p.f[0], p.N)
    ax = [np.arange(s) for s in dense.shape]
    pts = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1).reshape(-1, 3)
    rng = np.random.default_rng(5)
    tg = pts[rng.choice(len(pts), 400, replace=False)]
    ud = direct_sum(G, pts, dense.ravel(), tg)
    ub = dense_to_blocks(*(lambda x: (x, org))(np.zeros_like(dense)), p.coords[0], p.N)
    uf = np.zeros_like(dense)
    for b, c in enumerate(p.coords[0]):
        o = c * p.N
        uf[o[0]:o[0] + 8, o[1]:o[1] + 8, o[2]:o[2] + 8] = u[b]
    got = uf[tg[:, 0], tg[:, 1], tg[:, 2]]
    assert np.max(np.abs(got - ud)) < 1e-12 * np.max(np.abs(ud))


def test_operator_is_symmetric(G):
    """K is symmetric (G(n) = G(-n)) and R = J^T, so <A f, g> = <f, A g>."""
    rng = np.random.default_rng(7)
    coords = box_coords(6)
    coords = coords[rng.random(len(coords)) < 0.7]
    op = FLGF(G, coords, 4, 4)
    assert op.tree.top >= 1
    f = rng.standard_normal((len(coords), 4, 4, 4))
    g = rng.standard_normal((len(coords), 4, 4, 4))
    a = np.sum(op.apply(f) * g)
    b = np.sum(f * op.apply(g))
    assert abs(a - b) < 1e-12 * abs(a)


def test_interpolation_error_vs_exact(G):
    """FMM error against the exact free-space convolution is small and falls with n_I
    (measured, the paper prints no n_I = 6 bound; ~1e-12 claimed only for n_I <= 10)."""
    N, nb = 4, 8
    coords = box_coords(nb)
    x = np.arange(nb * N) + 0.5
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    c = nb * N / 2
    dense = np.exp(-((X - c) ** 2 + (Y - c - 2) ** 2 + (Z - c + 1) ** 2) / (2 * 4.0 ** 2))
    f = dense_to_blocks(dense, np.zeros(3, int), coords, N)
    ub = dense_to_blocks(hockney(G, dense), np.zeros(3, int), coords, N)
    errs = []
    for nI in (2, 4):
        u = FLGF(G, coords, N, nI).apply(f)
        errs.append(np.max(np.abs(u - ub)) / np.max(np.abs(ub)))
    assert errs[1] < errs[0] and errs[1] < 1e-3, errs


def test_target_subset_matches_full(G):
    rng = np.random.default_rng(9)
    coords = box_coords(6)
    f = rng.standard_normal((len(coords), 4, 4, 4))
    op = FLGF(G, coords, 4, 4)
    full = op.apply(f)
    sub = [3, 50, 100]
    part = op.apply(f, targets=sub)
    assert np.allclose(part[sub], full[sub], rtol=0, atol=1e-14 * np.abs(full).max())
