"""Pins of the block-refined scheme's oracle (Sec. 3)."""
import numpy as np

from oracle.flgf import FLGF
from oracle.multires import (Level, coarsen, interp_coarse_to_fine, laplacian_on_level,
                             leaf_masks, multires_solve)
from paper_1911_10228_gb300.inputs import box_coords, cell_centres, gaussians


def _two_level(N=4):
    c0 = box_coords(4)
    ref = c0[np.all((c0 >= 1) & (c0 <= 2), axis=1)]
    c1 = np.concatenate([2 * ref + np.array(a) for a in np.ndindex(2, 2, 2)])
    c1 = c1[np.lexsort(c1.T[::-1])]
    return c0, c1


def _src(coords, N, h):
    x = cell_centres(coords, N, h)
    return gaussians(x, [(8.3, 7.9, 8.1)], [2.0], [1.0])


def test_single_level_is_uniform_flgf(G):
    rng = np.random.default_rng(0)
    c = box_coords(5)
    f = rng.standard_normal((len(c), 4, 4, 4))
    u, leaf = multires_solve(G, [c], [f], 4, 4, h0=0.3)
    ref = FLGF(G, c, 4, 4).apply(f, h=0.3)
    assert np.array_equal(u[0], ref)


def test_coarse_fine_interp_exact_for_quadratics():
    N = 4
    c0 = box_coords(3)
    lv = Level(c0, N)
    q = lambda x: 0.3 * x[..., 0] ** 2 - x[..., 1] * x[..., 2] + 2.0 * x[..., 2] - 1.0
    u0 = q(cell_centres(c0, N, 1.0))
    fine_blk = np.array([[2, 3, 2]])  # a child of the centre block (1,1,1)
    xf = cell_centres(fine_blk, N, 0.5)
    ax = np.arange(N)
    cells = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1) + fine_blk[0] * N
    got = interp_coarse_to_fine(lv, u0, cells)
    assert np.max(np.abs(got - q(xf[0]))) < 1e-12


def test_coarsening_is_mean_and_exact_for_linear():
    N = 4
    cc = np.array([[0, 0, 0]])
    fine = np.concatenate([np.array([a]) for a in np.ndindex(2, 2, 2)])
    lin = lambda x: 1.5 * x[..., 0] - 0.5 * x[..., 1] + 0.25 * x[..., 2] + 2.0
    ff = lin(cell_centres(fine, N, 0.5))
    out = coarsen(Level(fine, N), ff, cc, np.array([True]))
    assert np.max(np.abs(out[0] - lin(cell_centres(cc, N, 1.0))[0])) < 1e-13


def _leaf_interior(levels, u, leaf, l, N):
    lv = Level(levels[l], N)
    ind = np.broadcast_to(leaf[l][:, None, None, None], u[l].shape).astype(float)
    lapi, mask = laplacian_on_level(lv, ind, 1.0)
    return mask & (ind == 1) & (np.abs(lapi) < 1e-12)


def test_source_correction_restores_consistency(G):
    """With the correction L_Q^{(h_l)} u = f holds on the leaf interior of every
    level (to round-off here: each level's tree has one octree level, so the
    convolutions are exact); without it the finer level is inconsistent."""
    N = 4
    c0, c1 = _two_level(N)
    f0, f1 = _src(c0, N, 1.0), _src(c1, N, 0.5)
    errs = {}
    for corr in (True, False):
        u, leaf = multires_solve(G, [c0, c1], [f0, f1], N, 4, 1.0, correction=corr)
        for l, ff in enumerate((f0, f1)):
            lap, _ = laplacian_on_level(Level([c0, c1][l], N), u[l], 1.0 / (1 << l))
            ok = _leaf_interior([c0, c1], u, leaf, l, N)
            errs[corr, l] = np.max(np.abs(lap - ff)[ok]) / np.max(np.abs(ff))
    assert errs[True, 0] < 1e-11 and errs[True, 1] < 1e-11, errs
    # without the correction the finer level is inconsistent by orders of magnitude
    assert errs[False, 1] > 1e-3 and errs[False, 1] > 1e6 * errs[True, 1], errs


def test_leaf_masks_reject_partial_refinement():
    c0 = box_coords(2)
    c1 = np.array([[0, 0, 0], [0, 0, 1]])
    try:
        leaf_masks([c0, c1])
    except ValueError:
        return
    raise AssertionError("partial refinement accepted")


def test_two_level_solution_matches_uniform_fine_solution(G):
    """Sec. 3.1: refinement keeps the target field close to the fine-lattice
    solution, and the source correction changes it only slightly.  The
    two-level solution on the refined blocks must agree with the free-space
    solution computed on the whole fine lattice (one Hockney convolution at the
    fine spacing), with and without the correction.  A reading that makes the
    interpolated coarse field jump at the coarse-fine interface fails this by
    orders of magnitude."""
    from oracle.conv import hockney
    N = 8
    h0 = 1.0 / (4 * N)
    c0 = box_coords(4)
    ref = c0[np.all((c0 >= 1) & (c0 <= 2), axis=1)]
    c1 = np.concatenate([2 * ref + np.array(a) for a in np.ndindex(2, 2, 2)])
    src = lambda x: gaussians(x, [(0.5, 0.49, 0.51)], [0.07], [1.0])
    f0, f1 = src(cell_centres(c0, N, h0)), src(cell_centres(c1, N, h0 / 2))
    hf = h0 / 2
    ax = (np.arange(8 * N) + 0.5) * hf
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    uf = hockney(G, src(np.stack([X, Y, Z], -1)), h=hf)
    cells = np.stack(np.meshgrid(*[np.arange(N)] * 3, indexing="ij"), -1)
    g = c1[:, None, None, None, :] * N + cells[None]
    exact = uf[g[..., 0], g[..., 1], g[..., 2]]
    sols = {}
    for corr in (True, False):
        u, _ = multires_solve(G, [c0, c1], [f0, f1], N, 4, h0, correction=corr)
        sols[corr] = u[1]
        assert np.max(np.abs(u[1] - exact)) / np.max(np.abs(exact)) < 5e-3, corr
    assert np.max(np.abs(sols[True] - sols[False])) / np.max(np.abs(exact)) < 5e-3
