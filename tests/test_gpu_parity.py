"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative to the max |reference| of the compared field):
FP64 path 1e-10, FP32 path 1e-5 (both against the FP64 oracle).
"""
import numpy as np
import pytest
import torch

from oracle.conv import direct_sum
from oracle.flgf import FLGF, kernel_block
from oracle.multires import Level, laplacian_on_level, multires_solve
from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import (Problem, box_coords, cell_centres, config_plain_32, gaussians,
                                           refine_mesh, torus)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


_CTX = {}
_ORACLE = {}


def cached(key, fn):
    """Oracle results are shared by the FP64 and FP32 cases of a test."""
    if key not in _ORACLE:
        _ORACLE[key] = fn()
    return _ORACLE[key]


def ctx(N=8, precision="fp64", n_interp=6):
    key = (N, precision, n_interp)
    if key not in _CTX:
        _CTX[key] = F.Context(N=N, n_interp=n_interp, precision=precision)
    return _CTX[key]


def gpu_solve(c, prob, correction=True):
    out = F.solve_problem(c, prob, correction=correction)
    return [u.double().cpu().numpy() for u in out]


def test_lgf_values_match_oracle(G):
    c = ctx(8, "fp64")
    rng = np.random.default_rng(0)
    pts = rng.integers(-100, 101, (400, 3))
    pts = np.concatenate([pts, [[0, 0, 0], [1, 0, 0], [100, 0, 0], [101, 0, 0], [60, 60, 50], [600, 0, 0],
                                [601, 0, 0], [-350, 350, 341], [2000, -5, 7]]])
    got = c.lgf(pts)
    ref = G(pts)
    assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k,d", [(0, (0, 0, 0)), (0, (1, -2, 3)), (1, (-3, -3, -3)), (2, (2, 0, -1))])
def test_kernel_spectra_match_oracle(G, precision, k, d):
    c = ctx(8, precision)
    got = c.kernel_spectrum(k, d)
    ref = np.fft.rfftn(kernel_block(G, 8, k, d), axes=(0, 1, 2))
    tol = 1e-13 if precision == "fp64" else 2e-7
    assert rel_err(got.real, ref.real) < tol and np.max(np.abs(got.imag - ref.imag)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plain_32_equals_direct_sum(G, precision):
    """4^3 blocks of 8^3: one octree level, every interaction an exact block
    convolution, so the result is Eq. discretConv itself."""
    p = config_plain_32()
    u = gpu_solve(ctx(8, precision), p)[0]
    ref = cached("plain32", lambda: FLGF(G, p.coords[0], 8, 6).apply(p.f[0]))
    assert rel_err(u, ref) < TOL[precision]
    # and directly against the brute-force sum at sampled cells
    rng = np.random.default_rng(1)
    cells = np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3)
    src_pts = (p.coords[0][:, None, :] * 8 + cells[None]).reshape(-1, 3)
    pick = rng.choice(src_pts.shape[0], 200, replace=False)
    ud = cached("plain32_direct", lambda: direct_sum(G, src_pts, p.f[0].reshape(-1), src_pts[pick]))
    assert rel_err(u.reshape(-1)[pick], ud) < TOL[precision]


def _gauss_problem(coords, N, seed, h0=1.0):
    rng = np.random.default_rng(seed)
    ext = (coords.max(axis=0) + 1) * N
    cen = rng.uniform(0.3, 0.7, (3, 3)) * ext
    x = cell_centres(coords, N, 1.0)
    f = gaussians(x, cen, rng.uniform(2.0, 5.0, 3), rng.uniform(-1, 1, 3))
    return Problem(N=N, h0=h0, coords=[coords], f=[f])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_uniform_fmm_matches_oracle(G, precision):
    """Dense 8^3 blocks of 8^3 (two octree levels, Lagrange n_I = 6)."""
    p = _gauss_problem(box_coords(8), 8, 2, h0=0.5)
    u = gpu_solve(ctx(8, precision), p)[0]
    ref = cached("uniform8", lambda: FLGF(G, p.coords[0], 8, 6).apply(p.f[0], h=0.5))
    assert rel_err(u, ref) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sparse_ragged_blockset_matches_oracle(G, precision):
    """Random 35 % of a 10^3 block box, offset origin: ragged tiles, missing
    sources and targets, three octree levels."""
    rng = np.random.default_rng(3)
    allc = box_coords(10, origin=(-3, 5, 2))
    coords = allc[np.sort(rng.choice(len(allc), 350, replace=False))]
    p = _gauss_problem(coords - coords.min(axis=0), 8, 4)
    p.coords[0] = coords
    op = FLGF(G, coords, 8, 6)
    assert op.tree.top == 2
    u = gpu_solve(ctx(8, precision), p)[0]
    assert rel_err(u, cached("sparse", lambda: op.apply(p.f[0]))) < TOL[precision]


def _two_level(N=8):
    h0 = 1.0 / (4 * N)
    src = lambda x: gaussians(x, [(0.52, 0.47, 0.5)], [0.08], [1.0])
    c0 = box_coords(4)
    ref = c0[np.all((c0 >= 1) & (c0 <= 2), axis=1)]
    c1 = np.concatenate([2 * ref + np.array(a) for a in np.ndindex(2, 2, 2)])
    c1 = c1[np.lexsort(c1.T[::-1])]
    f0 = src(cell_centres(c0, N, h0))
    f1 = src(cell_centres(c1, N, h0 / 2))
    return Problem(N=N, h0=h0, coords=[c0, c1], f=[f0, f1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("correction", [True, False])
def test_multires_two_levels_matches_oracle(G, precision, correction):
    p = _two_level()
    u = gpu_solve(ctx(8, precision), p, correction=correction)
    ref, leaf = cached(("mr2", correction), lambda: multires_solve(G, p.coords, p.f, 8, 6, p.h0, correction=correction))
    for l in range(2):
        assert rel_err(u[l][leaf[l]], ref[l][leaf[l]]) < TOL[precision], l


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multires_three_levels_matches_oracle(G, precision):
    """Torus source on a 4^3 base of 8^3 blocks with two refinements (closed
    buffer, interior levels with leaf and non-leaf blocks)."""
    N = 8
    h0 = 1.0 / (4 * N)
    p = refine_mesh(lambda x: torus(x, (0.5, 0.5, 0.5), 0.22, 0.05), box_coords(4), N, h0, 3, 0.3)
    assert p.n_levels == 3 and len(p.coords[2]) > 0
    u = gpu_solve(ctx(N, precision), p)
    ref, leaf = cached("mr3", lambda: multires_solve(G, p.coords, p.f, N, 6, p.h0))
    for l in range(3):
        assert rel_err(u[l][leaf[l]], ref[l][leaf[l]]) < TOL[precision], l


def test_laplacian_matches_oracle():
    c = ctx(8, "fp64")
    rng = np.random.default_rng(5)
    allc = box_coords(4)
    coords = allc[rng.random(len(allc)) < 0.6]
    bs = F.BlockSet(c, [[coords]], [0.25])
    u = rng.standard_normal((len(coords), 8, 8, 8))
    got = bs.laplacian(0, 0, torch.as_tensor(u)).cpu().numpy()
    ref, mask = laplacian_on_level(Level(coords, 8), u, 0.25)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.all(got[~mask] == 0.0)


@pytest.mark.parametrize("compensated", [0, 1])
def test_batched_problems_equal_single_solves(compensated):
    """Several independent problems in one block set run in the same launches
    and give bit-identical results to solving each alone (with the same
    FLGF_OPT_COMPENSATED setting: its default depends on the block set)."""
    c = ctx(8, "fp32")
    probs = [_gauss_problem(box_coords(3), 8, 7), _two_level(), _gauss_problem(box_coords(5), 8, 8)]
    singles = [[u.double().cpu().numpy() for u in F.solve_problem(c, p, compensated=bool(compensated))] for p in probs]
    bs = F.BlockSet(c, [p.coords for p in probs], [p.h0 for p in probs])
    bs.set_option(F.OPT_COMPENSATED, compensated)
    for i, p in enumerate(probs):
        for l, f in enumerate(p.f):
            bs.load_source(i, l, torch.as_tensor(f))
    bs.solve()
    for i, p in enumerate(probs):
        for l in range(p.n_levels):
            assert torch.equal(bs.potential(i, l).cpu(), torch.as_tensor(singles[i][l]).float())


def test_graph_replay_and_stage_timing():
    c = ctx(8, "fp64")
    p = _two_level()
    bs = F.BlockSet(c, [p.coords], [p.h0])
    for l, f in enumerate(p.f):
        bs.load_source(0, l, torch.as_tensor(f))
    bs.solve()
    plain = [bs.potential(0, l).clone() for l in range(2)]
    bs.set_option(F.OPT_GRAPH, 1)
    bs.set_option(F.OPT_TIMING, 1)
    for _ in range(3):
        bs.solve()
    for l in range(2):
        assert torch.equal(bs.potential(0, l), plain[l])
    times, n = bs.stage_times()
    assert n == 3 and times["spectrum_mac"] > 0 and times["fft_forward"] > 0


def test_mesh_errors_are_reported():
    c = ctx(8, "fp64")
    with pytest.raises(F.FLGFError, match="duplicate"):
        F.BlockSet(c, [[np.array([[0, 0, 0], [0, 0, 0]])]], [1.0])
    with pytest.raises(F.FLGFError, match="partially refined"):
        F.BlockSet(c, [[box_coords(3), np.array([[2, 2, 2]])]], [1.0])
    with pytest.raises(F.FLGFError, match="buffer"):
        F.BlockSet(c, [[box_coords(2), box_coords(2)]], [1.0])


def test_per_parent_anterpolation_equals_cluster_form():
    """Octree levels with at least 2048 parents take the one-CTA-per-parent
    anterpolation, smaller ones the 8-CTA cluster form; both add the children's
    contributions in rank order, so a batch large enough for the first form
    equals its problems solved alone (second form) bit for bit."""
    from paper_1911_10228_gb300.inputs import random_sparse_problem
    probs = [random_sparse_problem(s, N=8, nblk_range=(400, 900), max_levels=1) for s in range(16)]
    parents = [len(np.unique(np.asarray(p.coords[0]) >> 1, axis=0)) for p in probs]
    assert sum(parents) >= 2048 and max(parents) < 2048, parents   # one launch of each form
    c = ctx(8, "fp32")
    singles = [F.solve_problem(c, p)[0].cpu() for p in probs]
    bs = F.BlockSet(c, [p.coords for p in probs], [p.h0 for p in probs])
    for i, p in enumerate(probs):
        bs.load_source(i, 0, torch.as_tensor(p.f[0]))
    bs.solve()
    for i in range(len(probs)):
        assert torch.equal(bs.potential(i, 0).cpu(), singles[i]), i


def test_mac_product_forms_agree_bit_for_bit():
    """The FP32 frequency-lane MAC runs a phase in its two-path form when at
    least 90 % of the phase's rows are full, in the single-path form otherwise;
    both compute the same products in the same order.  A small uniform box
    alone (every row full: two-path form) and the same box in one block set
    with a sparse problem (mostly masked rows: single path) give the same
    potential bit for bit."""
    from paper_1911_10228_gb300.inputs import random_sparse_problem
    box = _gauss_problem(box_coords(4), 8, 3)
    sparse = random_sparse_problem(11, N=8, nblk_range=(600, 900), max_levels=1)
    c = ctx(8, "fp32")
    alone = F.solve_problem(c, box)[0].cpu()
    bs = F.BlockSet(c, [box.coords, sparse.coords], [box.h0, sparse.h0])
    bs.load_source(0, 0, torch.as_tensor(box.f[0]))
    bs.load_source(1, 0, torch.as_tensor(sparse.f[0]))
    bs.solve()
    assert torch.equal(bs.potential(0, 0).cpu(), alone)
    bs.close()
