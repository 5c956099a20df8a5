"""Seeded synthetic workloads: block sets, refinement and source fields.

This module builds inputs only.  It contains none of the solver's arithmetic
(no Green's function, no convolution, no interpolation operator), so both
the CUDA path and the CPU oracle can be fed from it.

Conventions
-----------
* A block set of one refinement level is an int array ``coords`` of shape
  (nb, 3): block (c0, c1, c2) covers global cells c*N .. c*N + N - 1 on each
  axis.  Block values are arrays (nb, N, N, N), C order, the last index along
  axis 2.
* Level l has spacing h_l = h0 / 2^l; cell i of level l has its centre at
  (i + 1/2) h_l.  Level l+1 block 2c + a (a in {0,1}^3) refines level-l
  block c.
* Sources are sampled at cell centres and set to zero where they fall below
  ``1e-14`` of the maximum (compact support).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TRUNC = 1e-14


def box_coords(n0: int, n1: int | None = None, n2: int | None = None, origin=(0, 0, 0)) -> np.ndarray:
    n1 = n0 if n1 is None else n1
    n2 = n0 if n2 is None else n2
    g = np.stack(np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij"), axis=-1)
    return (g.reshape(-1, 3) + np.asarray(origin, dtype=np.int64)).astype(np.int64)


def cell_centres(coords, N: int, h: float):
    """Physical cell-centre coordinates, shape (nb, N, N, N, 3)."""
    coords = np.asarray(coords, dtype=np.int64)
    ax = np.arange(N)
    loc = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1)
    return ((coords[:, None, None, None, :] * N + loc[None]) + 0.5) * h


def gaussians(x, centres, sigmas, amps):
    """Sum of isotropic Gaussians a exp(-|x - c|^2 / (2 s^2)) at points x (..., 3)."""
    out = np.zeros(x.shape[:-1])
    for c, s, a in zip(centres, sigmas, amps):
        d2 = np.sum((x - np.asarray(c)) ** 2, axis=-1)
        out += a * np.exp(-d2 / (2.0 * s * s))
    return out


def torus(x, centre, R: float, sigma: float, axis_rot=None):
    """Gaussian-core torus exp(-d^2 / (2 sigma^2)), d = distance to the core circle."""
    y = x - np.asarray(centre)
    if axis_rot is not None:
        y = y @ np.asarray(axis_rot).T
    rho = np.sqrt(y[..., 0] ** 2 + y[..., 1] ** 2)
    d2 = (rho - R) ** 2 + y[..., 2] ** 2
    return np.exp(-d2 / (2.0 * sigma * sigma))


def _vortex_ring_parts(x, centre, R, c1, c2):
    """Bump value f, azimuthal vorticity omega_theta and (sin, cos) of the
    azimuth at points x (..., 3); all zero outside the ring's support."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(centre, dtype=np.float64)
    r = np.hypot(d[..., 0], d[..., 1])
    rho = np.hypot(r - R, d[..., 2])
    t = rho / R
    inside = t < 1.0
    ts = np.where(inside, t, 0.0)
    s = 1.0 - ts * ts
    f = np.where(inside, c1 * np.exp(-c2 / s), 0.0)
    fp_over_rho = -2.0 * c2 * f / (s * s * R)               # f'(t) / rho, finite at rho = 0
    fpp = -2.0 * c2 * f / (s * s) * (1.0 - 2.0 * c2 * ts * ts / (s * s) + 4.0 * ts * ts / s)
    rs = np.where(inside, r, 1.0)                            # r > 0 on the support
    omega_t = fpp / (R * R) + fp_over_rho / R + fp_over_rho * (rs - R) / (R * rs) - f / (rs * rs)
    sin_t = np.where(inside, d[..., 1] / rs, 0.0)
    cos_t = np.where(inside, d[..., 0] / rs, 0.0)
    return f, np.where(inside, omega_t, 0.0), sin_t, cos_t


def vortex_ring(x, centre=(0.5, 0.5, 0.5), R: float = 0.125, c1: float = 1e3, c2: float = 10.0):
    """Manufactured solution of Sec. 3.1 (Eqs. streamfunc, streamfunc_f): the
    streamfunction Psi = f(sqrt((r - R)^2 + z^2) / R) e_theta of a vortex ring
    of radius R about the z axis through ``centre``, with the bump
    f(t) = c1 exp(-c2 / (1 - t^2)) for |t| < 1 and 0 elsewhere, and the
    vorticity omega = Laplacian(Psi) evaluated analytically.

    Returns the x components (psi_x, omega_x) at points x (..., 3); each
    Cartesian component satisfies the scalar Poisson equation on its own.
    For an azimuthal axisymmetric field psi(r, z) e_theta the Laplacian is
    (d_rr + d_r / r + d_zz - 1 / r^2) psi e_theta; with psi = f(rho / R),
    rho the distance to the core circle, d_rr + d_zz gives
    f'' / R^2 + f' / (R rho), and d_r psi = f' (r - R) / (R rho).
    """
    f, w, sin_t, _ = _vortex_ring_parts(x, centre, R, c1, c2)
    return -f * sin_t, -w * sin_t                            # e_theta = (-sin, cos, 0)


def vortex_ring_vector(x, centre=(0.5, 0.5, 0.5), R: float = 0.125, c1: float = 1e3, c2: float = 10.0):
    """All three Cartesian components of the vortex ring's streamfunction and
    vorticity (see vortex_ring): arrays (..., 3), the z components zero."""
    f, w, sin_t, cos_t = _vortex_ring_parts(x, centre, R, c1, c2)
    z = np.zeros_like(f)
    return np.stack([-f * sin_t, f * cos_t, z], axis=-1), np.stack([-w * sin_t, w * cos_t, z], axis=-1)


def split_blocks(coords_levels):
    """Global refinement with a fixed mesh topology: every block of every level
    becomes its 8 children (same physical regions, half the spacing)."""
    out = []
    for c in coords_levels:
        c = np.asarray(c, dtype=np.int64).reshape(-1, 3)
        kids = (2 * c[:, None, :] + np.array(list(np.ndindex(2, 2, 2)))[None]).reshape(-1, 3)
        out.append(kids[np.lexsort((kids[:, 2], kids[:, 1], kids[:, 0]))])
    return out


def config_vortex_ring(n_levels: int = 3, N: int = 8, nbase: int = 4, splits: int = 0, alpha: float = 1.0 / 32):
    """Single vortex ring of Sec. 3.1 (c1 = 1e3, c2 = 10, R = 0.125, centred in the
    unit cube) on nbase^3 base blocks.  Refinement reads Eq. ref_crit as: a
    level-l block (l < n_levels - 1) is refined where |omega| exceeds
    alpha^(n_levels - 1 - l) of its maximum on that level.  ``splits`` then
    refines the whole mesh globally that many times with a fixed topology.
    Returns (Problem, psi_x per level) with the source omega_x and the
    analytic solution sampled at cell centres."""
    h0 = 1.0 / (nbase * N)
    thr = [alpha ** (n_levels - 1 - l) for l in range(n_levels - 1)]
    prob = refine_mesh(lambda x: vortex_ring(x)[1], box_coords(nbase), N, h0, n_levels, thresholds=thr)
    coords = prob.coords
    for _ in range(splits):
        coords = split_blocks(coords)
        h0 = h0 / 2
    out = Problem(N=N, h0=h0, name=f"vortex_ring_L{n_levels}_b{nbase}_s{splits}")
    psi = []
    for l, c in enumerate(coords):
        p, w = vortex_ring(cell_centres(c, N, h0 / (1 << l)))
        out.coords.append(c)
        out.f.append(w)
        psi.append(p)
    return out, psi


def truncate(f: np.ndarray, ref: float | None = None) -> np.ndarray:
    m = np.max(np.abs(f)) if ref is None else ref
    return np.where(np.abs(f) < TRUNC * m, 0.0, f)


@dataclass
class Problem:
    """One (possibly refined) Poisson problem: block sets and sources per level."""
    N: int
    h0: float
    coords: list = field(default_factory=list)   # per level (nb_l, 3) int64
    f: list = field(default_factory=list)        # per level (nb_l, N, N, N) float64
    name: str = ""

    @property
    def n_levels(self) -> int:
        return len(self.coords)

    def leaf_masks(self):
        out = []
        for l, c in enumerate(self.coords):
            if l + 1 == len(self.coords):
                out.append(np.ones(len(c), dtype=bool))
                continue
            par = {tuple(v) for v in (np.asarray(self.coords[l + 1]) >> 1).tolist()}
            out.append(np.array([tuple(v) not in par for v in np.asarray(c).tolist()]))
        return out

    def dof(self) -> int:
        """Leaf cells over all levels (unknowns of the composite mesh)."""
        return int(sum(int(m.sum()) for m in self.leaf_masks()) * self.N ** 3)


# ----------------------------------------------------------------------------
# Uniform single-level workloads
# ----------------------------------------------------------------------------

def plain_gaussians(nblk: int, N: int, n_gauss: int, sigma_rng, inner, seed: int = 0,
                    h0: float = 1.0) -> Problem:
    """nblk^3 blocks of N^3 cells; Gaussians with sigma ~ U(sigma_rng) cells, centres
    ~ U(inner) cells (lattice units, cell centres at i + 1/2), amplitudes ~ U(-1, 1).

    The box is dense, so each Gaussian is evaluated as the product of its three
    1-D factors on the cell-centre axis and then cut into blocks.
    """
    rng = np.random.default_rng(seed)
    sig = rng.uniform(sigma_rng[0], sigma_rng[1], n_gauss)
    cen = rng.uniform(inner[0], inner[1], (n_gauss, 3))
    amp = rng.uniform(-1.0, 1.0, n_gauss)
    coords = box_coords(nblk)
    ax = np.arange(nblk * N) + 0.5
    dense = np.zeros((nblk * N,) * 3)
    for c, s, a in zip(cen, sig, amp):
        e = [np.exp(-(ax - c[d]) ** 2 / (2.0 * s * s)) for d in range(3)]
        dense += a * (e[0][:, None, None] * e[1][None, :, None] * e[2][None, None, :])
    f = dense.reshape(nblk, N, nblk, N, nblk, N).transpose(0, 2, 4, 1, 3, 5).reshape(-1, N, N, N)
    f = truncate(f)
    return Problem(N=N, h0=h0, coords=[coords], f=[f], name=f"gauss{nblk}x{N}")


def config_plain_32() -> Problem:
    """4x4x4 blocks of 8^3 (32^3 cells), 3 Gaussians, sigma 2-4 cells, centres in the
    inner 16^3 region (cells 8..24), seed 0."""
    return plain_gaussians(4, 8, 3, (2.0, 4.0), (8.0, 24.0), seed=0)


def config_uniform_256() -> Problem:
    """256^3 lattice as 16^3 blocks of 16^3, 16 Gaussians, sigma 3-10 cells, centres in
    the inner 128^3 region, seed 0."""
    return plain_gaussians(16, 16, 16, (3.0, 10.0), (64.0, 192.0), seed=0)


# ----------------------------------------------------------------------------
# Refined meshes
# ----------------------------------------------------------------------------

def _nbrs26(c):
    for e in np.ndindex(3, 3, 3):
        if e != (1, 1, 1):
            yield (c[0] + e[0] - 1, c[1] + e[1] - 1, c[2] + e[2] - 1)


def refine_mesh(src, base_coords, N: int, h0: float, n_levels: int, threshold: float = 1e-3, thresholds=None):
    """Block-refined mesh for a source callable src(x) -> f (x: (..., 3) physical).

    A block of level l < n_levels-1 is refined when any of its cells has
    |f| > threshold * max|f| on that level (``thresholds[l]`` when given).  The mesh is then closed so that
    every refined block has all 26 same-level neighbours (zero-source blocks
    are added where needed, refining coarser blocks if necessary) and every
    refined block has all 8 children.  Returns a Problem with sources sampled
    on every block of every level.
    """
    levels = [set(map(tuple, np.asarray(base_coords, dtype=np.int64).tolist()))]
    refined = [set() for _ in range(n_levels)]
    for l in range(n_levels - 1):
        h = h0 / (1 << l)
        cl = np.array(sorted(levels[l]), dtype=np.int64)
        vals = src(cell_centres(cl, N, h))
        m = np.max(np.abs(vals)) if vals.size else 0.0
        thr = threshold if thresholds is None else thresholds[l]
        hit = np.any(np.abs(vals) > thr * m, axis=(1, 2, 3)) if m > 0 else np.zeros(len(cl), bool)
        refined[l] = set(map(tuple, cl[hit].tolist()))
        # close: neighbours of refined blocks exist on this level (add them,
        # and refine their parents on coarser levels as far as needed)
        changed = True
        while changed:
            changed = False
            for c in list(refined[l]):
                for nb in _nbrs26(c):
                    if nb not in levels[l]:
                        levels[l].add(nb)
                        changed = True
                        _ensure_exists(levels, refined, l, nb)
        levels.append({(2 * c[0] + a[0], 2 * c[1] + a[1], 2 * c[2] + a[2])
                       for c in refined[l] for a in np.ndindex(2, 2, 2)})
    prob = Problem(N=N, h0=h0)
    for l in range(n_levels):
        cl = np.array(sorted(levels[l]), dtype=np.int64).reshape(-1, 3)
        prob.coords.append(cl)
    ref = max(np.max(np.abs(src(cell_centres(c, N, h0 / (1 << l))))) for l, c in enumerate(prob.coords))
    for l, cl in enumerate(prob.coords):
        prob.f.append(truncate(src(cell_centres(cl, N, h0 / (1 << l))), ref))
    return prob


def _ensure_exists(levels, refined, l, c):
    """Block c was added on level l (l > 0): its parent must be refined on l-1."""
    if l == 0:
        return
    p = (c[0] >> 1, c[1] >> 1, c[2] >> 1)
    if p not in levels[l - 1]:
        levels[l - 1].add(p)
        _ensure_exists(levels, refined, l - 1, p)
    if p not in refined[l - 1]:
        refined[l - 1].add(p)
        for a in np.ndindex(2, 2, 2):
            levels[l].add((2 * p[0] + a[0], 2 * p[1] + a[1], 2 * p[2] + a[2]))
        for nb in _nbrs26(p):
            if nb not in levels[l - 1]:
                levels[l - 1].add(nb)
                _ensure_exists(levels, refined, l - 1, nb)


def config_torus_128(n_levels: int = 3, N: int = 16, nbase: int = 8) -> Problem:
    """Base 128^3 (8^3 blocks of 16^3) on the unit cube, Gaussian torus R = 0.25,
    sigma = 0.03, centred, axis z; refined where |f| > 1e-3 max."""
    h0 = 1.0 / (nbase * N)
    src = lambda x: torus(x, (0.5, 0.5, 0.5), 0.25, 0.03)
    p = refine_mesh(src, box_coords(nbase), N, h0, n_levels, 1e-3)
    p.name = f"torus{nbase * N}_L{n_levels}"
    return p


def _rot_x90():
    return np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])


def linked_tori(x, R=0.2, sigma=0.03):
    c1 = np.array([0.5 - R / 2, 0.5, 0.5])
    c2 = c1 + np.array([R, 0.0, 0.0])
    return torus(x, c1, R, sigma) + torus(x, c2, R, sigma, axis_rot=_rot_x90())


def config_linked_tori(n_levels: int = 3, N: int = 16, nbase: int = 8, threshold: float = 1e-3) -> Problem:
    """Two linked Gaussian tori (R = 0.2, sigma = 0.03; ring 2 rotated 90 degrees about
    x and offset by R) on a base of nbase^3 blocks, refined where |f| > threshold max."""
    h0 = 1.0 / (nbase * N)
    p = refine_mesh(linked_tori, box_coords(nbase), N, h0, n_levels, threshold)
    p.name = f"tori{nbase * N}_L{n_levels}"
    return p


def smooth_field(x, seed: int = 1, n_modes: int = 4):
    """Smooth seeded random field: a few low-frequency cosines with random phases."""
    rng = np.random.default_rng(seed)
    out = np.zeros(x.shape[:-1])
    for _ in range(n_modes):
        k = rng.integers(1, 4, 3) * 2.0 * np.pi
        ph = rng.uniform(0, 2 * np.pi)
        out += rng.uniform(-1, 1) * np.cos(x @ k + ph)
    return out / n_modes


def gaussians_separable(coords, N: int, h: float, centres, sigmas, amps) -> np.ndarray:
    """Sum of Gaussians on the cells of a block set, each evaluated as the product
    of its three 1-D factors per block (same values as ``gaussians``)."""
    coords = np.asarray(coords, dtype=np.int64)
    out = np.zeros((len(coords), N, N, N))
    ax = np.arange(N)
    for c, s, a in zip(centres, sigmas, amps):
        e = [np.exp(-(((coords[:, d, None] * N + ax[None, :]) + 0.5) * h - c[d]) ** 2 / (2.0 * s * s))
             for d in range(3)]
        out += a * np.einsum("bi,bj,bk->bijk", e[0], e[1], e[2], optimize=True)
    return out


def random_sparse_problem(seed: int, N: int = 16, nblk_range=(8, 4096), max_levels: int = 3) -> Problem:
    """Random disjoint sparse block set with 1..max_levels levels and 1-4 Gaussians.

    Total block count over levels ~ round(exp U[ln a, ln b]).  The base level is a
    random subset of a cube of side ceil((4 nblk_base)^(1/3)); on every level the
    quarter of the blocks nearest to a random centre is refined (closed with the
    26-neighbour buffer), so each refinement roughly doubles the block count and
    the base holds about 1/(1 + 2 + 4) of the blocks for three levels.
    """
    rng = np.random.default_rng(seed)
    n_target = int(round(math.exp(rng.uniform(math.log(nblk_range[0]), math.log(nblk_range[1])))))
    L = int(rng.integers(1, max_levels + 1))
    n_base = max(1, int(round(n_target / sum(2 ** l for l in range(L)))))
    side = max(2, int(math.ceil((4 * n_base) ** (1.0 / 3.0))))
    allc = box_coords(side)
    pick = rng.choice(len(allc), size=min(n_base, len(allc)), replace=False)
    base = allc[np.sort(pick)]
    h0 = 1.0 / (side * N)
    ng = int(rng.integers(1, 5))
    cen = rng.uniform(0.25, 0.75, (ng, 3))
    sig = rng.uniform(0.03, 0.1, ng)
    amp = rng.uniform(-1, 1, ng)
    focus = rng.uniform(0.3, 0.7, 3)
    levels = [set(map(tuple, base.tolist()))]
    refined = [set() for _ in range(L)]
    for l in range(L - 1):
        cl = np.array(sorted(levels[l]), dtype=np.int64)
        k = max(1, int(round(0.25 * len(cl))))
        centre = focus * side * (1 << l)
        near = np.argsort(np.sum((cl + 0.5 - centre) ** 2, axis=1), kind="stable")[:k]
        refined[l] = {tuple(v) for v in cl[near].tolist()}
        changed = True
        while changed:
            changed = False
            for c in list(refined[l]):
                for nb in _nbrs26(c):
                    if nb not in levels[l]:
                        levels[l].add(nb)
                        changed = True
                        _ensure_exists(levels, refined, l, nb)
        levels.append({(2 * c[0] + a[0], 2 * c[1] + a[1], 2 * c[2] + a[2])
                       for c in refined[l] for a in np.ndindex(2, 2, 2)})
    p = Problem(N=N, h0=h0, name=f"rand{seed}")
    for l in range(L):
        p.coords.append(np.array(sorted(levels[l]), dtype=np.int64).reshape(-1, 3))
    vals = [gaussians_separable(c, N, h0 / (1 << l), cen, sig, amp) for l, c in enumerate(p.coords)]
    ref = max(np.max(np.abs(v)) for v in vals)
    p.f = [truncate(v, ref) for v in vals]
    return p


def config_batched(n_problems: int = 64, N: int = 16, first_seed: int = 0):
    """64 independent problems (seeds first_seed .. first_seed + 63): block counts
    log-uniform in [8, 4096] over 1-3 levels, random disjoint sparse base sets,
    random Gaussian sources."""
    return [random_sparse_problem(s, N=N) for s in range(first_seed, first_seed + n_problems)]
