"""The block-refined (multi-resolution) FLGF scheme (Sec. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Mesh: refinement levels l = 0..L_R-1, level 0 the coarsest, spacing
h_l = h_0 / 2^l.  Each level is a set of N^3-cell blocks; block c of level l
is refined (non-leaf) when its 8 children 2c + {0,1}^3 exist on level l+1
(all or none).  The source is given on the leaf blocks of every level.

Algorithm, in the paper's order (Sec. 3, the three numbered steps):
1. Regularisation: for l = L_R-2..0, f^l on a non-leaf block is the coarsening
   C of f^{l+1} on its children: each coarse cell is the mean of its 8 fine
   cells (the 1-D rule u^l_i = (u^{l+1}_{2i} + u^{l+1}_{2i+1}) / 2 per axis).
2. For l = 0..L_R-1:
   a. Convolution (Eq. amr_convs) with the two-FMM subtraction: one uniform
      FLGF of all level-l sources evaluated on all level-l blocks, and one of
      the non-leaf sources only; leaf targets keep the first, non-leaf
      targets the difference (= the field of the leaf sources).
   b. Accumulation: u~^l = v~^l + J^{l-1} W^{l-1}, where W^{l-1} is the
      field of the leaf sources of levels <= l-1 (next item).
   c. Source correction: f^{l+1} <- f^{l+1} - L_Q^{(h_{l+1})} J^l W^l on
      every level-(l+1) block.
3. The answer is u~^l on the leaf blocks of every level.

Readings (the paper is garbled or silent here):
* What J^l interpolates (Sec. 3, "Regularization and Interpolation
  operators": the interpolant is the interaction of a non-leaf octant with the
  leaf octants only, taken over a buffer layer around the octant): the
  leaf-source field W^l = (field of the level-l leaf sources) + J^{l-1} W^{l-1},
  i.e. the field of the leaf sources of all levels <= l, evaluated on the
  non-leaf blocks and their buffer of neighbouring blocks.  (On non-leaf
  blocks W^l equals u~^l; on leaf blocks it omits the coarsened finer sources,
  whose field the finer level computes itself.  Interpolating u~^l there
  instead makes the interpolant jump at the coarse-fine interface, and the
  correction turns that jump into a large spurious source.)
* The operand of the correction is that field, J^l W^l (the printed
  "J^l f~^l" cannot be a field).  With it L_Q^{(h_{l+1})} u~^{l+1} reproduces
  f^{l+1} on the interior of level l+1 (Sec. 3, the Laplacian-free
  requirement).
* Coarse-fine interpolation J^l ("second-order Lagrangian polynomials",
  cell-centred, staggered): per axis the fine cells 2i and 2i+1 sit at -1/4
  and +1/4 of the coarse cell i; each uses the quadratic through coarse cells
  i-1, i, i+1, i.e. weights (5/32, 15/16, -3/32) and the mirror
  (-3/32, 15/16, 5/32).  3-D: tensor product (27 coarse cells).
* The "buffer layer" is read as: every non-leaf block's 26 same-level
  neighbours exist (the mesh generator adds zero-source blocks), which gives
  the coarse halo that J^l and the correction stencil need.
* u = h_l^2 (G * f) on level l (lattice units scaled by the spacing).

Pins (tests/test_oracle_multires.py): one level reduces to the uniform FLGF;
J^l reproduces quadratics exactly; C is the exact adjoint-scaled mean;
with the correction, L_Q^{(h_l)} u = f on the leaf interiors of every level
to the FMM's accuracy (exactly, when every level's tree has a single octree
level); without it the residual is large.
"""
from __future__ import annotations

import numpy as np

from .flgf import FLGF

# Quadratic Lagrange weights for the fine cell at -1/4 (a = 0) and +1/4 (a = 1)
# of its coarse cell, on coarse cells (i-1, i, i+1).
_W = np.array([[5.0 / 32.0, 15.0 / 16.0, -3.0 / 32.0],
               [-3.0 / 32.0, 15.0 / 16.0, 5.0 / 32.0]])


class Level:
    def __init__(self, coords, N: int):
        self.coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
        self.N = N
        self.index = {tuple(int(v) for v in c): i for i, c in enumerate(self.coords)}

    def block_ids(self, blk):
        """Indices of blocks (M, 3); -1 where absent."""
        blk = np.asarray(blk, dtype=np.int64).reshape(-1, 3)
        uniq, inv = np.unique(blk, axis=0, return_inverse=True)
        ids = np.array([self.index.get(tuple(int(v) for v in u), -1) for u in uniq], dtype=np.int64)
        return ids[inv.ravel()]

    def cell_values(self, field, cells, missing_ok: bool = False):
        """field values at global cell coordinates (..., 3); KeyError if absent
        (or 0 and a False mask entry with missing_ok)."""
        N = self.N
        cells = np.asarray(cells, dtype=np.int64)
        flat = cells.reshape(-1, 3)
        blk = flat // N
        loc = flat - blk * N
        b = self.block_ids(blk)
        have = b >= 0
        if not missing_ok and not np.all(have):
            raise KeyError("cell outside the level's blocks")
        out = np.zeros(flat.shape[0])
        out[have] = field[b[have], loc[have, 0], loc[have, 1], loc[have, 2]]
        if missing_ok:
            return out.reshape(cells.shape[:-1]), have.reshape(cells.shape[:-1])
        return out.reshape(cells.shape[:-1])


def leaf_masks(levels_coords):
    """Per level, True for leaf blocks; checks that refinement is all-or-none."""
    masks = []
    for l, coords in enumerate(levels_coords):
        coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
        if l + 1 == len(levels_coords):
            masks.append(np.ones(coords.shape[0], dtype=bool))
            continue
        fine = {tuple(int(v) for v in c) for c in np.asarray(levels_coords[l + 1]).reshape(-1, 3)}
        m = np.ones(coords.shape[0], dtype=bool)
        for i, c in enumerate(coords):
            kids = [tuple(int(v) for v in (2 * c + np.array(a))) for a in np.ndindex(2, 2, 2)]
            n_have = sum(k in fine for k in kids)
            if n_have not in (0, 8):
                raise ValueError(f"level {l} block {tuple(c)} is partially refined")
            m[i] = n_have == 0
        masks.append(m)
    return masks


def coarsen(fine_level: Level, f_fine, coarse_coords, nonleaf):
    """C: each coarse cell of a non-leaf block = mean of its 8 fine cells."""
    N = fine_level.N
    out = {}
    for i in np.nonzero(nonleaf)[0]:
        c = coarse_coords[i]
        big = np.zeros((2 * N, 2 * N, 2 * N))
        for a in np.ndindex(2, 2, 2):
            j = fine_level.index[tuple(int(v) for v in (2 * c + np.array(a)))]
            big[a[0] * N:(a[0] + 1) * N, a[1] * N:(a[1] + 1) * N, a[2] * N:(a[2] + 1) * N] = f_fine[j]
        out[i] = big.reshape(N, 2, N, 2, N, 2).mean(axis=(1, 3, 5))
    return out


def interp_coarse_to_fine(coarse: Level, u_coarse, fine_cells):
    """J^l: quadratic cell-centred interpolation at fine global cells (..., 3)."""
    fine_cells = np.asarray(fine_cells, dtype=np.int64)
    flat = fine_cells.reshape(-1, 3)
    ic = flat >> 1
    a = flat & 1
    out = np.zeros(flat.shape[0])
    for e in np.ndindex(3, 3, 3):
        w = _W[a[:, 0], e[0]] * _W[a[:, 1], e[1]] * _W[a[:, 2], e[2]]
        vals = coarse.cell_values(u_coarse, ic + (np.array(e) - 1)[None, :])
        out += w * vals
    return out.reshape(fine_cells.shape[:-1])


def _block_cells(c, N, pad=0):
    ax = np.arange(-pad, N + pad)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1)
    return g + (np.asarray(c) * N)[None, None, None, :]


def laplacian_on_level(level: Level, u, h: float):
    """L_Q^{(h)} u on every cell of the level whose 6 neighbours exist (else 0),
    and the mask of those cells."""
    N = level.N
    out = np.zeros_like(u)
    mask = np.zeros(u.shape, dtype=bool)
    off = [np.array(v) for v in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]
    for b, c in enumerate(level.coords):
        cells = _block_cells(c, N)
        acc = -6.0 * u[b]
        ok = np.ones((N, N, N), dtype=bool)
        for o in off:
            vals, have = level.cell_values(u, cells + o, missing_ok=True)
            acc = acc + vals
            ok &= have
        out[b] = np.where(ok, acc / (h * h), 0.0)
        mask[b] = ok
    return out, mask


def multires_solve(G, levels_coords, levels_f, N: int, n_interp: int, h0: float = 1.0,
                   correction: bool = True, return_all: bool = False):
    """Solve the block-refined problem; returns u~^l on every block of every level.

    levels_coords[l]: (nb_l, 3) block coordinates on level l.
    levels_f[l]: (nb_l, N, N, N) source (values on non-leaf blocks are ignored).
    """
    L = len(levels_coords)
    lv = [Level(c, N) for c in levels_coords]
    leaf = leaf_masks(levels_coords)
    f = [np.array(levels_f[l], dtype=np.float64, copy=True) for l in range(L)]
    for l in range(L):
        f[l][~leaf[l]] = 0.0
    # 1. regularisation (coarsening), finest to coarsest
    for l in range(L - 2, -1, -1):
        for i, v in coarsen(lv[l + 1], f[l + 1], lv[l].coords, ~leaf[l]).items():
            f[l][i] = v
    u = [None] * L
    w = [None] * L  # leaf-source field W^l: what J^l interpolates
    for l in range(L):
        h = h0 / (1 << l)
        op = FLGF(G, lv[l].coords, N, n_interp)
        v_all = op.apply(f[l], h=h)
        if np.any(~leaf[l]):
            f_nl = np.where((~leaf[l])[:, None, None, None], f[l], 0.0)
            v_leaf = v_all - op.apply(f_nl, h=h)
        else:
            v_leaf = v_all
        v = np.where(leaf[l][:, None, None, None], v_all, v_leaf)
        wl = v_leaf.copy()
        if l > 0:
            for b, c in enumerate(lv[l].coords):
                jw = interp_coarse_to_fine(lv[l - 1], w[l - 1], _block_cells(c, N))
                v[b] += jw
                wl[b] += jw
        u[l] = v
        w[l] = wl
        if correction and l + 1 < L:
            hf = h0 / (1 << (l + 1))
            for b, c in enumerate(lv[l + 1].coords):
                jw = interp_coarse_to_fine(lv[l], w[l], _block_cells(c, N, pad=1))
                lap = (jw[2:, 1:-1, 1:-1] + jw[:-2, 1:-1, 1:-1] + jw[1:-1, 2:, 1:-1]
                       + jw[1:-1, :-2, 1:-1] + jw[1:-1, 1:-1, 2:] + jw[1:-1, 1:-1, :-2]
                       - 6.0 * jw[1:-1, 1:-1, 1:-1]) / (hf * hf)
                f[l + 1][b] -= lap
    if return_all:
        return u, leaf, f, w
    return u, leaf
