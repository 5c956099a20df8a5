"""Adjoint (transpose) of the FLGF solution operator, for gradients.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper gives no adjoint; it follows from the forward steps.  Every step of
``FLGF.apply`` and ``multires_solve`` is linear in the source, and this module
writes out the transpose of each step explicitly and applies them in reverse
order:

* FMM: apply = D K U (upward anterpolation U, level interactions K, downward
  interpolation D).  apply^T = U^T K^T D^T: the downward pass's transpose is an
  anterpolation pass over the adjoint field, the upward pass's transpose an
  interpolation pass, and K^T takes every pair (t <- s) to (s <- t): the
  correlation with the same kernel array, i.e. the conjugate kernel spectrum
  applied to the padded target field, extracted on the source block.
* Multi-resolution (forward order in ``oracle/multires.py``):
    u^l = P_leaf A_l f^l + P_nonleaf A_l (P_leaf f^l) + J^{l-1} W^{l-1}
    W^l = A_l (P_leaf f^l) + J^{l-1} W^{l-1}
    f^{l+1} -= L_Q^{(h_{l+1})} J^l W^l                       (correction)
  and, before the level loop, the coarsening f^l[non-leaf] = C f^{l+1}.
  Reverse: for l = L-1..0 the correction, accumulation, selection and FMMs
  are transposed; afterwards the coarsening is transposed from the coarsest
  level down (C^T spreads each coarse value over its 8 fine cells with
  weight 1/8) and the overwritten non-leaf entries get zero gradient.

Pins (tests/test_oracle_adjoint.py): <A f, g> = <f, A^T g> to round-off for
the FMM and for the multi-resolution operator (with and without correction);
the gradient of 0.5 ||u - t||^2 matches central finite differences.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from .flgf import FLGF, _WORKERS, _apply_axes
from .multires import Level, _W, _block_cells, coarsen, leaf_masks


def flgf_transpose(op: FLGF, g, h: float = 1.0) -> np.ndarray:
    """A^T g for the uniform FLGF operator ``op`` (g on the finest blocks)."""
    tr, N = op.tree, op.N
    P = 2 * N
    # D^T: anterpolate the adjoint field up the tree (transpose of u_C += J u_P)
    gt = [np.asarray(g, dtype=np.float64) * (h * h)]
    for k in range(1, tr.top + 1):
        lv = np.zeros((tr.levels[k].shape[0], N, N, N))
        for i in range(lv.shape[0]):
            for j, (a, b, c) in tr.children(k, i):
                lv[i] += _apply_axes([op.Jc[a].T, op.Jc[b].T, op.Jc[c].T], gt[k - 1][j])
        gt.append(lv)
    # K^T: every pair (t <- s, offset d = t - s) becomes s <- t with the
    # correlation: conj(K^_d) times the padded target field
    st = []
    for k in range(tr.top + 1):
        lv = tr.levels[k]
        out = np.zeros((lv.shape[0], N, N, N))
        spec = {}
        for t in range(lv.shape[0]):
            srcs = list(tr.influence(k, t))
            if k == 0:
                srcs = tr.near(t) + srcs
            if not srcs:
                continue
            Gt = spec.get(t)
            if Gt is None:
                Gt = sfft.rfftn(gt[k][t], s=(P, P, P), workers=_WORKERS)
                spec[t] = Gt
            for s in srcs:
                corr = sfft.irfftn(np.conj(op.kernel_spectrum(k, lv[t] - lv[s])) * Gt, s=(P, P, P),
                                   workers=_WORKERS)[:N, :N, :N]
                out[s] += corr
        st.append(out)
    # U^T: interpolate down the tree (transpose of f~_P = sum R f~_C)
    res = [None] * (tr.top + 1)
    res[tr.top] = st[tr.top]
    for k in range(tr.top, 0, -1):
        nxt = st[k - 1].copy()
        for i in range(tr.levels[k].shape[0]):
            for j, (a, b, c) in tr.children(k, i):
                nxt[j] += _apply_axes([op.Jc[a], op.Jc[b], op.Jc[c]], res[k][i])
        res[k - 1] = nxt
    return res[0]


def _interp_T(coarse: Level, gfine, fine_cells, out):
    """Transpose of J^l: spread adjoint values at fine cells onto coarse cells."""
    fine_cells = np.asarray(fine_cells, dtype=np.int64).reshape(-1, 3)
    gf = np.asarray(gfine).reshape(-1)
    ic = fine_cells >> 1
    a = fine_cells & 1
    N = coarse.N
    for e in np.ndindex(3, 3, 3):
        w = _W[a[:, 0], e[0]] * _W[a[:, 1], e[1]] * _W[a[:, 2], e[2]]
        cells = ic + (np.array(e) - 1)[None, :]
        blk = cells // N
        loc = cells - blk * N
        ids = coarse.block_ids(blk)
        if np.any(ids < 0):
            raise KeyError("coarse cell outside the level's blocks")
        np.add.at(out, (ids, loc[:, 0], loc[:, 1], loc[:, 2]), w * gf)


def _laplacian_T(gint, h):
    """Transpose of the 7-point stencil from an (N+2)^3 region to its N^3 interior."""
    N = gint.shape[0]
    r = np.zeros((N + 2, N + 2, N + 2))
    s = gint / (h * h)
    r[1:-1, 1:-1, 1:-1] -= 6.0 * s
    r[2:, 1:-1, 1:-1] += s
    r[:-2, 1:-1, 1:-1] += s
    r[1:-1, 2:, 1:-1] += s
    r[1:-1, :-2, 1:-1] += s
    r[1:-1, 1:-1, 2:] += s
    r[1:-1, 1:-1, :-2] += s
    return r


def multires_adjoint(G, levels_coords, g_levels, N: int, n_interp: int, h0: float = 1.0,
                     correction: bool = True):
    """Gradient of <g, u> with respect to the user source f on every level.

    g_levels[l]: (nb_l, N, N, N) adjoint of u on level l.  Returns per level the
    gradient with respect to the given source (zero on non-leaf blocks, whose
    source values the forward operator ignores).
    """
    L = len(levels_coords)
    lv = [Level(c, N) for c in levels_coords]
    leaf = leaf_masks(levels_coords)
    gu = [np.asarray(g, dtype=np.float64) for g in g_levels]
    gW = [np.zeros_like(x) for x in gu]
    gf = [np.zeros_like(x) for x in gu]
    for l in range(L - 1, -1, -1):
        h = h0 / (1 << l)
        if correction and l + 1 < L:   # f^{l+1} -= L_Q J^l W^l
            hf = h0 / (1 << (l + 1))
            for b, c in enumerate(lv[l + 1].coords):
                r = _laplacian_T(gf[l + 1][b], hf)
                _interp_T(lv[l], -r, _block_cells(c, N, pad=1), gW[l])
        lm = leaf[l][:, None, None, None]
        g_leafsrc = np.where(lm, 0.0, gu[l]) + gW[l]     # adjoint of A_l (P_leaf f^l)
        op = FLGF(G, lv[l].coords, N, n_interp)
        gf[l] += flgf_transpose(op, np.where(lm, gu[l], 0.0), h)
        gf[l] += np.where(lm, flgf_transpose(op, g_leafsrc, h), 0.0)
        if l > 0:                       # u^l, W^l += J^{l-1} W^{l-1}
            for b, c in enumerate(lv[l].coords):
                _interp_T(lv[l - 1], gu[l][b] + gW[l][b], _block_cells(c, N), gW[l - 1])
    # coarsening: f^l[non-leaf] = C f^{l+1}, applied before the level loop
    for l in range(0, L - 1):
        fine = lv[l + 1]
        for i in np.nonzero(~leaf[l])[0]:
            c = lv[l].coords[i]
            spread = np.repeat(np.repeat(np.repeat(gf[l][i], 2, 0), 2, 1), 2, 2) / 8.0
            for a in np.ndindex(2, 2, 2):
                j = fine.index[tuple(int(v) for v in (2 * c + np.array(a)))]
                gf[l + 1][j] += spread[a[0] * N:(a[0] + 1) * N, a[1] * N:(a[1] + 1) * N, a[2] * N:(a[2] + 1) * N]
            gf[l][i] = 0.0
    return gf
