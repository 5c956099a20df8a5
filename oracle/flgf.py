"""The uniform fast lattice Green's function method on one resolution (Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Steps, in the paper's order and notation
----------------------------------------
Octree (Sec. 2.1): the given blocks of n_b^3 = N^3 cells form the finest
octree level (called level 0 here, the paper's base level L_B - 1); block
(c0, c1, c2) at level k has parent (c >> 1) at level k + 1.  The top level is
the first k at which all parents (c >> (k+1)) lie within one block of each
other on every axis, so every pair of top-level blocks that is not near is
well separated and has no common coarser level.

Lists: near field N(B) = B and its face/edge/corner neighbours, finest level
only; influence list I(B) at level k = children of the neighbours of B's
parent that are not neighbours of B; at the top level: every block that is
not a neighbour.  Every (target, source) pair of finest blocks is then
handled exactly once.

Interpolation nodes (reading; the paper defers the FMM details to the FLGF
paper it builds on): every octree node is a Cartesian block of N^3 cells
(Sec. 2.1) and field values live at cell centres (Sec. 3), so the N^3 nodes
of a level-k block are the centres of its N^3 cells of width 2^k.  Node
differences are then multiples of 2^k lattice spacings and the level-k kernel
between node p of block t and node q of block s is the exact LGF value
G(2^k (N (t - s) + p - q)).  Along one axis, in units of the child spacing,
the 2N nodes of two sibling children sit at j + 1/2 (j = 0..2N-1) and the N
nodes of their parent at 2p + 1 (p = 0..N-1): no node coincides (staggered
as in Sec. 3).  J_1 (2N x N) interpolates each child node with n_I-point
Lagrange polynomials on the parent nodes nearest to it (window centred,
shifted inwards at the block faces, so the first and last child nodes are
extrapolated by a quarter of the parent spacing).  The regularisation
(anterpolation) operator is its adjoint, R = J^T.  The 3-D operators are
tensor products.

1. Upward pass:  f~^{k+1}_P = sum_{C in children(P)} R f~^k_C.
2. Level interaction:  v~^k_i = sum_{j in I(B_i^k)} conv(G_{i-j}, f~^k_j)
   (plus the near field N(B) at the finest level), each conv evaluated by a
   zero-padded (2N)^3 FFT: Hadamard product of the spectra, inverse FFT.
3. Downward pass:  u~^k_C = v~^k_C + J u~^{k+1}_{parent(C)}.

u on the finest blocks is h^2 u~^0.

Pins (tests/test_oracle_flgf.py): J_1 reproduces polynomials of degree < n_I;
a single-level tree (top level = finest) equals the brute-force direct sum to
round-off; the operator is symmetric (<A f, g> = <f, A g>); the interpolation
error against the exact Hockney convolution is small and decreases with n_I.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

_WORKERS = os.cpu_count() or 1


class Octree:
    """Block octree over a finest-level block set (coords: (nb, 3) int)."""

    def __init__(self, coords):
        coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
        if coords.shape[0] == 0:
            raise ValueError("empty block set")
        if np.unique(coords, axis=0).shape[0] != coords.shape[0]:
            raise ValueError("duplicate blocks")
        self.levels = [coords]
        k = 0
        while True:
            par = self.levels[k] >> 1
            span = par.max(axis=0) - par.min(axis=0)
            if np.all(span <= 1):
                break
            self.levels.append(np.unique(par, axis=0))
            k += 1
        self.top = k
        self.index = [{tuple(int(v) for v in c): i for i, c in enumerate(lv)} for lv in self.levels]

    def children(self, k: int, i: int):
        """Indices (at level k-1) of the existing children of block i at level k."""
        c = self.levels[k][i]
        out = []
        for a in range(2):
            for b in range(2):
                for d in range(2):
                    key = (int(2 * c[0] + a), int(2 * c[1] + b), int(2 * c[2] + d))
                    j = self.index[k - 1].get(key)
                    if j is not None:
                        out.append((j, (a, b, d)))
        return out

    def near(self, i: int):
        """N(B): block i of the finest level and its existing neighbours."""
        c = self.levels[0][i]
        out = []
        for e in np.ndindex(3, 3, 3):
            key = tuple(int(c[d] + e[d] - 1) for d in range(3))
            j = self.index[0].get(key)
            if j is not None:
                out.append(j)
        return out

    def influence(self, k: int, i: int):
        """I(B) at level k (all non-neighbours at the top level)."""
        lv = self.levels[k]
        c = lv[i]
        if k == self.top:
            far = np.max(np.abs(lv - c[None, :]), axis=1) > 1
            return [int(j) for j in np.nonzero(far)[0]]
        p = c >> 1
        out = []
        for e in np.ndindex(3, 3, 3):
            q = p + np.array(e) - 1
            for a in np.ndindex(2, 2, 2):
                s = 2 * q + np.array(a)
                if np.max(np.abs(s - c)) <= 1:
                    continue
                j = self.index[k].get(tuple(int(v) for v in s))
                if j is not None:
                    out.append(j)
        return out


def lagrange_J1(N: int, n_interp: int) -> np.ndarray:
    """1-D parent-to-children interpolation matrix J_1 (2N x N), cell-centred nodes."""
    if not (1 <= n_interp <= N):
        raise ValueError("need 1 <= n_I <= N")
    J = np.zeros((2 * N, N))
    parent = 2.0 * np.arange(N) + 1.0
    for j in range(2 * N):
        x = j + 0.5
        if n_interp % 2 == 0:
            lo = int(np.floor((x - 1.0) / 2.0))        # parent node just left of x
            start = lo - (n_interp // 2 - 1)
        else:
            start = int(np.argmin(np.abs(parent - x))) - n_interp // 2
        start = min(max(start, 0), N - n_interp)
        nodes = parent[start:start + n_interp]
        for m in range(n_interp):
            others = np.delete(nodes, m)
            J[j, start + m] = np.prod((x - others) / (nodes[m] - others))
    return J


def _apply_axes(mats, x):
    """y[a,b,c] = sum_{ijk} M0[a,i] M1[b,j] M2[c,k] x[i,j,k]."""
    return np.einsum("ai,bj,ck,ijk->abc", mats[0], mats[1], mats[2], x, optimize=True)


def kernel_block(G, N: int, k: int, d) -> np.ndarray:
    """(2N)^3 circular kernel array of level k, block offset d = t - s.

    Entry at circular index (Delta mod 2N) is G(2^k (N d + Delta)) for
    Delta in [-(N-1), N-1]^3; index N on any axis is never used and is 0.
    """
    P = 2 * N
    delta = np.arange(P)
    delta = np.where(delta < N, delta, delta - P)  # N maps to -N (unused)
    D = np.stack(np.meshgrid(delta, delta, delta, indexing="ij"), axis=-1)
    pts = (1 << k) * (N * np.asarray(d, dtype=np.int64)[None, None, None, :] + D)
    K = G(pts)
    unused = np.any(D == -N, axis=-1)
    K[unused] = 0.0
    return K


class FLGF:
    """Uniform FLGF operator on one block set (one resolution)."""

    def __init__(self, G, coords, N: int, n_interp: int):
        self.G = G
        self.N = int(N)
        self.n_interp = int(n_interp)
        self.tree = Octree(coords)
        J1 = lagrange_J1(self.N, self.n_interp)
        self.Jc = [J1[:self.N], J1[self.N:]]  # per child position along an axis
        self._kspec: dict = {}

    def kernel_spectrum(self, k: int, d) -> np.ndarray:
        key = (k,) + tuple(int(v) for v in d)
        K = self._kspec.get(key)
        if K is None:
            K = sfft.rfftn(kernel_block(self.G, self.N, k, d), workers=_WORKERS)
            self._kspec[key] = K
        return K

    # -- the three steps ------------------------------------------------
    def upward(self, f0):
        """f~^k for k = 0..top (f~^0 = f)."""
        tr = self.tree
        ft = [np.asarray(f0, dtype=np.float64)]
        for k in range(1, tr.top + 1):
            lv = np.zeros((tr.levels[k].shape[0], self.N, self.N, self.N))
            for i in range(lv.shape[0]):
                for j, (a, b, c) in tr.children(k, i):
                    R = [self.Jc[a].T, self.Jc[b].T, self.Jc[c].T]
                    lv[i] += _apply_axes(R, ft[k - 1][j])
            ft.append(lv)
        return ft

    def level_interaction(self, ft, targets=None):
        """v~^k on each level (restricted to the given target indices per level)."""
        tr, N = self.tree, self.N
        P = 2 * N
        vt = []
        for k in range(tr.top + 1):
            lv = tr.levels[k]
            spec = {}
            tk = range(lv.shape[0]) if targets is None else targets[k]
            out = np.zeros((lv.shape[0], N, N, N))
            for i in tk:
                srcs = list(tr.influence(k, i))
                if k == 0:
                    srcs = tr.near(i) + srcs
                if not srcs:
                    continue
                prods = []
                for j in srcs:
                    Fj = spec.get(j)
                    if Fj is None:
                        Fj = sfft.rfftn(ft[k][j], s=(P, P, P), workers=_WORKERS)
                        spec[j] = Fj
                    prods.append(self.kernel_spectrum(k, lv[i] - lv[j]) * Fj)
                conv = sfft.irfftn(np.stack(prods), s=(P, P, P), axes=(1, 2, 3),
                                   workers=_WORKERS)[:, :N, :N, :N]
                out[i] = conv.sum(axis=0)
            vt.append(out)
        return vt

    def downward(self, vt):
        tr = self.tree
        ut = [None] * (tr.top + 1)
        ut[tr.top] = vt[tr.top].copy()
        for k in range(tr.top - 1, -1, -1):
            uk = vt[k].copy()
            for i in range(tr.levels[k + 1].shape[0]):
                for j, (a, b, c) in tr.children(k + 1, i):
                    uk[j] += _apply_axes([self.Jc[a], self.Jc[b], self.Jc[c]], ut[k + 1][i])
            ut[k] = uk
        return ut

    def _ancestor_targets(self, finest):
        tr = self.tree
        sets = [sorted(set(int(i) for i in finest))]
        for k in range(1, tr.top + 1):
            keys = {tuple(int(v) for v in (tr.levels[0][i] >> k)) for i in sets[0]}
            sets.append(sorted(tr.index[k][key] for key in keys))
        return sets

    def apply(self, f, h: float = 1.0, targets=None) -> np.ndarray:
        """u = h^2 (FLGF approximation of G * f) on the finest blocks.

        f: (nb, N, N, N) values on the blocks in the order of ``coords``.
        targets: optional finest-block indices; u is then exact to the
        method only on those blocks (others are left at partial sums).
        """
        ft = self.upward(f)
        tsets = None if targets is None else self._ancestor_targets(targets)
        vt = self.level_interaction(ft, tsets)
        ut = self.downward(vt)
        return h * h * ut[0]


def blocks_to_dense(coords, vals, N: int):
    """Scatter block values into a dense box; returns (array, origin cell)."""
    coords = np.asarray(coords, dtype=np.int64)
    lo = coords.min(axis=0)
    ext = (coords.max(axis=0) - lo + 1) * N
    out = np.zeros(tuple(int(e) for e in ext))
    for c, v in zip(coords, vals):
        o = (c - lo) * N
        out[o[0]:o[0] + N, o[1]:o[1] + N, o[2]:o[2] + N] = v
    return out, lo * N


def dense_to_blocks(dense, origin, coords, N: int):
    coords = np.asarray(coords, dtype=np.int64)
    out = np.empty((coords.shape[0], N, N, N))
    for b, c in enumerate(coords):
        o = c * N - np.asarray(origin)
        out[b] = dense[o[0]:o[0] + N, o[1]:o[1] + N, o[2]:o[2] + N]
    return out
