"""One step of mesh generation: refining a level (Sec. 3.1, Eq. ref_crit).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Criterion (Eq. ref_crit): a block of level l is refined where the source
exceeds alpha^(L_R - l) times its largest magnitude on the level.  Reading:
the magnitude |f| of a cell is compared; a block is refined when any of its
cells passes, i.e. when max over the block of |f| > rel * max over the level
of |f| (rel = alpha^(L_R - l)); a level whose source is zero refines nothing.
The comparison is made in FP64 on the source values as given.

Refining a block (Sec. 3, the octree of refinement levels) makes its 8
children 2c + {0,1}^3 blocks of level l + 1.  The mesh must keep every refined
block's 26 same-level neighbours (the buffer that the coarse-fine coupling
reads), so the neighbours of refined blocks that are not blocks of the level
are listed as blocks to add.

Morton order of block lists: by the integer whose bit 3i + 2 is bit i of
x + 2^20, bit 3i + 1 bit i of y + 2^20 and bit 3i bit i of z + 2^20
(i = 0..20); the plain definition, one bit at a time.
"""
from __future__ import annotations

import numpy as np

BIAS = 1 << 20


def morton_key(x: int, y: int, z: int) -> int:
    """The Morton key of block (x, y, z), |x|, |y|, |z| < 2^20."""
    ux, uy, uz = x + BIAS, y + BIAS, z + BIAS
    k = 0
    for i in range(21):
        k |= ((ux >> i) & 1) << (3 * i + 2)
        k |= ((uy >> i) & 1) << (3 * i + 1)
        k |= ((uz >> i) & 1) << (3 * i)
    return k


def morton_sorted(blocks) -> np.ndarray:
    """The blocks (an iterable of 3-tuples) in Morton order, as an (n, 3) int64 array."""
    b = sorted({tuple(int(v) for v in c) for c in blocks}, key=lambda c: morton_key(*c))
    return np.array(b, dtype=np.int64).reshape(-1, 3)


def refine_level(coords, f, rel: float):
    """coords (n, 3) block coordinates of level l; f (n, N, N, N) its source;
    rel = alpha^(L_R - l).  Returns (flags (n,) bool, children (8 m, 3) and
    buffer (k, 3), both in Morton order)."""
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    f = np.asarray(f)
    bmax = np.abs(f.reshape(len(coords), -1)).max(axis=1).astype(np.float64)
    m = float(bmax.max()) if len(bmax) else 0.0
    flags = bmax > rel * m if m > 0.0 else np.zeros(len(coords), dtype=bool)
    level = {tuple(c) for c in coords.tolist()}
    children, buffer = [], set()
    for c, fl in zip(coords.tolist(), flags):
        if not fl:
            continue
        for a0 in (0, 1):
            for a1 in (0, 1):
                for a2 in (0, 1):
                    children.append((2 * c[0] + a0, 2 * c[1] + a1, 2 * c[2] + a2))
        for d0 in (-1, 0, 1):
            for d1 in (-1, 0, 1):
                for d2 in (-1, 0, 1):
                    nb = (c[0] + d0, c[1] + d1, c[2] + d2)
                    if (d0, d1, d2) != (0, 0, 0) and nb not in level:
                        buffer.add(nb)
    return flags, morton_sorted(children), morton_sorted(buffer)
