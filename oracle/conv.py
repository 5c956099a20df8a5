"""Plain definitions: discrete convolution with the LGF and the 7-point Laplacian.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``direct_sum``  -- Eq. discretConv written out: u(n) = sum_m G(n - m) f(m),
  an O(#targets x #sources) double loop over lattice points (vectorised over
  the targets only).  Pinned by: a unit point source reproduces G; the
  7-point Laplacian of the result reproduces f (Eq. for L_Q u = f).
* ``hockney``     -- the same sum evaluated on a dense box by one zero-padded
  FFT of size (2M)^3 (exact up to round-off, because a linear convolution of
  two length-M supports needs 2M - 1 <= 2M points).  Pinned by equality with
  ``direct_sum`` on small boxes.
* ``laplacian``   -- L_Q u(n) = sum of the 6 face neighbours - 6 u(n),
  divided by h^2 (Sec. 2: the sign follows the denominator of Eq. GL).

Units: the lattice has spacing h; u = h^2 (G * f) solves L_Q^{(h)} u = f.
"""
from __future__ import annotations

import numpy as np


def direct_sum(G, src_pts, src_vals, tgt_pts, h: float = 1.0, chunk: int = 4096) -> np.ndarray:
    """u(n) = h^2 sum_m G(n - m) f(m) over the given source points.

    G        callable mapping integer points (..., 3) to LGF values.
    src_pts  (S, 3) integer lattice coordinates of sources, src_vals (S,).
    tgt_pts  (T, 3) integer lattice coordinates of targets.
    """
    src_pts = np.asarray(src_pts, dtype=np.int64)
    src_vals = np.asarray(src_vals, dtype=np.float64)
    tgt_pts = np.asarray(tgt_pts, dtype=np.int64)
    keep = src_vals != 0.0
    src_pts, src_vals = src_pts[keep], src_vals[keep]
    # Every lattice difference that can occur lies in a box; tabulate G there.
    lo = tgt_pts.min(axis=0) - src_pts.max(axis=0) if src_pts.size else np.zeros(3, np.int64)
    hi = tgt_pts.max(axis=0) - src_pts.min(axis=0) if src_pts.size else np.zeros(3, np.int64)
    ax = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
    grid = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1)
    gtab = G(grid)
    u = np.zeros(tgt_pts.shape[0], dtype=np.float64)
    for s0 in range(0, src_pts.shape[0], chunk):
        sp = src_pts[s0:s0 + chunk]
        sv = src_vals[s0:s0 + chunk]
        for t0 in range(0, tgt_pts.shape[0], chunk):
            tp = tgt_pts[t0:t0 + chunk]
            d = tp[:, None, :] - sp[None, :, :] - lo[None, None, :]
            u[t0:t0 + chunk] += gtab[d[..., 0], d[..., 1], d[..., 2]] @ sv
    return h * h * u


def hockney(G, f: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Free-space convolution of a dense box source f (shape (M0, M1, M2)) with G.

    Zero-pads to (2 M_d) per axis; the kernel array holds G at every lattice
    difference in [-(M_d - 1), M_d - 1] placed circularly, so the circular
    convolution equals the linear one on the M0 x M1 x M2 output window.
    """
    f = np.asarray(f, dtype=np.float64)
    M = f.shape
    P = tuple(2 * m for m in M)
    ax = [np.fft.fftfreq(P[d], d=1.0 / P[d]).astype(np.int64) for d in range(3)]
    grid = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1)
    kern = G(grid)  # G at circular index i -> lattice difference i (or i - P)
    F = np.fft.rfftn(f, s=P, axes=(0, 1, 2))
    K = np.fft.rfftn(kern, s=P, axes=(0, 1, 2))
    u = np.fft.irfftn(F * K, s=P, axes=(0, 1, 2))[: M[0], : M[1], : M[2]]
    return h * h * u


def laplacian(u: np.ndarray, h: float = 1.0) -> np.ndarray:
    """7-point Laplacian on the interior of a dense box (output shape M - 2)."""
    c = u[1:-1, 1:-1, 1:-1]
    s = (u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1]
         + u[1:-1, 2:, 1:-1] + u[1:-1, :-2, 1:-1]
         + u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2])
    return (s - 6.0 * c) / (h * h)
