"""Lattice Green's function of the 7-point Laplacian (Sec. 2, Eqs. GL and GL_B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed
--------------------
* Eq. GL_B:  G(n) = - int_0^inf exp(-6t) I_{n1}(2t) I_{n2}(2t) I_{n3}(2t) dt.
  With the exponentially scaled Bessel function ive(k, z) = exp(-z) I_k(z)
  the integrand is ive(n1,2t) ive(n2,2t) ive(n3,2t).  The paper only asks for
  "an adaptive Gauss-Kronrod quadrature or alike"; here the integral over
  [0, T] is a fixed composite Gauss-Legendre rule on geometrically growing
  panels (identical nodes for every n, so one table of ive values serves all
  points), and [T, inf) is integrated term by term from the large-argument
  (Hankel) expansion of ive, which is exact up to the truncated terms.
* Far-field expansions A^2_G and A^3_G (Sec. 2).  The printed A^3 adds the
  degree-8 polynomial correction; numerically the correction has to be
  SUBTRACTED (with "+" the error of A^3 is exactly twice that of A^2).  This
  module implements A^3 = A^2 - p(x) / (128 pi |x|^13).
* Switch (Sec. 2): quadrature for |n| <= 100, A^3 for 100 < |n| <= 600,
  A^2 beyond; |n| is read as the Euclidean norm.

Pins (tests/test_oracle_lgf.py): Watson's closed form for G(0);
L_Q G = delta at many points (near and across the table radius); the decay
rates |G - A^2| ~ |n|^-5 and |G - A^3| ~ |n|^-7; agreement with an adaptive
scipy quadrature; the paper's |eps| <~ 1e-12 at the switch radii.
"""
from __future__ import annotations

import numpy as np
from scipy import special

TABLE_RADIUS = 100.0
ASYM_RADIUS = 600.0

# Quadrature on [0, T]: one panel [0, t0], then panels growing by ratio r.
_T = 1.0e7
_T0 = 1.0e-3
_RATIO = 1.5
_NGAUSS = 20
_TAIL_TERMS = 8


def _nodes():
    x, w = np.polynomial.legendre.leggauss(_NGAUSS)
    br = [0.0, _T0]
    while br[-1] < _T:
        br.append(min(br[-1] * _RATIO, _T))
    br = np.asarray(br)
    a, b = br[:-1], br[1:]
    t = (0.5 * (b - a)[:, None] * (x[None, :] + 1.0) + a[:, None]).ravel()
    wt = (0.5 * (b - a)[:, None] * w[None, :]).ravel()
    return t, wt


_t_nodes, _t_weights = _nodes()
_ive_cache: dict[int, np.ndarray] = {}


def _ive_row(k: int) -> np.ndarray:
    """ive(k, 2 t_j) on the fixed quadrature nodes (cached per order)."""
    row = _ive_cache.get(k)
    if row is None:
        row = special.ive(k, 2.0 * _t_nodes)
        _ive_cache[k] = row
    return row


def _hankel_series(k: int, terms: int) -> np.ndarray:
    """Coefficients b_m of ive(k, 2t) ~ (4 pi t)^-1/2 sum_m b_m t^-m.

    From ive(k, z) ~ (2 pi z)^-1/2 sum_m (-1)^m a_m(k) z^-m with
    a_m = prod_{j=1..m} (4k^2 - (2j-1)^2) / (m! 8^m), and z = 2t.
    """
    mu = 4.0 * k * k
    a = [1.0]
    for m in range(1, terms + 1):
        a.append(a[-1] * (mu - (2 * m - 1) ** 2) / (8.0 * m))
    return np.array([(-1) ** m * a[m] * 2.0 ** (-m) for m in range(terms + 1)])


def _tail(n) -> float:
    """int_T^inf of the product of three ive's, from their Hankel series."""
    c = np.array([1.0])
    for k in n:
        c = np.convolve(c, _hankel_series(abs(int(k)), _TAIL_TERMS))[: _TAIL_TERMS + 1]
    m = np.arange(c.size)
    return float((4.0 * np.pi) ** -1.5 * np.sum(c * _T ** (-0.5 - m) / (0.5 + m)))


def lgf_quadrature(n) -> float:
    """G(n) for one integer point by quadrature of Eq. GL_B (FP64)."""
    a, b, c = (abs(int(v)) for v in n)
    body = float(np.dot(_t_weights, _ive_row(a) * _ive_row(b) * _ive_row(c)))
    return -(body + _tail((a, b, c)))


def lgf_quadrature_many(pts, chunk: int = 512) -> np.ndarray:
    """G at many integer points (K, 3) by the same rule as ``lgf_quadrature``."""
    pts = np.abs(np.asarray(pts, dtype=np.int64).reshape(-1, 3))
    out = np.empty(pts.shape[0])
    # Hankel-series tails: product of the three per-axis series, truncated.
    m = np.arange(_TAIL_TERMS + 1)
    series = {}
    for k in np.unique(pts):
        series[int(k)] = _hankel_series(int(k), _TAIL_TERMS)
    for i0 in range(0, pts.shape[0], chunk):
        p = pts[i0:i0 + chunk]
        B0 = np.stack([_ive_row(int(k)) for k in p[:, 0]])
        B1 = np.stack([_ive_row(int(k)) for k in p[:, 1]])
        B2 = np.stack([_ive_row(int(k)) for k in p[:, 2]])
        body = (B0 * B1 * B2) @ _t_weights
        tail = np.empty(p.shape[0])
        for r, (a, b, c) in enumerate(p.tolist()):
            cc = np.convolve(np.convolve(series[a], series[b])[: m.size], series[c])[: m.size]
            tail[r] = (4.0 * np.pi) ** -1.5 * np.sum(cc * _T ** (-0.5 - m) / (0.5 + m))
        out[i0:i0 + chunk] = -(body + tail)
    return out


def asym2(x) -> np.ndarray:
    """Two-term far-field expansion A^2_G (Sec. 2); x has shape (..., 3)."""
    x = np.asarray(x, dtype=np.float64)
    x1, x2, x3 = x[..., 0], x[..., 1], x[..., 2]
    r2 = x1 * x1 + x2 * x2 + x3 * x3
    r = np.sqrt(r2)
    q = x1**4 + x2**4 + x3**4 - 3.0 * (x1**2 * x2**2 + x1**2 * x3**2 + x2**2 * x3**2)
    return -1.0 / (4.0 * np.pi * r) - q / (16.0 * np.pi * r**7)


def asym3(x) -> np.ndarray:
    """Three-term far-field expansion A^3_G with the sign-corrected last term."""
    x = np.asarray(x, dtype=np.float64)
    x1, x2, x3 = x[..., 0], x[..., 1], x[..., 2]
    a, b, c = x1 * x1, x2 * x2, x3 * x3
    r = np.sqrt(a + b + c)
    p = (-228.0 * (b * c * a * a + b * c * c * a + b * b * c * a)
         + 621.0 * (a * a * b * b + c * c * b * b + a * a * c * c)
         - 244.0 * (b * a**3 + c * a**3 + b**3 * a + c**3 * a + b * c**3 + b**3 * c)
         + 23.0 * (a**4 + b**4 + c**4))
    return asym2(x) - p / (128.0 * np.pi * r**13)


class LGF:
    """G(n) with the paper's table / A^3 / A^2 switch, memoised per point.

    Values inside the table radius are computed by quadrature on first use
    and cached under the canonical key (sorted absolute coordinates), which
    is valid because G has the 48-fold symmetry of the cubic lattice.
    """

    def __init__(self, table_radius: float = TABLE_RADIUS, asym_radius: float = ASYM_RADIUS):
        self.table_radius = float(table_radius)
        self.asym_radius = float(asym_radius)
        self._memo: dict[tuple[int, int, int], float] = {}

    def _table_many(self, keys: np.ndarray) -> np.ndarray:
        """Quadrature values for canonical keys (K, 3), memoised."""
        vals = np.empty(keys.shape[0])
        todo = []
        for i, key in enumerate(map(tuple, keys.tolist())):
            v = self._memo.get(key)
            if v is None:
                todo.append(i)
            else:
                vals[i] = v
        if todo:
            new = lgf_quadrature_many(keys[todo])
            vals[todo] = new
            for i, v in zip(todo, new.tolist()):
                self._memo[tuple(keys[i].tolist())] = v
        return vals

    def __call__(self, pts) -> np.ndarray:
        """Evaluate G at integer points, shape (..., 3) -> (...)."""
        pts = np.asarray(pts, dtype=np.int64)
        shape = pts.shape[:-1]
        flat = pts.reshape(-1, 3)
        out = np.empty(flat.shape[0], dtype=np.float64)
        r = np.sqrt(np.sum(flat.astype(np.float64) ** 2, axis=1))
        near = r <= self.table_radius
        mid = (~near) & (r <= self.asym_radius)
        far = r > self.asym_radius
        if np.any(near):
            canon = np.sort(np.abs(flat[near]), axis=1)[:, ::-1]
            uniq, inv = np.unique(canon, axis=0, return_inverse=True)
            vals = self._table_many(uniq)
            out[near] = vals[inv.ravel()]
        if np.any(mid):
            out[mid] = asym3(flat[mid])
        if np.any(far):
            out[far] = asym2(flat[far])
        return out.reshape(shape)

    def table(self, reach: int) -> np.ndarray:
        """Dense array T[i+reach, j+reach, k+reach] = G(i, j, k), |i|,|j|,|k| <= reach."""
        ax = np.arange(-reach, reach + 1)
        grid = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1)
        return self(grid)


def watson_g0() -> float:
    """Watson's closed form: G(0) = -(sqrt 6 / (32 pi^3)) Gamma(1/24) Gamma(5/24)
    Gamma(7/24) Gamma(11/24) / 6 (the simple-cubic Watson integral over -6)."""
    g = special.gamma
    w = np.sqrt(6.0) / (32.0 * np.pi**3) * g(1 / 24) * g(5 / 24) * g(7 / 24) * g(11 / 24)
    return -w / 6.0
