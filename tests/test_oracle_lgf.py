"""Pins of the oracle's lattice Green's function (Sec. 2) against facts that do
not come from the oracle itself."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle.lgf import LGF, asym2, asym3, lgf_quadrature, lgf_quadrature_many, watson_g0

# Watson's constant for the simple cubic lattice (the value the closed form
# gives; also the classical literature value 1.516386059151978...).
WATSON_SC = 1.516386059151978


def test_watson_closed_form():
    assert abs(watson_g0() + WATSON_SC / 6.0) < 1e-14
    assert abs(lgf_quadrature((0, 0, 0)) - watson_g0()) < 2e-15


def _lq(G, n):
    n = np.asarray(n)
    e = np.eye(3, dtype=np.int64)
    pts = np.stack([n + e[0], n - e[0], n + e[1], n - e[1], n + e[2], n - e[2], n])
    v = G(pts)
    return v[:6].sum() - 6.0 * v[6]


def test_lq_of_g_is_delta(G):
    """L_Q G = delta: the LGF is the fundamental solution of the 7-point operator."""
    assert abs(_lq(G, (0, 0, 0)) - 1.0) < 1e-14
    rng = np.random.default_rng(3)
    pts = [(1, 0, 0), (1, 1, 0), (1, 1, 1), (5, 3, 2), (17, -4, 9)]
    pts += [tuple(v) for v in rng.integers(-50, 51, (40, 3)) if np.any(v)]
    for n in pts:
        assert abs(_lq(G, n)) < 5e-15, n


def test_neighbour_identity(G):
    """Consequence of L_Q G = delta at the origin and symmetry: G(1,0,0) = G(0) + 1/6."""
    assert abs(G([1, 0, 0]) - G([0, 0, 0]) - 1.0 / 6.0) < 1e-15


def test_adaptive_quadrature_agrees():
    """An independent adaptive quadrature of Eq. GL_B (scipy QUADPACK)."""
    for n in [(2, 1, 0), (7, 3, 1), (12, 0, 5)]:
        f = lambda t: special.ive(n[0], 2 * t) * special.ive(n[1], 2 * t) * special.ive(n[2], 2 * t)
        a = integrate.quad(f, 0, 50, limit=400, epsabs=1e-15, epsrel=1e-13)[0]
        b = integrate.quad(f, 50, np.inf, limit=400, epsabs=1e-15, epsrel=1e-13)[0]
        assert abs(-(a + b) - lgf_quadrature(n)) < 1e-11, n


@pytest.mark.parametrize("direction", [(1, 0, 0), (1, 1, 0), (1, 1, 1), (3, 2, 1)])
def test_asymptotic_orders(direction):
    """G - A^2 = O(|n|^-5) and G - A^3 = O(|n|^-7) (q-term error O(|n|^{-2q-1}))."""
    d = np.asarray(direction)
    scales = [12, 24, 48]
    pts = np.stack([s * d for s in scales])
    g = lgf_quadrature_many(pts)
    e2 = np.abs(g - asym2(pts))
    e3 = np.abs(g - asym3(pts))
    r2 = np.log2(e2[:-1] / e2[1:])
    r3 = np.log2(e3[:-1] / e3[1:])
    assert np.all(np.abs(r2 - 5.0) < 0.5), r2
    assert np.all(np.abs(r3 - 7.0) < 0.5), r3


def test_switch_radii_error_bound():
    """The paper's switch keeps |eps| <~ 1e-12: A^3 just outside |n| = 100,
    A^2 just outside |n| = 600."""
    p100 = np.array([[101, 0, 0], [60, 60, 50], [71, 71, 1]])
    assert np.max(np.abs(lgf_quadrature_many(p100) - asym3(p100))) < 1e-12
    p600 = np.array([[601, 0, 0], [350, 350, 340]])
    assert np.max(np.abs(lgf_quadrature_many(p600) - asym2(p600))) < 1e-12


def test_farfield_leading_term(G):
    n = np.array([[80, 0, 0], [0, 0, 300], [400, 400, 400]])
    r = np.linalg.norm(n, axis=1)
    assert np.all(np.abs(G(n) * (-4 * np.pi * r) - 1.0) < 1e-4)


def test_cubic_symmetry(G):
    rng = np.random.default_rng(0)
    for n in rng.integers(-40, 41, (10, 3)):
        perm = rng.permutation(3)
        sgn = rng.choice([-1, 1], 3)
        assert G(n) == G(n[perm] * sgn)
