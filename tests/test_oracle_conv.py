"""Pins of the plain definitions: direct sum, Hockney convolution, 7-point Laplacian."""
import numpy as np

from oracle.conv import direct_sum, hockney, laplacian


def test_laplacian_of_quadratic():
    """L_Q^{(h)} |x|^2 = 6 for any spacing h (second differences of x^2 are 2h^2)."""
    h = 0.37
    ax = np.arange(7) * h
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    u = X**2 + Y**2 + Z**2 + 3.0 * X - Y
    assert np.allclose(laplacian(u, h), 6.0, atol=1e-12)


def test_direct_sum_inverts_laplacian(G):
    """L_Q^{(h)} (h^2 G * f) = f on a box that contains supp f plus one cell."""
    rng = np.random.default_rng(1)
    M = 7
    f = np.zeros((M, M, M))
    f[1:-1, 1:-1, 1:-1] = rng.standard_normal((M - 2, M - 2, M - 2))
    ax = np.arange(M)
    pts = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    h = 0.5
    u = direct_sum(G, pts, f.ravel(), pts, h=h).reshape(M, M, M)
    assert np.max(np.abs(laplacian(u, h) - f[1:-1, 1:-1, 1:-1])) < 1e-12


def test_point_source_gives_g(G):
    pts = np.array([[0, 0, 0]])
    tg = np.array([[3, 1, 0], [0, 0, 0], [-5, 2, 2]])
    u = direct_sum(G, pts, np.array([2.0]), tg)
    assert np.allclose(u, 2.0 * G(tg), rtol=0, atol=1e-16)


def test_hockney_equals_direct(G):
    rng = np.random.default_rng(2)
    f = rng.standard_normal((6, 5, 7))
    u = hockney(G, f, h=2.0)
    ax = [np.arange(s) for s in f.shape]
    pts = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1).reshape(-1, 3)
    ud = direct_sum(G, pts, f.ravel(), pts, h=2.0).reshape(f.shape)
    assert np.max(np.abs(u - ud)) < 1e-13 * np.max(np.abs(ud))
