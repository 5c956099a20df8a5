"""Pins of the vortex-ring manufactured solution (Sec. 3.1, Eqs. streamfunc,
streamfunc_f): the analytic vorticity omega = Laplacian(Psi) used as the source
must be the Laplacian of the analytic streamfunction used as the answer."""
import numpy as np

from paper_1911_10228_gb300.inputs import config_vortex_ring, split_blocks, vortex_ring, vortex_ring_vector

C = np.array([0.5, 0.5, 0.5])
R = 0.125


def _points(n, seed=0):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform([0.25, 0.25, 0.4], [0.75, 0.75, 0.6])
        d = p - C
        if np.hypot(np.hypot(d[0], d[1]) - R, d[2]) < 0.9 * R:
            pts.append(p)
    return np.array(pts)


def _fd_laplacian(f, pts, h):
    """Fourth-order central differences along each axis."""
    out = np.zeros(len(pts))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        out += (-f(pts + 2 * e) + 16 * f(pts + e) - 30 * f(pts) + 16 * f(pts - e) - f(pts - 2 * e)) / (12 * h * h)
    return out


def test_vorticity_is_the_laplacian_of_the_streamfunction():
    pts = _points(200)
    w = vortex_ring(pts)[1]
    errs = []
    for h in (4e-3, 2e-3, 1e-3):
        lap = _fd_laplacian(lambda q: vortex_ring(q)[0], pts, h)
        errs.append(np.max(np.abs(lap - w)) / np.max(np.abs(w)))
    assert errs[-1] < 1e-6
    # fourth-order decay of the difference: the formula, not the stencil, is exact
    assert errs[0] / errs[1] > 12 and errs[1] / errs[2] > 12


def test_support_and_symmetry():
    pts = _points(100, seed=1)
    psi, w = vortex_ring(pts)
    mirror = pts.copy()
    mirror[:, 1] = 2 * C[1] - mirror[:, 1]          # psi_x is odd under y -> -y
    psi_m, w_m = vortex_ring(mirror)
    assert np.allclose(psi_m, -psi, rtol=1e-12, atol=0) and np.allclose(w_m, -w, rtol=1e-12, atol=1e-9)
    far = np.array([[0.5, 0.5, 0.5], [0.5, 0.5 + 2.01 * R, 0.5], [0.5, 0.5 + R, 0.5 + 1.01 * R]])
    assert np.all(vortex_ring(far)[0] == 0) and np.all(vortex_ring(far)[1] == 0)


def test_global_split_keeps_the_topology():
    p, psi = config_vortex_ring(3, 8, 4, 0)
    q, _ = config_vortex_ring(3, 8, 4, 1)
    assert [8 * len(c) for c in p.coords] == [len(c) for c in q.coords]
    assert np.isclose(q.h0, p.h0 / 2)
    # every split block's parent is a block of the coarser mesh on the same level
    for a, b in zip(p.coords, split_blocks(p.coords)):
        assert {tuple(x) for x in (b >> 1).tolist()} == {tuple(x) for x in a.tolist()}
    # the mesh satisfies the solver's nesting rule: non-leaf blocks have all 8 children
    leaf = q.leaf_masks()
    for l in range(len(q.coords) - 1):
        kids = {tuple(x) for x in q.coords[l + 1].tolist()}
        for c in q.coords[l][~leaf[l]]:
            assert all((2 * c[0] + i, 2 * c[1] + j, 2 * c[2] + k) in kids for i, j, k in np.ndindex(2, 2, 2))


def test_vector_components():
    """The y component is the x component rotated by 90 degrees about the ring
    axis, its vorticity is its Laplacian, and the field is divergence-free."""
    pts = _points(150, seed=2)
    psi, w = vortex_ring_vector(pts)
    assert np.array_equal(psi[:, 0], vortex_ring(pts)[0]) and np.all(psi[:, 2] == 0) and np.all(w[:, 2] == 0)
    rot = pts.copy()                                    # (x, y) -> (y', -x') about the axis
    d = pts - C
    rot[:, 0], rot[:, 1] = C[0] - d[:, 1], C[1] + d[:, 0]
    psi_rot = vortex_ring_vector(rot)[0]              # Psi(R p) = R Psi(p), R (vx, vy) = (-vy, vx)
    assert np.allclose(psi_rot[:, 1], psi[:, 0], rtol=1e-10, atol=1e-12 * np.max(np.abs(psi)))
    assert np.allclose(psi_rot[:, 0], -psi[:, 1], rtol=1e-10, atol=1e-12 * np.max(np.abs(psi)))
    lap = _fd_laplacian(lambda q: vortex_ring_vector(q)[0][:, 1], pts, 1e-3)
    assert np.max(np.abs(lap - w[:, 1])) < 1e-6 * np.max(np.abs(w[:, 1]))
    h = 1e-3                                            # fourth-order first derivatives
    div = np.zeros(len(pts))
    size = np.zeros(len(pts))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        g = lambda q: vortex_ring_vector(q)[0][:, a]
        da = (-g(pts + 2 * e) + 8 * g(pts + e) - 8 * g(pts - e) + g(pts - 2 * e)) / (12 * h)
        div += da
        size += np.abs(da)
    assert np.max(np.abs(div)) < 1e-6 * np.max(size)
