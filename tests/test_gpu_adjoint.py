"""The adjoint solve (gradients) against the oracle's explicit transposes,
dot-product identities, finite differences, and the autograd integration."""
import numpy as np
import pytest
import torch

from oracle.adjoint import multires_adjoint
from paper_1911_10228_gb300 import autograd as AG
from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import box_coords, config_linked_tori, refine_mesh, torus

pytestmark = pytest.mark.gpu

_REF = {}


def _mesh():
    N, h0 = 8, 1.0 / 32
    p = refine_mesh(lambda x: torus(x, (0.5, 0.5, 0.5), 0.22, 0.05), box_coords(4), N, h0, 3, 0.3)
    return p


def _adjoint_gpu(c, p, g, correction=True):
    bs = F.BlockSet(c, [p.coords], [p.h0])
    if not correction:
        bs.set_option(F.OPT_CORRECTION, 0)
    for l, x in enumerate(g):
        bs.load_adjoint(0, l, torch.as_tensor(x))
    bs.solve_adjoint()
    out = [bs.gradient(0, l).double().cpu().numpy() for l in range(p.n_levels)]
    bs.close()
    return out


# FP32 (compensated coarse octree levels, the default on refined meshes):
# measured 4.3e-6 with the source correction, 1.3e-6 without.
@pytest.mark.parametrize("precision,correction,tol", [("fp64", True, 1e-10), ("fp64", False, 1e-10),
                                                      ("fp32", False, 1e-5), ("fp32", True, 1e-5)])
def test_adjoint_matches_oracle(G, precision, correction, tol):
    p = _mesh()
    rng = np.random.default_rng(21)
    g = [rng.standard_normal((len(c), 8, 8, 8)) for c in p.coords]
    key = correction
    if key not in _REF:
        _REF[key] = multires_adjoint(G, p.coords, g, 8, 6, p.h0, correction=correction)
    ref = _REF[key]
    c = F.Context(N=8, n_interp=6, precision=precision)
    got = _adjoint_gpu(c, p, g, correction)
    c.close()
    scale = max(np.max(np.abs(r)) for r in ref)
    for l in range(p.n_levels):
        err = np.max(np.abs(got[l] - ref[l])) / scale
        print(f"adjoint {precision} correction={correction} level {l}: rel err {err:.3e}")
        assert err < tol, (l, err)


@pytest.mark.parametrize("list_pct", [30, 0, 100], ids=["default", "dense", "list"])
def test_dot_product_identity_fp64(list_pct):
    """<A f, g> = <f, A^T g> on the GPU alone (sources on leaf blocks only),
    with the spectrum MAC on the dense kernel, the pair-list kernel or both."""
    p = _mesh()
    leaf = p.leaf_masks()
    rng = np.random.default_rng(22)
    f = [np.where(m[:, None, None, None], rng.standard_normal((len(c), 8, 8, 8)), 0.0) for c, m in zip(p.coords, leaf)]
    g = [rng.standard_normal((len(c), 8, 8, 8)) for c in p.coords]
    c = F.Context(N=8, n_interp=6, precision="fp64")
    c.set_plan(list_pct=list_pct)
    bs = F.BlockSet(c, [p.coords], [p.h0])
    for l in range(p.n_levels):
        bs.load_source(0, l, torch.as_tensor(f[l]))
        bs.load_adjoint(0, l, torch.as_tensor(g[l]))
    bs.solve()
    bs.solve_adjoint()
    a = sum(float(np.sum(bs.potential(0, l).cpu().numpy() * g[l])) for l in range(p.n_levels))
    b = sum(float(np.sum(f[l] * bs.gradient(0, l).cpu().numpy())) for l in range(p.n_levels))
    bs.close()
    c.close()
    assert abs(a - b) < 1e-12 * abs(a)


def test_autograd_gradient_linked_tori_against_finite_differences():
    """Two linked tori, 3 levels, 16^3 blocks (~26 M DoF): loss = 0.5 ||u - u_t||^2
    on leaf cells with u_t from a perturbed source.  The gradient from the
    backward pass (FP64 and FP32) is checked against central differences of the
    FP64 forward (h = 1e-3, exact for a quadratic loss) on 32 random entries."""
    from paper_1911_10228_gb300.inputs import cell_centres, smooth_field
    p = config_linked_tori()
    leaf = p.leaf_masks()
    keys = [(0, l) for l in range(p.n_levels)]
    pert = [f * (1.0 + 0.1 * smooth_field(cell_centres(c, 16, p.h0 / (1 << l)))) for l, (c, f) in
            enumerate(zip(p.coords, p.f))]
    masks = [torch.as_tensor(m[:, None, None, None], device="cuda") for m in leaf]
    grads = {}
    for prec in ("fp64", "fp32"):
        c = F.Context(N=16, n_interp=6, precision=prec)
        bs = F.BlockSet(c, [p.coords], [p.h0])
        with torch.no_grad():
            target = [t.clone() for t in AG.solve(bs, [torch.as_tensor(x, device="cuda") for x in pert])]
        src = [torch.as_tensor(x, device="cuda", dtype=c.dtype).requires_grad_(True) for x in p.f]
        u = AG.solve(bs, src)
        loss = 0.5 * sum(((ui - ti) * m).double().pow(2).sum() for ui, ti, m in zip(u, target, masks))
        loss.backward()
        grads[prec] = [s.grad.double().cpu().numpy() for s in src]
        if prec == "fp64":
            bs64, c64, target64 = bs, c, target
        else:
            bs.close()
            c.close()

    def loss64(ff):
        with torch.no_grad():
            uu = AG.solve(bs64, [torch.as_tensor(x, device="cuda") for x in ff])
            return float(0.5 * sum(((ui - ti) * m).pow(2).sum() for ui, ti, m in zip(uu, target64, masks)))

    rng = np.random.default_rng(0)
    checked = 0
    h = 1e-3
    while checked < 32:
        l = int(rng.integers(0, p.n_levels))
        b = int(rng.integers(0, len(p.coords[l])))
        if not leaf[l][b]:
            continue
        i, j, k = (int(v) for v in rng.integers(0, 16, 3))
        fp = [x.copy() for x in p.f]
        fm = [x.copy() for x in p.f]
        fp[l][b, i, j, k] += h
        fm[l][b, i, j, k] -= h
        fd = (loss64(fp) - loss64(fm)) / (2 * h)
        scale = max(abs(fd), 1e-6 * max(np.abs(x).max() for x in grads["fp64"]))
        assert abs(grads["fp64"][l][b, i, j, k] - fd) < 1e-6 * scale + 1e-9, (l, b, fd, grads["fp64"][l][b, i, j, k])
        checked += 1
    gmax = max(np.abs(x).max() for x in grads["fp64"])
    for l in range(p.n_levels):
        err = np.max(np.abs(grads["fp32"][l] - grads["fp64"][l])) / gmax
        print(f"linked tori gradient level {l}: FP32 vs FP64 rel err {err:.3e}")
        # The FP32 adjoint is held to 1e-4, the bound the hot-path contract sets for
        # it: the transposed source correction applies the 7-point stencil (x
        # 1/h^2) to the finer level's FP32 adjoint field, which amplifies its
        # rounding into the coarsest level's gradient (measured 2.4e-5 there,
        # 3e-6 and 2e-7 on the finer levels).
        assert err < 1e-4, (l, err)
    bs64.close()
    c64.close()
