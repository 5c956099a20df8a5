"""Error paths of the C ABI, exercised by host-side failure injection.

Nothing here faults the GPU: an allocation failure is reported by the
library's allocation wrapper without allocating (FLGF_CTX_FAIL_ALLOC), and a
missing halo block is simulated by marking one entry of a coarse-fine
interpolation list absent (FLGF_OPT_FAULT_HALO), a case the kernel handles by
reading zero and raising the device error flag that flgf_get_potential
reports.  The adjoint's scatter-adds use atomics, so repeated gradients agree
to round-off, which is checked here too.
"""
import numpy as np
import pytest
import torch

from oracle.adjoint import multires_adjoint
from oracle.multires import multires_solve
from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import box_coords, refine_mesh, torus

pytestmark = pytest.mark.gpu


def _mesh():
    return refine_mesh(lambda x: torus(x, (0.5, 0.5, 0.5), 0.22, 0.05), box_coords(4), 8, 1.0 / 32, 2, 0.3)


def _load(bs, p):
    for l, f in enumerate(p.f):
        bs.load_source(0, l, torch.as_tensor(f))


@pytest.mark.parametrize("which", [1, 2, 6, 11])
def test_allocation_failure_reports_enomem_and_retry_succeeds(G, which):
    """The which-th of the 11 device allocations of block-set creation fails:
    ENOMEM, the partly built block set is released, and the next creation
    works."""
    p = _mesh()
    ctx = F.Context(N=8, n_interp=6, precision="fp64")
    ctx.fail_alloc(which)
    with pytest.raises(F.FLGFError) as ei:
        F.BlockSet(ctx, [p.coords], [p.h0])
    assert ei.value.code == F.FLGF_ENOMEM, str(ei.value)
    bs = F.BlockSet(ctx, [p.coords], [p.h0])   # the hook is one-shot
    _load(bs, p)
    bs.solve()
    ref, leaf = multires_solve(G, p.coords, p.f, 8, 6, p.h0)
    scale = max(np.max(np.abs(r[m])) for r, m in zip(ref, leaf))
    for l in range(p.n_levels):
        u = bs.potential(0, l).cpu().numpy()
        assert np.max(np.abs(u[leaf[l]] - ref[l][leaf[l]])) < 1e-10 * scale
    bs.close()
    ctx.close()


def test_adjoint_allocation_failure_then_retry_matches_oracle(G):
    """The adjoint buffers are allocated on first use: a failure there gives
    ENOMEM and leaves the block set usable; the retry builds them and the
    gradient matches the oracle's explicit transposes."""
    p = _mesh()
    rng = np.random.default_rng(5)
    g = [rng.standard_normal((len(c), 8, 8, 8)) for c in p.coords]
    ctx = F.Context(N=8, n_interp=6, precision="fp64")
    bs = F.BlockSet(ctx, [p.coords], [p.h0])
    ctx.fail_alloc(3)
    with pytest.raises(F.FLGFError) as ei:
        bs.load_adjoint(0, 0, torch.as_tensor(g[0]))
    assert ei.value.code == F.FLGF_ENOMEM, str(ei.value)
    for l, x in enumerate(g):
        bs.load_adjoint(0, l, torch.as_tensor(x))
    bs.solve_adjoint()
    ref = multires_adjoint(G, p.coords, g, 8, 6, p.h0)
    scale = max(np.max(np.abs(r)) for r in ref)
    for l in range(p.n_levels):
        got = bs.gradient(0, l).cpu().numpy()
        assert np.max(np.abs(got - ref[l])) < 1e-10 * scale
    bs.close()
    ctx.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_missing_halo_block_reports_edevice(graph):
    """A coarse-fine interpolation list that names an absent halo block: the
    solve completes, and reading the potential returns FLGF_EDEVICE (host and
    device reads alike).  A block set without the injected fault is clean."""
    p = _mesh()
    assert p.n_levels == 2
    ctx = F.Context(N=8, n_interp=6, precision="fp32")
    clean = F.BlockSet(ctx, [p.coords], [p.h0])
    bad = F.BlockSet(ctx, [p.coords], [p.h0])
    for bs in (clean, bad):
        _load(bs, p)
        bs.set_option(F.OPT_GRAPH, graph)
    bad.set_option(F.OPT_FAULT_HALO, 1)
    for bs in (clean, bad):
        bs.solve()
    clean.potential(0, 1)
    clean.potential_host(0, 1)
    with pytest.raises(F.FLGFError) as ei:
        bad.potential(0, 1)
    assert ei.value.code == F.FLGF_EDEVICE, str(ei.value)
    with pytest.raises(F.FLGFError) as ei:
        bad.potential_host(0, 1)
    assert ei.value.code == F.FLGF_EDEVICE
    # the flag belongs to the faulted block set's solves only
    clean.solve()
    clean.potential(0, 1)
    clean.close()
    bad.close()
    ctx.close()


def test_fault_hooks_reject_bad_values():
    ctx = F.Context(N=8, n_interp=6, precision="fp32")
    with pytest.raises(F.FLGFError):
        ctx.fail_alloc(-1)
    bs = F.BlockSet(ctx, [[box_coords(2)]], [1.0])
    with pytest.raises(F.FLGFError):
        bs.set_option(F.OPT_FAULT_HALO, 2)
    with pytest.raises(F.FLGFError):       # one level: no coarse-fine interpolation to corrupt
        bs.set_option(F.OPT_FAULT_HALO, 1)
    bs.close()
    ctx.close()


def test_fp64_adjoint_repeats_to_round_off():
    """Two adjoint solves of the same seeds: identical up to the order of the
    atomic scatter-adds of the transposed coarse-fine interpolation."""
    p = _mesh()
    rng = np.random.default_rng(9)
    ctx = F.Context(N=8, n_interp=6, precision="fp64")
    bs = F.BlockSet(ctx, [p.coords], [p.h0])
    for l, c in enumerate(p.coords):
        bs.load_adjoint(0, l, torch.as_tensor(rng.standard_normal((len(c), 8, 8, 8))))
    runs = []
    for _ in range(2):
        bs.solve_adjoint()
        runs.append([bs.gradient(0, l).cpu().numpy() for l in range(p.n_levels)])
    scale = max(np.max(np.abs(x)) for x in runs[0])
    # a coarse cell sums up to ~64 fine contributions; reordering a sum of M
    # terms moves it by at most about M eps sum|terms|, a few times 64 * 1.1e-16
    # of the scale (measured up to 1.06e-14); a race or a lost update would be
    # orders of magnitude larger
    for a, b in zip(*runs):
        assert np.max(np.abs(a - b)) <= 1e-13 * scale
    bs.close()
    ctx.close()
