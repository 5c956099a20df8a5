"""The allocation-free entry point flgf_convolve_static.

It serves callers that cannot allocate device memory while they compute
(another framework owns the memory pool, a latency-critical loop must avoid
cudaMalloc's implicit synchronisation, or all device memory is reserved up
front): its scratch lives in a fixed array the library declares statically.
Its results must match the block-set path on the same blocks and the oracle's
exact convolution, call after call, since every call reuses the same scratch.
This file is collected last so a failure here leaves every other test
already run.
"""
import numpy as np
import pytest
import torch

from oracle.conv import direct_sum, hockney
from oracle.flgf import blocks_to_dense, dense_to_blocks
from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import box_coords

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_convolution_matches_blockset_solve(precision):
    ctx = F.Context(N=8, n_interp=6, precision=precision)
    coords = box_coords(4, 4, 2, origin=(2, -4, 6))   # 32 blocks in one aligned 4x4x4 box
    bs = F.BlockSet(ctx, [[coords]], [0.5])
    rng = np.random.default_rng(11)
    for call in range(2):                              # two calls in a row share the scratch
        f = torch.as_tensor(rng.standard_normal((len(coords), 8, 8, 8)), device="cuda")
        bs.load_source(0, 0, f)
        bs.solve()
        ref = bs.potential(0, 0).double().cpu().numpy()
        got = ctx.convolve_static(coords, f, h=0.5).double().cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < TOL[precision], (call, err)
    bs.close()
    ctx.close()


@pytest.mark.parametrize("N", [8, 16])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_convolution_matches_oracle_exact_convolution(G, N, precision):
    """u = h^2 (G * f) over 32 blocks: the oracle's whole-box zero-padded FFT
    convolution (exact up to round-off, Eq. discretConv) on two calls in a row
    with different sources; at N = 8 also the brute-force direct sum on a few
    target cells."""
    ctx = F.Context(N=N, n_interp=6, precision=precision)
    coords = box_coords(4, 4, 2, origin=(-2, 0, 4))
    h = 0.25
    rng = np.random.default_rng(100 + N)
    for call in range(2):
        f = rng.standard_normal((len(coords), N, N, N))
        dense, origin = blocks_to_dense(coords, f, N)
        ref = dense_to_blocks(hockney(G, dense, h), origin, coords, N)
        got = ctx.convolve_static(coords, torch.as_tensor(f, device="cuda"), h=h).double().cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < TOL[precision], (call, err)
        if N == 8 and call == 0:
            pts = np.argwhere(np.ones(dense.shape, bool)) + origin
            tgt = pts[rng.choice(len(pts), 16, replace=False)]
            ds = direct_sum(G, pts, dense.reshape(-1), tgt, h)
            gi = [got[np.nonzero(np.all(coords == (t // N), axis=1))[0][0]][tuple(t % N)] for t in tgt]
            assert np.max(np.abs(np.array(gi) - ds)) / np.max(np.abs(ref)) < TOL[precision]
    ctx.close()


def test_static_convolution_rejects_oversized_input():
    ctx = F.Context(N=8, n_interp=6, precision="fp32")
    coords = box_coords(4, 4, 3)                       # 48 blocks: above the fixed scratch
    f = torch.zeros((len(coords), 8, 8, 8), device="cuda")
    with pytest.raises(F.FLGFError, match="32 blocks"):
        ctx.convolve_static(coords, f)
    with pytest.raises(F.FLGFError, match="4x4x4"):
        ctx.convolve_static(np.array([[0, 0, 0], [5, 0, 0]]), torch.zeros((2, 8, 8, 8), device="cuda"))
    ctx.close()


def test_static_convolution_checks_buffer_shapes_before_launch():
    """The C entry point cannot see buffer sizes, so the binding checks them:
    a source or output that does not hold one N^3 block per coordinate is
    rejected before anything is enqueued."""
    ctx = F.Context(N=8, n_interp=6, precision="fp32")
    coords = box_coords(2, 2, 2)
    good = torch.zeros((8, 8, 8, 8), device="cuda")
    with pytest.raises(ValueError):
        ctx.convolve_static(coords, torch.zeros((7, 8, 8, 8), device="cuda"))
    with pytest.raises(ValueError):
        ctx.convolve_static(coords, good, out=torch.empty((4, 8, 8, 8), device="cuda"))
    with pytest.raises(ValueError):
        ctx.convolve_static(coords, good, out=torch.empty((8, 8, 8, 8), device="cuda", dtype=torch.float64))
    with pytest.raises(ValueError):
        ctx.convolve_static(coords, good, out=torch.empty((8, 8, 8, 16), device="cuda")[..., ::2])
    out = torch.empty((8, 8, 8, 8), device="cuda")
    assert ctx.convolve_static(coords, good, out=out) is out
    ctx.close()
