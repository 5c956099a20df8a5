"""The allocation-free entry point flgf_convolve_static.

It serves callers that cannot allocate device memory while they compute
(another framework owns the memory pool, a latency-critical loop must avoid
cudaMalloc's implicit synchronisation, or all device memory is reserved up
front): its scratch lives in a fixed array the library declares statically.
Its results must match the block-set path on the same blocks, call after
call, since every call reuses the same scratch.  This file is collected last
so a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

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


def test_static_convolution_rejects_oversized_input():
    ctx = F.Context(N=8, n_interp=6, precision="fp32")
    coords = box_coords(4, 4, 3)                       # 48 blocks: above the fixed scratch
    f = torch.zeros((len(coords), 8, 8, 8), device="cuda")
    with pytest.raises(F.FLGFError, match="32 blocks"):
        ctx.convolve_static(coords, f)
    with pytest.raises(F.FLGFError, match="4x4x4"):
        ctx.convolve_static(np.array([[0, 0, 0], [5, 0, 0]]), torch.zeros((2, 8, 8, 8), device="cuda"))
    ctx.close()
