"""Host source loads run on the library's copy stream and may overlap the solve
in flight: a load issued while a solve runs must not change that solve's
result, and the next solve must see the new source."""
import numpy as np
import pytest
import torch

from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import config_plain_32

pytestmark = pytest.mark.gpu


def _alone(c, p, f):
    bs = F.BlockSet(c, [p.coords], [p.h0])
    bs.load_source(0, 0, f)
    bs.solve()
    u = bs.potential(0, 0).cpu().numpy()
    bs.close()
    return u


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_overlapped_loads_keep_each_solve_consistent(precision, graph):
    p = config_plain_32()
    c = F.Context(N=p.N, n_interp=6, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    rng = np.random.default_rng(5)
    srcs = [torch.as_tensor(p.f[0]).to(dt), torch.as_tensor(rng.standard_normal(p.f[0].shape)).to(dt),
            torch.as_tensor(np.roll(p.f[0], 3, axis=1)).to(dt)]
    ref = [_alone(c, p, f) for f in srcs]
    bs = F.BlockSet(c, [p.coords], [p.h0])
    bs.set_option(F.OPT_GRAPH, graph)
    host = [f.pin_memory() for f in srcs]
    bs.load_source(0, 0, host[0])
    bs.solve()
    for i in range(1, len(srcs) + 1):
        if i < len(srcs):
            if i == 2:   # a device load between host loads takes the same order
                bs.load_source(0, 0, srcs[i].cuda())
            else:
                bs.load_source(0, 0, host[i])     # overlaps the solve in flight
        out = np.empty(p.f[0].shape, dtype=np.float64 if precision == "fp64" else np.float32)
        bs.potential_host(0, 0, out=out)
        assert np.array_equal(out, ref[i - 1]), i - 1
        if i < len(srcs):
            bs.solve()
    bs.close()
    c.close()
