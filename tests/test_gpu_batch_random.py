"""Batched random sparse refined problems (the batched workload's generator at
small sizes) against the oracle, problem by problem."""
import numpy as np
import pytest
import torch

from oracle.multires import multires_solve
from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import random_sparse_problem

pytestmark = pytest.mark.gpu

_REF = {}


# plan: (pair-list percentage, dense tile); 0 sends every tile to the dense
# parent-group kernel, 100 every tile that is not completely full to the
# pair-list kernel
PLANS = [None, (0, (4, 4, 8)), (100, (2, 4, 8)), (50, (4, 4, 4))]


@pytest.mark.parametrize("plan", PLANS, ids=["default", "dense", "list", "mixed"])
# FP32: within 1e-5 of the FP64 oracle (measured 8e-7 to 1e-6 on these problems)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_random_sparse_batch_matches_oracle(G, precision, tol, plan):
    probs = [random_sparse_problem(s, N=8, nblk_range=(8, 120)) for s in (1, 4, 7, 9)]
    assert max(p.n_levels for p in probs) >= 2
    c = F.Context(N=8, n_interp=6, precision=precision)
    if plan is not None:
        c.set_plan(list_pct=plan[0], tile=plan[1])
    bs = F.BlockSet(c, [p.coords for p in probs], [p.h0 for p in probs])
    for i, p in enumerate(probs):
        for l, f in enumerate(p.f):
            bs.load_source(i, l, torch.as_tensor(f))
    bs.set_option(F.OPT_GRAPH, 1)
    bs.solve()
    for i, p in enumerate(probs):
        if i not in _REF:  # shared by the FP64 and FP32 cases
            _REF[i] = multires_solve(G, p.coords, p.f, 8, 6, p.h0)
        ref, leaf = _REF[i]
        scale = max(np.max(np.abs(r[m])) for r, m in zip(ref, leaf))
        for l in range(p.n_levels):
            u = bs.potential(i, l).double().cpu().numpy()
            assert np.max(np.abs(u[leaf[l]] - ref[l][leaf[l]])) < tol * scale, (i, l)
    bs.close()
    c.close()


def test_plan_options_are_validated():
    c = F.Context(N=8, n_interp=4, precision="fp32")
    for bad in (dict(list_pct=-1), dict(list_pct=101), dict(tile=(0, 4, 4)), dict(tile=(8, 8, 8)),
                dict(tile=(2, 8, 8))):
        with pytest.raises(F.FLGFError):
            c.set_plan(**bad)
    c.set_plan(list_pct=0, tile=(8, 4, 4))
    c.close()
