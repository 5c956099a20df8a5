"""The plan autotuner: every candidate plan computes the same operator, and the
chosen plan is left on the context."""
import numpy as np
import pytest
import torch

from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.autotune import autotune
from paper_1911_10228_gb300.inputs import random_sparse_problem

pytestmark = pytest.mark.gpu


def _solve(c, probs):
    bs = F.BlockSet(c, [p.coords for p in probs], [p.h0 for p in probs])
    for i, p in enumerate(probs):
        for l, f in enumerate(p.f):
            bs.load_source(i, l, torch.as_tensor(f))
    bs.solve()
    out = [bs.potential(i, l).cpu().numpy() for i, p in enumerate(probs) for l in range(p.n_levels)]
    bs.close()
    return out


def test_autotune_picks_a_plan_and_plans_agree():
    probs = [random_sparse_problem(s, N=8, nblk_range=(40, 300)) for s in (2, 5, 11)]
    c = F.Context(N=8, n_interp=6, precision="fp64")
    ref = _solve(c, probs)
    cands = [(0, (4, 4, 8)), (100, (4, 4, 8)), (30, (2, 4, 8))]
    best, table = autotune(c, [p.coords for p in probs], [p.h0 for p in probs],
                           sources=[[torch.as_tensor(f) for f in p.f] for p in probs], candidates=cands, reps=2)
    assert set(table) == {(p, t) for p, t in cands}
    assert all(v > 0 for v in table.values())
    assert best == min(table, key=table.get) and c.plan == best
    got = _solve(c, probs)
    scale = max(np.max(np.abs(r)) for r in ref)
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) < 1e-12 * scale
    c.close()
