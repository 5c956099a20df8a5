"""Method of manufactured solutions (Sec. 3.1, Fig. convergence_amr): the vortex
ring's analytic vorticity as the source, the analytic streamfunction as the
answer.  Global refinement with a fixed mesh topology must converge at second
order, with and without the source correction, whose influence on this
global-refinement study is negligible."""
import numpy as np
import pytest
import torch

from paper_1911_10228_gb300 import flgf as F
from paper_1911_10228_gb300.inputs import config_vortex_ring

pytestmark = pytest.mark.gpu


def _errors(c, p, psi, correction=True):
    bs = F.BlockSet(c, [p.coords], [p.h0])
    if not correction:
        bs.set_option(F.OPT_CORRECTION, 0)
    for l, f in enumerate(p.f):
        bs.load_source(0, l, torch.as_tensor(f))
    bs.solve()
    leaf = p.leaf_masks()
    num = den = s2 = a2 = 0.0
    for l in range(p.n_levels):
        u = bs.potential(0, l).double().cpu().numpy()[leaf[l]]
        ex = psi[l][leaf[l]]
        num = max(num, float(np.max(np.abs(u - ex))))
        den = max(den, float(np.max(np.abs(ex))))
        w = (p.h0 / (1 << l)) ** 3
        s2 += w * float(np.sum((u - ex) ** 2))
        a2 += w * float(np.sum(ex ** 2))
    bs.close()
    return num / den, np.sqrt(s2 / a2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n_levels", [1, 3])
def test_vortex_ring_second_order(precision, n_levels):
    c = F.Context(N=8, n_interp=6, precision=precision)
    runs = {}
    for corr in ((True, False) if n_levels > 1 else (True,)):
        errs = []
        for sp in (0, 1, 2):
            p, psi = config_vortex_ring(n_levels, 8, 4, sp)
            errs.append(_errors(c, p, psi, corr))
        for norm in (0, 1):
            orders = [np.log2(errs[i][norm] / errs[i + 1][norm]) for i in range(2)]
            print(f"{precision} L={n_levels} correction={corr} {'Linf' if norm == 0 else 'L2'}: "
                  f"{[f'{e[norm]:.3e}' for e in errs]} orders {[round(o, 3) for o in orders]}")
            assert 1.85 < orders[1] < 2.15, (corr, norm, orders)
            assert orders[0] > 1.8, (corr, norm, orders)
        runs[corr] = errs
    if n_levels > 1:   # correction on or off: the same error to 1 % (global refinement, 3 levels)
        for a, b in zip(runs[True], runs[False]):
            assert abs(a[0] - b[0]) < 0.01 * a[0] and abs(a[1] - b[1]) < 0.01 * a[1]
    c.close()


def test_vortex_ring_added_levels_and_correction():
    """Fixed base resolution, more refinement levels (Eq. ref_crit): the error on
    the finest level falls about fourfold per added level, and with five levels
    dropping the source correction leaves a visibly larger error there."""
    c = F.Context(N=8, n_interp=6, precision="fp64")
    fine = {}
    for L in (3, 4, 5):
        p, psi = config_vortex_ring(L, 8, 4, 0)
        for corr in (True, False):
            bs = F.BlockSet(c, [p.coords], [p.h0])
            if not corr:
                bs.set_option(F.OPT_CORRECTION, 0)
            for l, f in enumerate(p.f):
                bs.load_source(0, l, torch.as_tensor(f))
            bs.solve()
            leaf = p.leaf_masks()
            scale = max(np.max(np.abs(psi[l][leaf[l]])) for l in range(L))
            u = bs.potential(0, L - 1).double().cpu().numpy()[leaf[L - 1]]
            fine[(L, corr)] = np.max(np.abs(u - psi[L - 1][leaf[L - 1]])) / scale
            bs.close()
    print({k: f"{v:.3e}" for k, v in fine.items()})
    assert fine[(3, True)] / fine[(4, True)] > 3 and fine[(4, True)] / fine[(5, True)] > 3
    assert fine[(5, False)] > 1.1 * fine[(5, True)]
    c.close()
