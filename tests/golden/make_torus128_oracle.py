"""Write torus128_oracle.txt: FP64 oracle values of the 3-level torus workload
(base 128^3 in 8^3 blocks of 16^3 cells, Gaussian-core torus R = 0.25,
sigma = 0.03, refined where |f| > 1e-3 max, n_I = 6, source correction on;
Sec. 3) at sampled cells of sampled leaf blocks of every level.

Calls only the oracle (oracle/multires.py) and the input recipe; the result
is a fixed expected value for tests/test_gpu_fullsize.py.  Samples: on each
level, 12 leaf blocks (seeded choice, the block holding the level's largest
|u| among them), and in each block its 8 corner cells, the centre cell and 7
seeded cells -- the corners are where the downward-pass extrapolation makes
FP32 rounding largest.  Also written: the largest |u| over all leaf cells
(the normalisation of the relative error).  Takes several minutes of CPU.

    python tests/golden/make_torus128_oracle.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.lgf import LGF  # noqa: E402
from oracle.multires import multires_solve  # noqa: E402
from paper_1911_10228_gb300.inputs import config_torus_128  # noqa: E402


def main(out=os.path.join(HERE, "torus128_oracle.txt")):
    p = config_torus_128()
    u, leaf = multires_solve(LGF(), p.coords, p.f, p.N, 6, p.h0)
    umax = max(float(np.max(np.abs(x[m]))) for x, m in zip(u, leaf))
    rng = np.random.default_rng(2024)
    N = p.N
    corners = [(i, j, k) for i in (0, N - 1) for j in (0, N - 1) for k in (0, N - 1)]
    lines = [f"# FP64 oracle u at sampled cells of the 3-level torus workload (written by {os.path.basename(__file__)})",
             f"umax {umax:.17e}",
             "# level block i j k u"]
    for l in range(p.n_levels):
        leaves = np.nonzero(leaf[l])[0]
        pick = list(rng.choice(leaves, size=min(11, leaves.size), replace=False))
        pick.append(int(leaves[np.argmax([np.max(np.abs(u[l][b])) for b in leaves])]))
        for b in sorted(set(int(v) for v in pick)):
            cells = corners + [(N // 2, N // 2, N // 2)] + [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(7)]
            for (i, j, k) in cells:
                lines.append(f"{l} {b} {i} {j} {k} {u[l][b, i, j, k]:.17e}")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {out}: {len(lines) - 3} samples, umax {umax:.6e}")


if __name__ == "__main__":
    main()
