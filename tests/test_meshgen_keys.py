"""Host logic of the on-device refinement step: the library's Morton key and
its decoding (meshgen.cu, compiled with the library's own source and run on the
CPU) against the oracle's bit-by-bit definition (Sec. 4 orders octants by
Morton code; the bit order is fixed in the oracle's docstring)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.meshgen import morton_key

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc to compile the host code")
def test_library_keys_equal_the_oracle_definition(tmp_path):
    exe = tmp_path / "morton_check"
    src = os.path.join(ROOT, "tests", "cpp", "morton_check.cu")
    subprocess.run(["nvcc", "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-o", str(exe), src], check=True, capture_output=True,
                   timeout=600)
    rng = np.random.default_rng(2)
    pts = rng.integers(-(1 << 19) + 1, 1 << 19, size=(300, 3)).tolist()
    lim = (1 << 19) - 1
    pts += [[0, 0, 0], [-1, -1, -1], [lim, lim, lim], [-lim, -lim, -lim], [1, 0, 0], [0, 1, 0], [0, 0, 1],
            [2 * lim + 1, 0, -2 * lim]]   # a child coordinate of the largest level block
    stdin = "".join(f"{x} {y} {z}\n" for x, y, z in pts)
    out = subprocess.run([str(exe)], input=stdin, capture_output=True, text=True, timeout=60)
    assert out.returncode == 0
    rows = [ln.split() for ln in out.stdout.splitlines()]
    assert len(rows) == len(pts)
    for (x, y, z), (k, back) in zip(pts, rows):
        assert int(k) == morton_key(x, y, z), (x, y, z)
        assert back == "1", (x, y, z)
