"""Host logic of block-set compilation: the planner (octrees, interaction
tiles, dense parent groups, pair lists) runs on the CPU in a harness compiled
with the library's own source, and every interaction of every octree level must
appear exactly once in the spectrum-MAC launch lists, with the right kernel
offset, under every plan and both precisions (see tests/cpp/planner_check.cu)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1911_10228_gb300.inputs import box_coords, config_plain_32, random_sparse_problem, refine_mesh, torus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PLANS = [(0, (4, 4, 8)), (30, (4, 4, 8)), (100, (2, 4, 8)), (50, (4, 4, 4)), (30, (8, 4, 4))]
# FP32 MAC forms (FLGF_CTX_MAC): frequency-lane groups with frequency-lane pair lists (default, 1) or with
# the shared-memory pair lists (2), and the parent groups with the shared-memory pair lists (0)


def _write_mesh(path, N, problems):
    """problems: list over problems of lists over levels of (nb, 3) coordinates."""
    vals = [N, len(problems)] + [len(p) for p in problems] + [len(c) for p in problems for c in p]
    coords = np.concatenate([np.asarray(c, dtype=np.int32).reshape(-1, 3) for p in problems for c in p])
    with open(path, "wb") as f:
        f.write(np.asarray(vals, dtype=np.int32).tobytes())
        f.write(coords.astype(np.int32).tobytes())


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("nvcc") is None:
        pytest.skip("needs nvcc to compile the host code")
    from paper_1911_10228_gb300 import build as B
    B.build()                                   # the other translation units' objects
    exe = tmp_path_factory.mktemp("planner") / "planner_check"
    objs = [os.path.join(B.BUILD, n.replace(".cu", ".o")) for n in B.SOURCES if n != "flgf_api.cu"]
    subprocess.run(["nvcc", "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "cpp", "planner_check.cu")] + objs + ["-lpthread"],
                   check=True, capture_output=True, timeout=900)
    return exe


def _meshes():
    ring = refine_mesh(lambda x: torus(x, (0.5, 0.5, 0.5), 0.22, 0.05), box_coords(4), 8, 1.0 / 32, 3, 0.3)
    sparse = [random_sparse_problem(s, N=8, nblk_range=(8, 400)) for s in (1, 4, 7, 9, 12)]
    return {
        "plain": (8, [config_plain_32().coords]),
        "torus": (8, [ring.coords]),
        "batch": (8, [p.coords for p in sparse]),
    }


@pytest.mark.parametrize("fp64,mac", [(0, 1), (0, 2), (0, 0), (1, 0)],
                         ids=["fp32-lane", "fp32-lane-smemlists", "fp32-groups", "fp64"])
def test_every_interaction_once_in_the_launch_lists(harness, tmp_path, fp64, mac):
    for name, (N, problems) in _meshes().items():
        mesh = tmp_path / f"{name}.bin"
        _write_mesh(mesh, N, problems)
        for pct, tile in (PLANS[1:3] if mac >= 1 else PLANS):
            out = subprocess.run([str(harness), str(mesh), str(pct), *map(str, tile), str(fp64), str(mac)],
                                 capture_output=True, text=True, timeout=300)
            assert out.returncode == 0 and out.stdout.strip().endswith("ok"), (name, pct, tile, out.stdout)


def test_vector_groups_cover_every_component(harness, tmp_path):
    """A vector block set (three copies of one mesh): component 0's
    frequency-lane groups, shifted by the component stride, must cover the
    dense interactions of all three components exactly once."""
    for name, (N, problems) in _meshes().items():
        if name == "batch":
            continue
        mesh = tmp_path / f"{name}3.bin"
        _write_mesh(mesh, N, problems * 3)
        for pct, tile in PLANS[1:3]:
            out = subprocess.run([str(harness), str(mesh), str(pct), *map(str, tile), "0", "1", "3"],
                                 capture_output=True, text=True, timeout=300)
            assert out.returncode == 0 and out.stdout.strip().endswith("ok"), (name, pct, tile, out.stdout)
            dense = int(out.stdout.split("dense kernel ")[1].split(",")[0])
            assert dense > 0, out.stdout
