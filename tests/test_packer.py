"""Host logic of the dense spectrum MAC: the parent-group packer, compiled with
the library's own source and run on the CPU (no GPU call)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc to compile the host code")
def test_parent_group_packer(tmp_path):
    exe = tmp_path / "packer_check"
    src = os.path.join(ROOT, "tests", "cpp", "packer_check.cu")
    lib_src = os.path.join(ROOT, "paper_1911_10228_gb300", "csrc", "hadamard.cu")
    subprocess.run(["nvcc", "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", str(exe), src, lib_src], check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout
