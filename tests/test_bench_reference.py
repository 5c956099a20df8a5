"""The reference arm of bench.py (the FP64 CPU oracle timed on bounded samples of
the benchmark workload) runs without a GPU and prints one JSON line with the
keys the measurement contract needs."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "DoF/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["n_gpus"] == 1 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_traffic_summary_parses_and_keys_the_current_sources():
    """profiles/traffic.txt holds one entry per (kernel, workload) with the
    checksum of the sources it was captured on; bench.py reports the traffic
    only while that checksum matches (a stale entry reads as null, never as a
    wrong number)."""
    sys.path.insert(0, ROOT)
    import bench
    entries = []
    with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
            assert {"kernel", "src_sha", "workload", "dram_bytes_per_step"} <= set(kv), line
            assert len(kv["src_sha"]) == 16 and float(kv["dram_bytes_per_step"]) > 0
            entries.append(kv)
    assert any(e["kernel"] == "spectrum_mac" and e["workload"] == "batched64" for e in entries)
    got = bench.ncu_traffic("hadamard_fl.cu", "spectrum_mac", "batched64")
    csrc = os.path.join(ROOT, "paper_1911_10228_gb300", "csrc")
    sha = bench.files_sha([os.path.join(csrc, "hadamard_fl.cu"), os.path.join(csrc, "internal.h")])
    want = [float(e["dram_bytes_per_step"]) for e in entries if e["src_sha"] == sha and e["kernel"] == "spectrum_mac"]
    assert got == (want[0] if want else None)
