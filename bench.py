#!/usr/bin/env python
"""Benchmark of the FLGF Poisson solve (arXiv:1911.10228) on GB300.

Headline workload: the batched form -- 64 independent random sparse problems
of 16^3 blocks (block counts log-uniform in [8, 4096] over 1-3 refinement
levels, 1-4 Gaussians each, seeds 64 r .. 64 r + 63 on rank r) in one block
set, every stage of every problem in the same kernel launches, the solve
replayed as a CUDA graph.  One step = one full multi-resolution solve of the
batch (Sec. 3: coarsening, per level the FLGF of Sec. 2.1 -- anterpolation,
forward FFTs, spectrum multiply-accumulate, inverse FFTs, interpolation --
and the coarse-fine coupling) with the sources resident in HBM; L2 is flushed
(256 MB write) before every timed step.  The headline value is the FP32
form's DoF/s (leaf cells per second); the plain FP64 solve of the same batch
is timed beside it, and the FP32 error is stated against it and, on a sample
of problems, against the FP64 CPU oracle.

Further legs (keys of the JSON line): the 256^3 uniform lattice (16^3 blocks,
n_I = 6), the 3-level torus with the FP32 compensation off and on, the
adjoint solve on the linked tori, the three-component vortex ring as one
vector block set beside one scalar component, and the end-to-end batched solve
through the C ABI with host buffers.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (torchrun) every rank solves its own 64 problems (no exchange):
value = all ranks' DoF / slowest rank's time.  ``--impl reference`` times the
FP64 CPU oracle on bounded samples of the batched workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson DoF/s at stated rel err: FP32 batched vs FP64 plain; % HBM roofline"
BATCH_WORKLOAD = ("batched: 64 independent random sparse problems per GPU (seeds 64 r .. 64 r + 63 on rank r), "
                  "16^3 blocks, block counts log-uniform in [8, 4096] over 1-3 refinement levels, 1-4 Gaussians "
                  "each, n_I = 6, one block set, CUDA graph")
UNIFORM_WORKLOAD = ("uniform 256^3 lattice, 16^3 blocks of 16^3 cells, octree levels 0-2 + root, n_I=6, "
                    "16 Gaussians sigma 3-10 cells in the inner 128^3, seed 0")
FP32_LANES = 128          # FP32 FMA lanes per SM
FP64_NOMINAL_TFLOPS = 1.25
FALLBACK_HBM_GBS = 6800.0
FALLBACK_SM_MHZ = 2070.0


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--problems", type=int, default=64, help="problems of the batched workload per GPU")
    ap.add_argument("--legs", default="batched,uniform,multires,adjoint,vector,meshgen",
                    help="legs to run; the batched leg (the headline) always runs")
    ap.add_argument("--precisions", default="fp32,fp64", help="contexts to time (profiling runs use fp32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle budget of the cpu_baseline sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the batched solve's kernels one by one instead of replaying its CUDA graph "
                         "(profiling runs: ncu's replay of the graph's kernel nodes failed to launch the MAC)")
    ap.add_argument("--plan", default=None,
                    help="fixed MAC plan for the batched leg, e.g. 30/4x4x4 (list percentage / tile); default: autotune")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBs", "hbm"):
            if key in d:
                return float(d[key]), "measured", float(d.get("sm_max_mhz", FALLBACK_SM_MHZ))
    return FALLBACK_HBM_GBS, "fallback", FALLBACK_SM_MHZ


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while a timed
    region runs; samples accumulate over several regions (start/stop)."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines += [l for l in out.splitlines() if l.strip()]
        self.proc = None

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def files_sha(paths):
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_src: str, kernel: str, workload: str):
    """DRAM bytes per step (all launches of one solve) of a kernel from the
    committed ncu summary, if it was taken on the current kernel source and
    the launch constants of internal.h (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    csrc = os.path.join(ROOT, "paper_1911_10228_gb300", "csrc")
    sha = files_sha([os.path.join(csrc, kernel_src), os.path.join(csrc, "internal.h")])
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
            if kv.get("kernel") == kernel and kv.get("src_sha") == sha and kv.get("workload") == workload:
                return float(kv["dram_bytes_per_step"])
    return None


def leaf_linf(outs_a, outs_b, probs):
    """max over problems and leaf cells of |a - b|, over max |b| (per problem)."""
    import torch
    worst = 0.0
    for ua, ub, p in zip(outs_a, outs_b, probs):
        num, den = 0.0, 0.0
        for xa, xb, lm in zip(ua, ub, p.leaf_masks()):
            if not lm.any():
                continue
            m = torch.as_tensor(lm, device=xb.device)
            num = max(num, float((xa.double() - xb.double())[m].abs().max()))
            den = max(den, float(xb.double()[m].abs().max()))
        worst = max(worst, num / den if den > 0 else 0.0)
    return worst


def oracle_batch_sample(probs, budget_s: float):
    """FP64 oracle (multi-resolution solve) on the smallest problems of the
    batch, in order of size, until the budget is used; returns
    [(index, u levels, leaf masks)], seconds, DoF."""
    from oracle.lgf import LGF
    from oracle.multires import multires_solve
    G = LGF()
    order = sorted(range(len(probs)), key=lambda i: sum(len(c) for c in probs[i].coords))
    out, t_used, dof = [], 0.0, 0
    for i in order:
        p = probs[i]
        t = time.perf_counter()
        u, leaf = multires_solve(G, p.coords, p.f, p.N, 6, p.h0)
        t_used += time.perf_counter() - t
        out.append((i, u, leaf))
        dof += p.dof()
        if t_used >= budget_s:
            break
    return out, t_used, dof


def run_reference(a, rank, world):
    """The oracle arm: the FP64 CPU oracle on bounded samples of the batched workload."""
    if rank != 0:
        return
    from oracle.lgf import LGF
    from oracle.multires import multires_solve
    from paper_1911_10228_gb300.inputs import config_batched
    probs = config_batched(a.problems)
    order = sorted(range(len(probs)), key=lambda i: sum(len(c) for c in probs[i].coords))
    G = LGF()
    times, dofs = [], []
    for s in range(a.warmup + a.steps):
        p = probs[order[s % 2]]           # the two smallest problems in turn, so the run stays within minutes
        t = time.perf_counter()
        multires_solve(G, p.coords, p.f, p.N, 6, p.h0)
        if s >= a.warmup:
            times.append(time.perf_counter() - t)
            dofs.append(p.dof())
    value = float(np.sum(dofs) / np.sum(times))
    ms = 1e3 * float(np.mean(times))
    sample = (f"one of the 2 smallest of the {len(probs)} problems per step, in turn (full multi-resolution "
              f"solve), {np.mean(dofs):.0f} DoF per step on average")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "problems": len(probs), "parallelism": "oracle on host cores"},
        "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(a, rank, world):
    import torch

    from paper_1911_10228_gb300 import flgf as F
    from paper_1911_10228_gb300 import multirank as MR
    from paper_1911_10228_gb300.inputs import config_batched

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    hbm, hbm_src, sm_mhz_peak = peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(dev)
    legs = set(x for x in a.legs.split(",") if x)
    precs = [p for p in a.precisions.split(",") if p]
    if "fp32" not in precs:
        raise SystemExit("the headline value is the FP32 form: --precisions must include fp32")

    def timed(stream, fn, n):
        """ms per call of fn over n calls (CUDA events on the library stream,
        L2 flushed before each), max over ranks."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        MR.barrier("cuda")
        torch.cuda.synchronize()
        sampler.start()
        for s0, s1 in ev:
            with torch.cuda.stream(stream):
                flush.zero_()
            s0.record(stream)
            fn()
            s1.record(stream)
        torch.cuda.synchronize()
        sampler.stop()
        MR.barrier("cuda")
        return MR.all_max(float(np.mean([s0.elapsed_time(s1) for s0, s1 in ev])), "cuda")

    def fp32_alu_peak():
        return n_sm * FP32_LANES * 2 * sm_mhz_peak * 1e6 / 1e12

    torch.cuda.nvtx.range_push("batched")  # one NVTX range per leg (profilers select a leg by it)
    # ------------------------------------------------------------------ batched
    seeds = MR.problem_seeds(a.problems, rank)
    probs = config_batched(a.problems, first_seed=seeds[0])
    bdof_rank = sum(p.dof() for p in probs)
    bdof = MR.all_sum(bdof_rank, "cuda")
    batched = {"problems": len(probs), "blocks_rank0": int(sum(len(c) for p in probs for c in p.coords)),
               "dof": int(bdof), "dof_rank0": int(bdof_rank)}
    plan = None
    if a.plan:
        pct, tile = a.plan.split("/")
        plan = (int(pct), tuple(int(v) for v in tile.split("x")))
        batched["plan"] = {"list_pct": plan[0], "tile": list(plan[1]), "source": "--plan"}
    outs, res = {}, {}
    for prec in precs:
        bctx = F.Context(N=16, n_interp=6, precision=prec)
        if plan is None:
            from paper_1911_10228_gb300.autotune import autotune
            t0 = time.time()
            plan, table = autotune(bctx, [p.coords for p in probs], [p.h0 for p in probs], reps=2)
            batched["plan"] = {"list_pct": plan[0], "tile": list(plan[1]), "source": "autotune",
                               "seconds": round(time.time() - t0, 1),
                               "ms_per_solve": {f"{k[0]}/{'x'.join(map(str, k[1]))}": round(v, 2)
                                                for k, v in table.items()}}
        bctx.set_plan(list_pct=plan[0], tile=plan[1])
        t_create = time.time()
        bbs = F.BlockSet(bctx, [p.coords for p in probs], [p.h0 for p in probs])
        torch.cuda.synchronize()
        t_create = time.time() - t_create   # host planner (octrees, lists, groups) and device allocation
        for i, p in enumerate(probs):
            for l, f in enumerate(p.f):
                bbs.load_source(i, l, torch.as_tensor(f))
        bbs.set_option(F.OPT_GRAPH, 0 if a.no_graph else 1)
        bbs.set_option(F.OPT_TIMING, 1)    # stage events inside the captured graph
        # the FP64 batched solve takes seconds: one warm-up and one step (it also serves the error check)
        for _ in range(max(1, a.warmup) if prec == "fp32" else 1):
            bbs.solve()
        torch.cuda.synchronize()
        bbs.stage_times(reset=True)
        nb = a.steps if prec == "fp32" else 1
        ms = timed(bctx.stream, bbs.solve, nb)
        stage, n_timed = bbs.stage_times(reset=True)
        res[prec] = {"value": bdof / (ms / 1e3), "unit": "DoF/s", "ms_per_step": ms, "steps": nb,
                     "blockset_create_s": t_create,
                     "launches_per_step": bbs.launch_count(),
                     "stages_ms": {k: v / max(n_timed, 1) for k, v in stage.items()},
                     "work": bbs.work_counts()}
        outs[prec] = [[bbs.potential(i, l) for l in range(p.n_levels)] for i, p in enumerate(probs)]
        if prec == "fp32":
            keep_ctx, keep_bs = bctx, bbs
        else:
            bbs.close()
            bctx.close()
    if "fp64" in outs:
        batched["fp32_vs_fp64_linf"] = leaf_linf(outs["fp32"], outs["fp64"], probs)
    N = 16
    NW = 2 * N * 2 * N * (N + 1)
    r32 = res["fp32"]
    mac_ms = r32["stages_ms"]["spectrum_mac"]
    mac_flops = r32["work"]["pairs"] * NW * 8.0
    mac_tflops = mac_flops / (mac_ms / 1e3) / 1e12 if mac_ms > 0 else None
    batched["fp32"] = {k: v for k, v in r32.items() if k != "work"}
    batched["fp32"]["pairs"] = r32["work"]["pairs"]
    if "fp64" in res:
        r64 = res["fp64"]
        batched["fp64"] = {k: v for k, v in r64.items() if k != "work"}
        batched["fp32_over_fp64"] = r32["value"] / r64["value"]

    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("uniform")  # one NVTX range per leg (profilers select a leg by it)
    # ------------------------------------------------------------------ uniform 256^3
    uniform = None
    if "uniform" in legs:
        from paper_1911_10228_gb300.inputs import config_uniform_256
        up = config_uniform_256()
        udof = up.dof()
        f64 = torch.as_tensor(up.f[0])
        uniform = {"workload": UNIFORM_WORKLOAD, "dof": udof}
        for prec in precs:
            ctx = F.Context(N=16, n_interp=6, precision=prec)
            bs = F.BlockSet(ctx, [up.coords], [up.h0])
            bs.load_source(0, 0, f64.to("cuda"))
            bs.set_option(F.OPT_TIMING, 1)
            for _ in range(a.warmup):
                bs.solve()
            torch.cuda.synchronize()
            bs.stage_times(reset=True)
            n = a.steps if prec == "fp32" else max(3, min(a.steps, 10))
            ms = timed(ctx.stream, bs.solve, n)
            stage, nt = bs.stage_times(reset=True)
            st = {k: v / max(nt, 1) for k, v in stage.items()}
            w = bs.work_counts()
            rs = 4 if prec == "fp32" else 8
            flops = w["pairs"] * NW * 8.0
            row = {"value": udof * world / (ms / 1e3), "unit": "DoF/s", "ms_per_step": ms, "steps": n,
                   "stages_ms": st, "launches_per_step": bs.launch_count(),
                   "spectrum_mac_tflops": flops / (st["spectrum_mac"] / 1e3) / 1e12,
                   "fft_forward_gbs": w["fwd_ffts"] * (N ** 3 * rs + NW * 2 * rs) / (st["fft_forward"] / 1e3) / 1e9,
                   "fft_inverse_gbs": w["inv_ffts"] * (N ** 3 * rs + NW * 2 * rs) / (st["fft_inverse"] / 1e3) / 1e9}
            if prec == "fp32":
                row["spectrum_mac_frac_of_fp32_fma"] = row["spectrum_mac_tflops"] / fp32_alu_peak()
                row["fft_forward_frac_of_hbm"] = row["fft_forward_gbs"] / hbm
                row["fft_inverse_frac_of_hbm"] = row["fft_inverse_gbs"] / hbm
            else:
                row["spectrum_mac_frac_of_fp64_nominal"] = row["spectrum_mac_tflops"] / FP64_NOMINAL_TFLOPS
            uniform[prec] = row
            uniform.setdefault("_u", {})[prec] = bs.potential(0, 0).double().cpu().numpy()
            bs.close()
            ctx.close()

    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("meshgen")  # one NVTX range per leg (profilers select a leg by it)
    # ------------------------------------------------------------------ on-device refinement step
    meshgen = None
    if "meshgen" in legs:
        from paper_1911_10228_gb300.inputs import config_uniform_256
        mp = config_uniform_256()
        mctx = F.Context(N=16, n_interp=6, precision="fp32")
        mf = torch.as_tensor(mp.f[0]).to("cuda", torch.float32)
        mc = torch.as_tensor(mp.coords[0], dtype=torch.int32).cuda()
        flags, ch, buf = mctx.refine_level(mf, mc, 1e-3)   # warm-up
        torch.cuda.synchronize()
        reps = 5
        t0 = time.time()
        for _ in range(reps):
            flags, ch, buf = mctx.refine_level(mf, mc, 1e-3)
        torch.cuda.synchronize()
        meshgen = {"workload": "refinement step (Eq. ref_crit, rel 1e-3) of the 256^3 lattice's 4096 blocks of 16^3: "
                               "flags, Morton-sorted children and 26-neighbour buffer on the device",
                   "ms_per_call": (time.time() - t0) / reps * 1e3, "refined": int(flags.sum()),
                   "children": int(ch.shape[0]), "buffer": int(buf.shape[0]),
                   "note": "wall clock: the call synchronises (it returns the list lengths to the host)"}
        mctx.close()
    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("multires")  # one NVTX range per leg (profilers select a leg by it)
    # ------------------------------------------------------------------ refined torus
    multires = None
    if "multires" in legs:
        from paper_1911_10228_gb300.inputs import config_torus_128
        tp = config_torus_128()
        tdof = tp.dof()
        multires = {"workload": "Gaussian-core torus (R 0.25, sigma 0.03), base 128^3 in 8^3 blocks of 16^3, 3 levels "
                                "refined where |f| > 1e-3 max, n_I=6, source correction on, CUDA graph",
                    "dof": tdof, "blocks": int(sum(len(c) for c in tp.coords))}
        touts = {}
        for prec, comp in ([("fp32", 1), ("fp32", 0)] + ([("fp64", 0)] if "fp64" in precs else [])):
            mctx = F.Context(N=16, n_interp=6, precision=prec)
            mbs = F.BlockSet(mctx, [tp.coords], [tp.h0])
            if prec == "fp32":
                mbs.set_option(F.OPT_COMPENSATED, comp)
            for l, f in enumerate(tp.f):
                mbs.load_source(0, l, torch.as_tensor(f))
            mbs.set_option(F.OPT_GRAPH, 1)
            for _ in range(max(1, a.warmup)):
                mbs.solve()
            n = a.steps if prec == "fp32" else 2
            ms = timed(mctx.stream, mbs.solve, n)
            key = prec if prec == "fp64" else ("fp32" if comp else "fp32_uncompensated")
            multires[key] = {"value": tdof * world / (ms / 1e3), "unit": "DoF/s", "ms_per_step": ms, "steps": n,
                             "launches_per_step": mbs.launch_count()}
            touts[key] = [mbs.potential(0, l) for l in range(tp.n_levels)]
            mbs.close()
            mctx.close()
        if "fp64" in touts:
            multires["fp32_vs_fp64_linf"] = leaf_linf([touts["fp32"]], [touts["fp64"]], [tp])
            multires["fp32_uncompensated_vs_fp64_linf"] = leaf_linf([touts["fp32_uncompensated"]], [touts["fp64"]],
                                                                    [tp])
        del touts

    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("adjoint")  # one NVTX range per leg (profilers select a leg by it)
    # ------------------------------------------------------------------ adjoint
    adjoint = None
    if "adjoint" in legs:
        from paper_1911_10228_gb300.inputs import config_linked_tori
        lt = config_linked_tori()
        ldof = lt.dof()
        actx = F.Context(N=16, n_interp=6, precision="fp32")
        abs_ = F.BlockSet(actx, [lt.coords], [lt.h0])
        rng = np.random.default_rng(0)
        for l, f in enumerate(lt.f):
            abs_.load_source(0, l, torch.as_tensor(f))
            abs_.load_adjoint(0, l, torch.as_tensor(rng.standard_normal(f.shape).astype(np.float32)))
        abs_.solve()
        for _ in range(max(1, a.warmup)):
            abs_.solve_adjoint()
        n = min(a.steps, 10)
        ms = timed(actx.stream, abs_.solve_adjoint, n)
        adjoint = {"workload": "linked Gaussian tori (R 0.2, sigma 0.03), base 128^3 in 8^3 blocks of 16^3, 3 levels "
                               "(512^3-equivalent finest level), FP32, source correction on: A^T g for random seeds",
                   "dof": ldof, "value": ldof * world / (ms / 1e3), "unit": "DoF/s (gradient)", "ms_per_step": ms,
                   "steps": n, "launches_per_step": abs_.launch_count()}
        abs_.close()
        actx.close()

    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("vector")  # one NVTX range per leg (profilers select a leg by it)
    # ------------------------------------------------------------------ vector (three components, one mesh)
    vector = None
    if "vector" in legs:
        from paper_1911_10228_gb300.inputs import cell_centres, config_vortex_ring, vortex_ring_vector
        vp, _ = config_vortex_ring(3, 16, 8)
        comps = [[], [], []]
        for l, c in enumerate(vp.coords):
            _, w = vortex_ring_vector(cell_centres(c, 16, vp.h0 / (1 << l)))
            for k in range(3):
                comps[k].append(torch.as_tensor(np.ascontiguousarray(w[..., k]).astype(np.float32)))
        vector = {"workload": "vortex ring (Sec. 3.1: c1 1e3, c2 10, R 0.125), base 128^3 in 8^3 blocks of 16^3, "
                              "3 levels, the three vorticity components as one vector block set, FP32, CUDA graph",
                  "dof_per_component": vp.dof(), "blocks": int(sum(len(c) for c in vp.coords))}
        vctx = F.Context(N=16, n_interp=6, precision="fp32")
        for key, nc in (("vector3", 3), ("scalar1", 1)):
            vbs = F.BlockSet(vctx, [vp.coords] * nc, [vp.h0] * nc, vector=nc > 1)
            for k in range(nc):
                for l in range(vp.n_levels):
                    vbs.load_source(k, l, comps[k][l])
            vbs.set_option(F.OPT_GRAPH, 1)
            vbs.set_option(F.OPT_TIMING, 1)
            for _ in range(max(1, a.warmup)):
                vbs.solve()
            torch.cuda.synchronize()
            vbs.stage_times(reset=True)
            n = min(a.steps, 10)
            ms = timed(vctx.stream, vbs.solve, n)
            stage, nt = vbs.stage_times(reset=True)
            vector[key] = {"ms_per_step": ms, "steps": n, "spectrum_mac_ms": stage["spectrum_mac"] / max(nt, 1),
                           "value": nc * vp.dof() * world / (ms / 1e3), "unit": "DoF/s (all components)"}
            vbs.close()
        vctx.close()
        vector["mac_ms_over_3_scalar"] = vector["vector3"]["spectrum_mac_ms"] / (3 * vector["scalar1"]["spectrum_mac_ms"])
        vector["solve_ms_over_3_scalar"] = vector["vector3"]["ms_per_step"] / (3 * vector["scalar1"]["ms_per_step"])

    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("e2e")  # one NVTX range per leg (profilers select a leg by it)
    # ------------------------------------------------------------------ end to end (batched, host buffers)
    e2e = None
    if not a.no_e2e:
        keys = [(i, l) for i, p in enumerate(probs) for l in range(p.n_levels)]
        h_src = {k: torch.empty(tuple(probs[k[0]].f[k[1]].shape), dtype=torch.float32, pin_memory=True) for k in keys}
        for (i, l), t in h_src.items():
            t.copy_(torch.as_tensor(probs[i].f[l]).float())
        h_out = {k: torch.empty_like(t, pin_memory=True) for k, t in h_src.items()}
        nbytes = sum(t.numel() * 4 for t in h_src.values())

        # As a time-stepping caller runs it: the next step's sources are loaded
        # (host to device, on the library's copy stream) while the current solve
        # runs, then the current potentials are read back and the next solve is
        # enqueued.  Every step moves all inputs in and all results out.
        def load_all():
            for (i, l), t in h_src.items():
                keep_bs.load_source(i, l, t)

        def read_all():
            for (i, l), t in h_out.items():
                keep_bs.potential_host(i, l, out=t.numpy())

        def e2e_run(n):
            load_all()
            keep_bs.solve()
            for s in range(n):
                if s + 1 < n:
                    load_all()
                read_all()
                if s + 1 < n:
                    keep_bs.solve()

        keep_bs.set_option(F.OPT_TIMING, 0)
        e2e_run(max(1, a.warmup))
        MR.barrier("cuda")
        t = time.perf_counter()
        e2e_run(a.steps)
        e2e_ms = MR.all_max(1e3 * (time.perf_counter() - t), "cuda") / a.steps
        e2e = {"value": bdof / (e2e_ms / 1e3), "unit": "DoF/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms,
               "note": "pinned host buffers through the C ABI (flgf_load_source / flgf_get_potential with host "
                       "pointers); the next step's loads overlap the current solve"}

    torch.cuda.nvtx.range_pop()
    # ------------------------------------------------------------------ CPU oracle baseline and errors
    cpu, err = None, None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        sample, secs, sdof = oracle_batch_sample(probs, a.cpu_seconds)
        err = {"sample": f"{len(sample)} smallest of the {len(probs)} problems, FP64 oracle (full multi-resolution "
                         f"solve), leaf cells"}
        for prec in outs:
            worst = 0.0
            for i, u, leaf in sample:
                scale = max(np.max(np.abs(x[m])) for x, m in zip(u, leaf) if m.any())
                for l in range(probs[i].n_levels):
                    if leaf[l].any():
                        g = outs[prec][i][l].double().cpu().numpy()
                        worst = max(worst, float(np.max(np.abs(g[leaf[l]] - u[l][leaf[l]])) / scale))
            err[prec + "_vs_oracle_linf"] = worst
        cpu = {"value": sdof / secs, "unit": "DoF/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(sample)} smallest of the {len(probs)} problems of the batched workload "
                         f"({sdof} DoF), full multi-resolution solve, {secs:.1f} s"}
        if uniform is not None:
            # the 256^3 leg against the oracle on 8 sampled target blocks
            from oracle.flgf import FLGF
            from oracle.lgf import LGF
            from paper_1911_10228_gb300.inputs import config_uniform_256
            up = config_uniform_256()
            op = FLGF(LGF(), up.coords[0], up.N, 6)
            nz = np.nonzero(np.any(up.f[0] != 0, axis=(1, 2, 3)))[0]
            tg = np.sort(np.random.default_rng(0).choice(nz, 8, replace=False))
            ref = op.apply(up.f[0], h=up.h0, targets=tg)[tg]
            for prec, u in uniform["_u"].items():
                d = u[tg] - ref
                uniform[prec]["vs_oracle_linf"] = float(np.max(np.abs(d)) / np.max(np.abs(ref)))
                uniform[prec]["vs_oracle_l2"] = float(np.linalg.norm(d) / np.linalg.norm(ref))
            uniform["oracle_sample"] = "8 of 4096 target blocks (seeded), FP64 oracle"
    if uniform is not None:
        uniform.pop("_u", None)

    peak = fp32_alu_peak()
    line = {
        "metric": METRIC,
        "value": r32["value"],
        "unit": "DoF/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": r32["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "problems": len(probs), "N": 16, "n_interp": 6,
                   "dof": int(bdof), "l2": "flushed before every timed step (256 MB write)",
                   "compensated_coarse_levels": True, "cuda_graph": not a.no_graph,
                   "parallelism": "independent problems per rank" if world > 1 else "single GPU"},
        "rel_err": {"fp32_vs_fp64_linf": batched.get("fp32_vs_fp64_linf"), **(err or {})},
        "roofline": {"bound": "alu", "kernel": "spectrum MAC (hadamard_fl_kernel + hadamard_fll_kernel), "
                                               "all launches of one batched solve",
                     "achieved": mac_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": (mac_tflops / peak) if mac_tflops else None,
                     "traffic": ncu_traffic("hadamard_fl.cu", "spectrum_mac", f"batched{a.problems}"),
                     "peak_note": f"FP32 FMA: {n_sm} SMs x {FP32_LANES} lanes x 2 flop x {sm_mhz_peak:.0f} MHz",
                     "flops_per_step": mac_flops,
                     "flops_note": "useful (target, source) block pairs x 2N*2N*(N+1) frequencies x 8 flop"},
        "hbm": {"peak_gbs": hbm, "peak_source": hbm_src},
        "batched": batched,
        "uniform256": uniform,
        "multires": multires,
        "adjoint": adjoint,
        "vector": vector,
        "meshgen": meshgen,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": r32["launches_per_step"] * a.steps,
        "clocks": sampler.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    keep_bs.close()
    keep_ctx.close()


def main():
    a = args_parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = world > 1
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if dist:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    run_ours(a, rank, world)
    if dist:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
