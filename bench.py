#!/usr/bin/env python
"""Benchmark: continuous max-flow segmentation on GB300.

Headline workload: the 16-label Potts model on a 4096 x 4096 image (Voronoi
partition of 512 seeds, 16 grey levels i/15, noise sigma 0.05), costs
C_i = (I - c_i)^2, edge-weighted alpha(x) = 0.3 exp(-10 |grad I|).  One step =
one solve from a cold start to a relative primal-dual gap <= 1e-4
(certificates every 50 iterations) with the fused rpADMMII solver in two
phases: flows q_i and p_i stored as float16 until the certified gap stalls
(the first phase's stall test, with the switch gap 1.5e-4 just above the
target: near 6e-4 on this workload), then float32 (16-bit rounding of q_i and
p_i holds this workload's gap near 3e-4); p_s, u and the arithmetic are
float32, the certificates double-float / FP64.

Metric: pixel*label*iterations per second, plus the time to the 1e-4 gap
(fused vs the plain one-kernel-per-step form, float16 vs float32 flows).  The
inputs and state (several GB) are far larger than the 129 MB L2.

Side measurements on the same JSON line: the binary 1024^2 workload (its
state stays in L2: bound "l2"), the 4-label 2048^2 workload in float32,
float16 and bfloat16 storage, the 256-instance batch, the FP64 oracle's error
against the GPU results, and the oracle's own speed on one host core and on
all of them.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own instance (seed 5 + rank): weak
scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 4096
L = 16
TOL = 1e-4
FLAGSHIP = 2          # rpADMMII
STORAGE = 0           # the caller's state buffers: float32
PHASE_STORAGE = 1     # first phase in float16 flows (q_i, p_i), inside the workspace
PHASE_GAP = 1.5e-4    # switch gap just above the target: the stall test decides
                      # (measured at c = 0.3: 4.28 s against 4.57 s switching at 2e-3)
TUNE_PHASE_GAP = 2e-3 # the autotuned leg's base switch (it also tries the stall test
                      # alone; at c = 1.2 switching at 2e-3 is faster)
COSTS = 0             # cost planes as given (float32)
CHECK_EVERY = 50      # a 16-label certificate launch costs about 1.7 iterations
CHECK_SIDE = 10       # the side workloads check every 10 iterations
BATCH_CHECK = 20      # the batch (and its one-by-one comparison) every 20: its tile
                      # certificates cost about an iteration of all instances
MAX_ITER = 12000
# Algorithmic bytes of one iteration of this workload counted with every
# stored field in 16 bits: L (8 s + s_c) + 2 s + 4 with s = s_c = 2 (u, q_i,
# p_i and p_s read and written once, the costs and the alpha field read once):
# 296 B per pixel.  The solver keeps u and p_s in float32 and reads float32
# cost planes (design_bytes_per_px below).
BYTES_PER_PX_16BIT = 296
WORKLOAD = ("potts L=16 4096x4096 Voronoi (512 seeds), edge-weighted alpha, float16 flows "
            "until their gap stalls then float32, solve to gap 1e-4")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def job_totals(step_ms, iters, world: int, device):
    """Whole-job figures from one rank's timed steps: the slowest rank's total
    time (max over ranks) and the units all ranks processed (H*W*L pixel-labels
    per iteration, summed over ranks).  Replicas: each rank solves its own
    instance, so the only communication is this reduction of two scalars."""
    import torch

    total_ms = float(np.sum(step_ms))
    units = H * W * L * float(np.sum(iters))
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(u)
        total_ms, units = float(t.item()), float(u.item())
    return total_ms, units


def job_max_ms(step_ms, world: int, device) -> float:
    """The slowest rank's total of step_ms (max over ranks)."""
    return job_totals(step_ms, [0], world, device)[0]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[2 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _traffic(kernel_src: str, kernel_name: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[kernel_name]
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()
        if ent.get("src_sha256") != sha:
            return None
        return float(ent["dram_bytes_per_launch_full_size"])
    except (OSError, KeyError, ValueError):
        return None


def phase_one_end(hist, phase_gap: float, check_every: int) -> int:
    """Row of a two-phase solve's history at which its float16 phase ended:
    the first check whose gap is <= phase_gap or, tested every
    ceil(200 / check_every) checks from the first, whose gap is below
    10 phase_gap and above 0.7 times the gap at the previous tested check
    (cmf_solve_potts's switch rule, recomputed from the rows)."""
    w = -(-200 // check_every)
    ref = None
    for n in range(len(hist)):
        g = hist[n, 3]
        if g <= phase_gap:
            return n
        if n % w == 0:
            if n > 0 and g < 10 * phase_gap and g > 0.7 * ref:
                return n
            ref = g
    return len(hist) - 1


def rank_instance(rank: int, n: int = H):
    """The headline instance of one rank: replicas solve their own seeds."""
    from paper_2004_11227_gb300 import synth

    return synth.config5(n, n, seed=5 + rank)


def algorithmic_bytes_per_px(model: str, L: int, storage: int, alpha_field: bool,
                             costs: str = "f32") -> int:
    """State read and written once, costs and alpha read once (halos and
    recomputed values excluded).  Binary: u float32, four flow planes in the
    storage type.  Potts: u float32, q_i and p_i in the storage type, p_s
    float32; costs "f32" or "f16" planes, or "levels" (one float32 image
    plane)."""
    s = 4 if storage == 0 else 2
    al = 4 if alpha_field else 0
    if model == "binary":
        return 4 * 2 + 4 * s * 2 + 8 + al
    c = {"f32": 4 * L, "f16": 2 * L, "levels": 4}[costs]
    return L * (4 * 2 + 3 * s * 2) + c + 4 * 2 + al


def _timed(fn, reps=1):
    """Median CUDA-event time of fn() over reps calls (ms) and its last result."""
    import torch

    ts, out = [], None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), out


def oracle_rate(inst, algo: int, n_iter: int, threads: int):
    """The FP64 oracle on a bounded sample: n_iter iterations of `algo` from a
    cold start on the whole instance with `threads` host threads (0: all).
    Returns (pixel*label*iterations/s, seconds, threads used)."""
    import oracle

    oracle.build()
    used = oracle.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    p = oracle.default_params(algo, inst.L)
    alpha = inst.alpha if np.isscalar(inst.alpha) else inst.alpha.astype(np.float64)
    if inst.kind == "binary":
        cs, ct = (inst.costs[i].astype(np.float64) for i in range(2))
        t0 = time.perf_counter()
        oracle.binary_run(cs, ct, alpha, p, n_iter)
    else:
        c = inst.costs.astype(np.float64)
        t0 = time.perf_counter()
        oracle.potts_run(c, alpha, p, n_iter)
    dt = time.perf_counter() - t0
    return inst.H * inst.W * inst.L * n_iter / dt, dt, used


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the paper ships no code) on the
    headline workload, rank 0 only, all host cores, each step a bounded sample
    of one rpADMMII iteration of the whole 4096^2 x 16 instance."""
    ws, rank = _dist()
    if rank != 0:
        return
    inst = rank_instance(0)
    oracle_rate(inst, FLAGSHIP, 1, 0)  # build, page in
    for _ in range(args.warmup):
        oracle_rate(inst, FLAGSHIP, 1, 0)
    rates, times, used = [], [], 1
    for _ in range(args.steps):
        r, dt, used = oracle_rate(inst, FLAGSHIP, 1, 0)
        rates.append(r)
        times.append(dt)
    value = float(np.mean(rates))
    sample = (f"1 rpADMMII iteration of the full 4096x4096x16 workload per step, FP64 C "
              f"oracle, {used} threads")
    line = {
        "impl": "reference", "metric": "pixel*label*iterations/s", "value": value,
        "unit": "px*label*it/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "H": H, "W": W, "L": L,
                                        "algo": "rpADMMII"},
        "cpu_baseline": {"value": value, "unit": "px*label*it/s", "cores": used,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "px*label*it/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


KERNEL_CASES = {
    # name: (model, algo, H, W, L, storage, impl)
    "binary-admm-1024": ("binary", 2, 1024, 1024, 2, 0, 0),
    "binary-admm-4096": ("binary", 2, 4096, 4096, 2, 0, 0),
    "binary-dr-4096": ("binary", 3, 4096, 4096, 2, 0, 0),
    "binary-dr-1024": ("binary", 3, 1024, 1024, 2, 0, 0),
    "binary-dr-plain-1024": ("binary", 3, 1024, 1024, 2, 0, 1),
    "binary-cp-1024": ("binary", 5, 1024, 1024, 2, 0, 0),
    "potts4-dr-plain-2048": ("potts", 3, 2048, 2048, 4, 0, 1),
    "binary-plain-4096": ("binary", 2, 4096, 4096, 2, 0, 1),
    "potts4-admm-2048": ("potts", 2, 2048, 2048, 4, 0, 0),
    "potts4-admm-2048-f16": ("potts", 2, 2048, 2048, 4, 1, 0),
    "potts4-dr-2048": ("potts", 3, 2048, 2048, 4, 0, 0),
    "potts4-dr-2048-f16": ("potts", 3, 2048, 2048, 4, 1, 0),
    "potts16-admm-2048-f16": ("potts", 2, 2048, 2048, 16, 1, 0),
    "potts16-admm-4096-f16": ("potts", 2, 4096, 4096, 16, 1, 0),
    "potts16-admm-2048-f32": ("potts", 2, 2048, 2048, 16, 0, 0),
    "potts16-admm-1024-f32": ("potts", 2, 1024, 1024, 16, 0, 0),
    "potts16-admm-1024-f16": ("potts", 2, 1024, 1024, 16, 1, 0),
    "potts16-eval-1024-f32": ("potts-eval", 2, 1024, 1024, 16, 0, 0),
    # one two-phase solve of the 4096^2 workload (the bench's step), for a launch list
    "potts16-solve-4096": ("potts-solve", 2, 4096, 4096, 16, 0, 0),
    # the same solve host-driven (use_graph = 0): a profiler sees every launch
    "potts16-solve-host-4096": ("potts-solve-host", 2, 4096, 4096, 16, 0, 0),
    "potts16-admm-4096-f32": ("potts", 2, 4096, 4096, 16, 0, 0),
    "potts16-eval-2048-f32": ("potts-eval", 2, 2048, 2048, 16, 0, 0),
    "potts4-plain-2048": ("potts", 2, 2048, 2048, 4, 0, 1),
    # a host-driven solve to gap 1e-4 (use_graph = 0), so a profiler sees every launch
    "binary-solve-host-1024": ("binary-solve", 2, 1024, 1024, 2, 0, 0),
    # 16 painted-shapes instances (seeds 100..115) as one host-driven batch, `iters`
    # iterations: even and odd widths
    "potts4-batch-16x512": ("potts-batch", 2, 512, 512, 4, 0, 0),
    "potts4-batch-16x511": ("potts-batch", 2, 511, 511, 4, 0, 0),
}


def binary_workload(cmf, synth, flush, peak) -> dict:
    """The binary 1024^2 workload (eight disks / rectangles, edge-weighted
    alpha): time to the 1e-4 gap of every algorithm, fused and plain, and the
    two-iterations-per-launch warp-strip kernel's bandwidth.  Its state (about
    75 MB) stays in the 129 MB L2, so the bound is L2, not HBM."""
    import torch

    inst = synth.config2()
    out = {"workload": "binary 1024x1024 shapes, edge-weighted alpha, solve to gap 1e-4",
           "time_to_gap_ms": {}}
    for algo in (0, 1, 2, 3, 4, 5):
        for impl in (0, 1):
            q = cmf.default_params(algo, 2, tol_gap=TOL, max_iter=20000,
                                   check_every=CHECK_SIDE, impl=impl)
            bb = cmf.alloc_binary(inst, q)
            cmf.cmf_solve_binary(bb)  # warm (graph instantiation)
            ts = []
            for _ in range(3):
                flush.zero_()
                ms, (st, it, _) = _timed(lambda: cmf.cmf_solve_binary(bb))
                ts.append(ms)
            out["time_to_gap_ms"][f"{cmf.ALGO_NAMES[algo]}_{'fused' if impl == 0 else 'plain'}"] = {
                "ms": round(float(np.median(ts)), 3), "iters": it, "converged": st == cmf.OK}
            del bb
    t = out["time_to_gap_ms"]
    out["speedup_fused_vs_plain_rpADMMII"] = round(t["rpADMMII_plain"]["ms"] /
                                                   t["rpADMMII_fused"]["ms"], 3)
    # the fused kernel: 200 iterations = 100 two-iteration launches, back to back
    p = cmf.default_params(FLAGSHIP, 2)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    cmf.cmf_iterate_binary(b, 20)
    flush.zero_()
    ms, _ = _timed(lambda: cmf.cmf_iterate_binary(b, 200))
    launch_ms = ms / 100
    nbytes = 2 * algorithmic_bytes_per_px("binary", 2, 0, True) * inst.H * inst.W
    out["roofline"] = {"bound": "l2", "kernel": "k_binary_strip2", "launch_ms": launch_ms,
                       "iterations_per_launch": 2, "algorithmic_bytes_per_launch": nbytes,
                       "achieved": nbytes / launch_ms / 1e6, "unit": "GB/s",
                       "frac_of_hbm_peak": nbytes / launch_ms / 1e6 / peak,
                       "traffic": _traffic("paper_2004_11227_gb300/csrc/cmf_binary_strip2.cu",
                                           "k_binary_strip2"),
                       "note": "effective: iteration k+1 stays on chip and the state in L2"}
    return out


def potts4_workload(cmf, synth, flush, peak) -> dict:
    """The 4-label 2048^2 Voronoi workload (alpha 0.3): per flow storage the
    fused iteration's time and bandwidth and the time to the 1e-4 gap, the
    plain float32 form's time to the gap, and the same for rPDRQ (one
    red-black sweep, fused: k_potts_dr_strip)."""
    inst = synth.config3()
    out = {"workload": "potts L=4 2048x2048 Voronoi (64 seeds), alpha 0.3, solve to gap 1e-4"}
    for algo, storage, name, impl, max_iter in ((FLAGSHIP, 0, "float32", 0, 20000),
                                                (FLAGSHIP, 1, "float16", 0, 4000),
                                                (FLAGSHIP, 2, "bfloat16", 0, 4000),
                                                (FLAGSHIP, 0, "float32_plain", 1, 20000),
                                                (3, 0, "rPDRQ_float32", 0, 20000)):
        p = cmf.default_params(algo, inst.L, storage=storage, impl=impl, tol_gap=TOL,
                               max_iter=max_iter, check_every=CHECK_SIDE)
        s = cmf.alloc_potts(inst, p)
        cmf.cmf_init_potts(s)
        cmf.cmf_iterate_potts(s, 20)
        ms, _ = _timed(lambda: cmf.cmf_iterate_potts(s, 50))
        ms /= 50
        nb = algorithmic_bytes_per_px("potts", inst.L, storage, False) * inst.H * inst.W
        cmf.cmf_solve_potts(s)  # warm
        flush.zero_()
        ttg, (st, iters, hist) = _timed(lambda: cmf.cmf_solve_potts(s))
        out[name] = {"ms_per_iter": round(ms, 4), "px_label_it_per_s": inst.H * inst.W * inst.L / ms * 1e3,
                     "algorithmic_GBps": nb / ms / 1e6, "hbm_frac_of_measured": nb / ms / 1e6 / peak,
                     "bytes_per_px": nb // (inst.H * inst.W), "time_to_gap_ms": round(ttg, 2),
                     "iterations": iters, "converged": st == cmf.OK,
                     "final_gap": float(hist[-1, 3])}
        del s
    out["speedup_fused_vs_plain_float32"] = round(out["float32_plain"]["time_to_gap_ms"] /
                                                  out["float32"]["time_to_gap_ms"], 3)
    return out


def potts16_other_forms(cmf, inst, flush) -> dict:
    """The headline workload in one storage throughout: float32 flows, fused
    and plain, to the 1e-4 gap, and float16 flows alone (capped at 3000
    iterations: the certified gap stalls near 3e-4).  One solve each; building
    the solve graph, well under a millisecond of host time, is inside the
    timed region."""
    out = {}
    for name, storage, impl, max_iter in (("float32_fused", 0, 0, MAX_ITER),
                                          ("float32_plain", 0, 1, MAX_ITER),
                                          ("float16_fused_alone", 1, 0, 3000)):
        p = cmf.default_params(FLAGSHIP, L, storage=storage, impl=impl, tol_gap=TOL,
                               max_iter=max_iter, check_every=CHECK_EVERY)
        s = cmf.alloc_potts(inst, p)
        flush.zero_()
        ms, (st, iters, hist) = _timed(lambda: cmf.cmf_solve_potts(s))
        out[name] = {"time_to_gap_ms": round(ms, 1), "iterations": iters,
                     "converged": st == cmf.OK, "final_gap": float(hist[-1, 3]),
                     "ms_per_iter": round(ms / iters, 4)}
        del s
    return out


def tuned_step(cmf, inst, flush) -> dict:
    """The step-size search: cmf_autotune_potts with tune_step = 1 (c, 2c, 4c,
    8c beside the launch variants, each also with the switch left to the
    stall test) on the 1024^2 instance of the recipe, then one two-phase
    solve of the 4096^2 instance with the chosen c and switch gap."""
    small = rank_instance(0, 1024)
    p = cmf.default_params(FLAGSHIP, L, tol_gap=TOL, max_iter=MAX_ITER, check_every=CHECK_EVERY,
                           phase_storage=PHASE_STORAGE, phase_gap=TUNE_PHASE_GAP, tune_step=1)
    s = cmf.alloc_potts(small, p)
    t0 = time.perf_counter()
    best, ms_small = cmf.cmf_autotune_potts(s)
    tune_s = time.perf_counter() - t0
    del s
    q = cmf.default_params(FLAGSHIP, L, tol_gap=TOL, max_iter=MAX_ITER, check_every=CHECK_EVERY,
                           phase_storage=PHASE_STORAGE, phase_gap=best.phase_gap, c=best.c,
                           variant=best.variant)
    g = cmf.alloc_potts(inst, q)
    flush.zero_()
    ms, (st, iters, hist) = _timed(lambda: cmf.cmf_solve_potts(g))
    del g
    return {"c": best.c, "phase_gap": best.phase_gap, "variant": best.variant,
            "tuned_on": "1024x1024 instance of the recipe",
            "tuning_s": round(tune_s, 1), "time_to_gap_ms": round(ms, 1), "iterations": iters,
            "converged": st == cmf.OK, "final_gap": float(hist[-1, 3])}


def batch_workload(cmf, synth, flush) -> dict:
    """256 instances of uneven size (64^2..1024^2) and label count (2, 3, 4,
    8) solved as one batch (one graph, per-instance convergence masks) to the
    1e-4 gap with fused float32 rpADMMII: the time of the whole batch and the
    aggregate pixel*label*iterations/s (each instance counted to its own
    stopping iteration)."""
    import torch

    insts = synth.batch_instances()
    p = cmf.default_params(2, 2, tol_gap=1e-4, max_iter=5000, check_every=BATCH_CHECK)
    items = [cmf.alloc_binary(i, p) if i.kind == "binary" else cmf.alloc_potts(i, p)
             for i in insts]
    for it in items:  # the single-solve workspaces are not used by the batch
        it.ws = torch.empty(0, dtype=torch.uint8, device=it.u.device)
    torch.cuda.empty_cache()
    batch = cmf.Batch(items, p)
    batch.solve()  # warm (graph instantiation, module load)
    flush.zero_()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    st, res = batch.solve()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    units = sum(i.H * i.W * i.L * r["iters"] for i, r in zip(insts, res))
    iters = [r["iters"] for r in res]
    out = {"instances": len(insts), "check_every": BATCH_CHECK, "time_ms": round(ms, 2),
           "px_label_it_per_s": units / ms * 1e3,
           "converged": sum(1 for r in res if r["status"] == cmf.OK),
           "iters_min": min(iters), "iters_median": int(np.median(iters)), "iters_max": max(iters),
           "label_pixels": sum(i.H * i.W * i.L for i in insts)}
    # every instance's final state certified by the FP64 oracle: its relative
    # gap recomputed from the state the batch left in the caller's buffers
    import oracle as O

    O.build()
    O.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    og = []
    for inst, item in zip(insts, items):
        op = O.default_params(O.RPADMM_EB, inst.L)
        if inst.kind == "binary":
            og.append(O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, item.state(), op)[2])
        else:
            op.a2 = max(op.a2, 2.0 * inst.L)
            og.append(O.potts_eval(inst.costs, inst.alpha, item.state(), op)[2])
    og = np.array(og)
    gg = np.array([r["gap"] for r in res])
    out["oracle_certified"] = {
        "instances_at_or_below_1e-4": int(np.sum(og <= TOL * 1.01)),
        "oracle_gap_max": float(og.max()), "max_abs_gap_diff_vs_gpu": float(np.abs(og - gg).max()),
        "oracle_s": round(time.perf_counter() - t0, 1)}
    del batch, items
    torch.cuda.empty_cache()
    # the same instances solved one after another by the single-instance
    # solver (its automatic kernel choice, device-driven loop; allocation
    # outside the timed calls, graph building inside them)
    seq_ms, seq_units, seq_ok = 0.0, 0, 0
    for inst in insts:
        q = cmf.default_params(2, inst.L, tol_gap=1e-4, max_iter=5000, check_every=BATCH_CHECK)
        one = cmf.alloc_binary(inst, q) if inst.kind == "binary" else cmf.alloc_potts(inst, q)
        torch.cuda.synchronize()
        e0.record()
        st1, it1, _ = (cmf.cmf_solve_binary(one) if inst.kind == "binary"
                       else cmf.cmf_solve_potts(one))
        e1.record()
        e1.synchronize()
        seq_ms += e0.elapsed_time(e1)
        seq_units += inst.H * inst.W * inst.L * it1
        seq_ok += int(st1 == cmf.OK)
        del one
    torch.cuda.empty_cache()
    out["sequential_single_solves"] = {
        "time_ms": round(seq_ms, 2), "px_label_it_per_s": seq_units / seq_ms * 1e3,
        "converged": seq_ok, "batch_rate_over_sequential": (units / ms) / (seq_units / seq_ms)}
    return out


def batch_tuned(cmf, synth, flush) -> dict:
    """cmf_autotune_batch (check interval 20, 40, 100 x strip band height 12,
    16, 24) on a 64-instance batch of the same recipe (other seeds), then the
    256-instance batch solved with the chosen settings."""
    import torch

    small = synth.batch_instances(n=64, seed0=1000)
    p = cmf.default_params(2, 2, tol_gap=1e-4, max_iter=5000, check_every=BATCH_CHECK)
    items = [cmf.alloc_binary(i, p) if i.kind == "binary" else cmf.alloc_potts(i, p)
             for i in small]
    for it in items:
        it.ws = torch.empty(0, dtype=torch.uint8, device=it.u.device)
    t0 = time.perf_counter()
    best, ms_small = cmf.cmf_autotune_batch(items, p)
    tune_s = time.perf_counter() - t0
    del items
    insts = synth.batch_instances()
    items = [cmf.alloc_binary(i, best) if i.kind == "binary" else cmf.alloc_potts(i, best)
             for i in insts]
    for it in items:
        it.ws = torch.empty(0, dtype=torch.uint8, device=it.u.device)
    torch.cuda.empty_cache()
    batch = cmf.Batch(items, best)
    batch.solve()
    flush.zero_()
    ms, (st, res) = _timed(batch.solve)
    units = sum(i.H * i.W * i.L * r["iters"] for i, r in zip(insts, res))
    del batch, items
    torch.cuda.empty_cache()
    return {"check_every": best.check_every, "batch_rows": best.batch_rows,
            "tuned_on": "64 instances of the recipe (seeds 1000..1063)",
            "tuning_s": round(tune_s, 1), "time_ms": round(ms, 2),
            "px_label_it_per_s": units / ms * 1e3,
            "converged": sum(1 for r in res if r["status"] == cmf.OK)}


def oracle_checks(cmf, s, inst, flush) -> dict:
    """The FP64 oracle against the GPU on the headline workload.
    * one_step_windows: from the solved state, one GPU iteration against one
      oracle iteration of the same stored state on four windows (corners,
      interior), float16 results compared after rounding the oracle's;
    * certificate: the oracle's E, D and gap of the solved state (the whole
      4096^2 x 16 grid) against the GPU's;
    * labelling: the 256^2 instance of the same recipe solved to 1e-4 by the
      GPU (the same two-phase solve) and by the oracle; agreement of the argmax
      labels and max |u - u_oracle|."""
    import torch

    import oracle as O

    O.build()
    O.set_threads(os.cpu_count() or 1)
    out = {}
    po = O.default_params(FLAGSHIP, L)
    alpha = inst.alpha_field()
    # --- certificate of the solved state ---------------------------------------------
    t0 = time.perf_counter()
    st = s.state()
    E, D, gap, res = cmf.cmf_eval_potts(s)
    Eo, Do, gapo, reso = O.potts_eval(inst.costs, inst.alpha, st, po)
    out["certificate"] = {"gap_gpu": gap, "gap_oracle": gapo, "gap_diff": abs(gap - gapo),
                          "E_rel_diff": abs(E - Eo) / abs(Eo), "D_rel_diff": abs(D - Do) / abs(Eo),
                          "oracle_s": round(time.perf_counter() - t0, 1)}
    # --- one step on windows -----------------------------------------------------------
    keys = ("u", "qx", "qy", "p", "ps")
    Wd = s.W
    before = {k: getattr(s, k)[..., :Wd].float().clone() for k in keys}
    del st
    cmf.cmf_iterate_potts(s, 1)
    torch.cuda.synchronize()
    err = {k: 0.0 for k in keys}
    margin = 8
    for (r0, c0, h, w) in [(0, 0, 40, 40), (H - 37, W - 45, 37, 45), (2001, 3007, 64, 64),
                           (0, 1111, 33, 70)]:
        R0, C0 = max(r0 - margin, 0), max(c0 - margin, 0)
        R1, C1 = min(r0 + h + margin, H), min(c0 + w + margin, W)
        stw = {k: v[..., R0:R1, C0:C1].cpu().double().numpy() for k, v in before.items()}
        ref = O.potts_run(inst.costs[:, R0:R1, C0:C1], alpha[R0:R1, C0:C1], po, 1, stw)
        ri0, ci0 = r0 - R0, c0 - C0
        for k in keys:
            got = getattr(s, k)[..., r0:r0 + h, c0:c0 + w].float().cpu().double().numpy()
            rk = ref[k][..., ri0:ri0 + h, ci0:ci0 + w]
            t = getattr(s, k).dtype
            if k != "u":  # one rounding of the oracle's result to the stored type
                rk = torch.as_tensor(rk).to(t).double().numpy()
            err[k] = max(err[k], float(np.abs(got - rk).max()))
    out["one_step_windows_max_abs"] = err
    # --- 256^2: both solved to the gap -------------------------------------------------
    small = rank_instance(0, 256)
    p = cmf.default_params(FLAGSHIP, L, storage=STORAGE, costs=COSTS, tol_gap=TOL,
                           max_iter=MAX_ITER, check_every=CHECK_SIDE,
                           phase_storage=PHASE_STORAGE, phase_gap=PHASE_GAP)
    g = cmf.alloc_potts(small, p)
    stg, itg, hg = cmf.cmf_solve_potts(g)
    t0 = time.perf_counter()
    sto, ito, ho = O.solve(small, FLAGSHIP, tol=TOL, max_iter=MAX_ITER, check_every=50)
    ug = g.state()["u"]
    out["labelling_256"] = {
        "gpu_iters": itg, "gpu_gap": float(hg[-1, 3]), "oracle_iters": ito,
        "oracle_gap": float(ho[-1][3]),
        "agreement": float(np.mean(O.potts_labels(ug) == O.potts_labels(sto["u"]))),
        "max_abs_u_diff": float(np.abs(ug - sto["u"]).max()),
        "oracle_s": round(time.perf_counter() - t0, 1)}
    return out


def oracle_speed() -> dict:
    """The FP64 oracle's own speed on the two HBM-bound Potts workloads, on
    one host thread and on all of them (bounded samples, extrapolated to a
    whole solve with the GPU's iteration count)."""
    from paper_2004_11227_gb300 import synth

    out = {"host_cpu_count": os.cpu_count()}
    for name, inst, n1, nall in (("potts L=4 2048x2048", synth.config3(), 2, 10),
                                 ("potts L=16 4096x4096", rank_instance(0), 1, 4)):
        r1, dt1, _ = oracle_rate(inst, FLAGSHIP, n1, 1)
        ra, dta, used = oracle_rate(inst, FLAGSHIP, nall, 0)
        out[name] = {"one_thread": {"px_label_it_per_s": r1, "iterations": n1, "s": round(dt1, 2)},
                     "all_threads": {"px_label_it_per_s": ra, "iterations": nall,
                                     "s": round(dta, 2), "threads": used}}
    return out


def precision_study(size: int, max_iter: int):
    """Convergence of the 16-label Voronoi workload (edge-weighted alpha) at
    size x size under float32, float16 and bfloat16 flow storage: one JSON
    line per certificate check (iteration, E, D, gap) and per storage the
    relative primal-energy error against the float32 run's final energy."""
    import torch

    import __graft_entry__
    from paper_2004_11227_gb300 import cmf, synth

    __graft_entry__.build()
    inst = synth.config5(size, size)
    runs = {}
    for storage, name in ((0, "float32"), (1, "float16"), (2, "bfloat16")):
        p = cmf.default_params(2, 16, storage=storage, tol_gap=0.0, max_iter=max_iter,
                               check_every=50)
        s = cmf.alloc_potts(inst, p)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st, iters, hist = cmf.cmf_solve_potts(s, hist_cap=max_iter // 50 + 2)
        e1.record()
        e1.synchronize()
        runs[name] = (hist, e0.elapsed_time(e1) / iters)
        del s
        torch.cuda.empty_cache()
    e_ref = runs["float32"][0][-1, 1]
    for name, (hist, ms) in runs.items():
        rel = np.abs(hist[:, 1] - e_ref) / abs(e_ref)
        hit_gap = [int(h[0]) for h in hist if h[3] <= 1e-4]
        hit_rel = [int(hist[i, 0]) for i in range(len(hist)) if rel[i] <= 1e-4]
        print(json.dumps({"storage": name, "size": size, "ms_per_iter": ms,
                          "final_gap": float(hist[-1, 3]), "min_gap": float(hist[:, 3].min()),
                          "iters_to_gap_1e-4": hit_gap[0] if hit_gap else None,
                          "iters_to_primal_rel_1e-4_vs_f32_final": hit_rel[0] if hit_rel else None,
                          "trajectory": [[int(h[0]), float(h[3]), float(r)]
                                         for h, r in zip(hist[::4], rel[::4])]}))


def run_kernel_case(name: str, iters: int, time_it: bool = False, variant: int = 0):
    """Cold start plus `iters` iterations of one configuration: untimed for
    profiler captures (ncu -k <kernel> -c <n>), or timed with CUDA events."""
    import torch

    import __graft_entry__
    from paper_2004_11227_gb300 import cmf, synth

    __graft_entry__.build()
    model, algo, h, w, nl, storage, impl = KERNEL_CASES[name]
    p = cmf.default_params(algo, nl, storage=storage, impl=impl, variant=variant)
    if model in ("potts-solve", "potts-solve-host"):
        q = cmf.default_params(FLAGSHIP, nl, tol_gap=TOL, max_iter=MAX_ITER,
                               check_every=CHECK_EVERY, phase_storage=PHASE_STORAGE,
                               phase_gap=PHASE_GAP, use_graph=int(model == "potts-solve"))
        st = cmf.alloc_potts(rank_instance(0, h), q)
        print(name, cmf.cmf_solve_potts(st)[:2])
        torch.cuda.synchronize()
        return
    if model == "potts-batch":
        ins = [synth.potts_shapes(h, w, nl, seed=100 + k) for k in range(16)]
        q = cmf.default_params(algo, 2, tol_gap=1e-12, max_iter=max(10, (iters + 9) // 10 * 10),
                               check_every=10, use_graph=0)
        items = [cmf.alloc_potts(i, q) for i in ins]
        st_b, res = cmf.cmf_solve_batch(items, q)
        print(name, st_b, [r["iters"] for r in res][:4])
        torch.cuda.synchronize()
        return
    if model == "binary-solve":
        p.use_graph = 0
        b = cmf.alloc_binary(synth.config2(h, w), p)
        for _ in range(max(iters, 1)):
            print(name, cmf.cmf_solve_binary(b)[:2])
        torch.cuda.synchronize()
        return
    if model == "binary":
        inst = synth.config2(h, w)
        st = cmf.alloc_binary(inst, p)
        init, step, ev = cmf.cmf_init_binary, cmf.cmf_iterate_binary, cmf.cmf_eval_binary
    else:
        inst = synth.config3(h, w) if nl == 4 else synth.config5(h, w)
        st = cmf.alloc_potts(inst, p)
        init, step, ev = cmf.cmf_init_potts, cmf.cmf_iterate_potts, cmf.cmf_eval_potts
        if model == "potts-eval":  # certificate launches only, after `iters` iterations
            init(st)
            step(st, iters)
            for _ in range(3):
                print(name, ev(st))
            torch.cuda.synchronize()
            return
    init(st)
    step(st, iters)
    if time_it:
        n = max(iters, 20)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        step(st, n)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        nb = algorithmic_bytes_per_px(model, nl, storage,
                                      isinstance(inst.alpha, np.ndarray)) * h * w
        print(json.dumps({"case": name, "variant": variant, "ms_per_iter": ms,
                          "algorithmic_GBps": nb / ms / 1e6,
                          "px_label_it_per_s": h * w * nl / ms * 1e3}))
    print(name, ev(st))
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel-case", default=None, choices=sorted(KERNEL_CASES),
                    help="run one untimed configuration for a profiler capture")
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--time", action="store_true", help="time the kernel case")
    ap.add_argument("--variant", type=int, default=0, help="cmf_params.variant")
    ap.add_argument("--skip-side", action="store_true",
                    help="skip the side measurements (other workloads, oracle checks)")
    ap.add_argument("--precision-study", type=int, default=0, metavar="SIZE",
                    help="convergence of the 16-label workload at SIZE^2 per storage type")
    ap.add_argument("--study-iters", type=int, default=6000)
    args = ap.parse_args()
    if args.precision_study:
        precision_study(args.precision_study, args.study_iters)
        return
    if args.kernel_case:
        run_kernel_case(args.kernel_case, args.iters, args.time, args.variant)
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2004_11227_gb300 import cmf, synth

    world, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peak, peak_kind = _peaks()
    inst = rank_instance(rank)
    p = cmf.default_params(FLAGSHIP, L, storage=STORAGE, costs=COSTS, tol_gap=TOL,
                           max_iter=MAX_ITER, check_every=CHECK_EVERY,
                           phase_storage=PHASE_STORAGE, phase_gap=PHASE_GAP)
    s = cmf.alloc_potts(inst, p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        st, iters, hist = cmf.cmf_solve_potts(s)
        assert st == cmf.OK, f"solve did not reach the gap (status {st}, gap {hist[-1, 3]})"
        return iters, hist

    warmup = max(args.warmup, 3)
    for _ in range(warmup):
        step()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    times, iters_all, gaps, phase1 = [], [], [], []
    for _ in range(args.steps):
        flush.zero_()
        ms, (iters, hist) = _timed(step)
        times.append(ms)
        iters_all.append(iters)
        gaps.append(float(hist[-1, 3]))
        # the check that ended the 16-bit phase
        phase1.append(int(hist[phase_one_end(hist, PHASE_GAP, CHECK_EVERY), 0]))
    barrier()
    clocks = sampler.stop()
    total_ms, total_units = job_totals(times, iters_all, world, dev)
    value = total_units / (total_ms / 1000.0)
    iters = int(np.median(iters_all))
    it16 = int(np.median(phase1))
    # per solve: cold start, two loop resets, the float16-to-float32 switch;
    # per check: check_every iteration launches, the launch that turns w back
    # into u, the certificate launch (its last block reduces and takes the
    # stop decision)
    launches = args.steps * (4 + (iters // CHECK_EVERY) * (CHECK_EVERY + 2))

    # --- end to end through the C ABI with host buffers -------------------------------
    cdt = s.C.dtype
    costs_h = torch.empty(tuple(s.C.shape), dtype=cdt).pin_memory()
    costs_h.copy_(s.C.cpu())
    alpha_h = torch.empty(tuple(s.alpha.shape), dtype=torch.float32).pin_memory()
    alpha_h.copy_(s.alpha.cpu())
    u_h = torch.empty(tuple(s.u.shape), dtype=torch.float32).pin_memory()
    e2e_times = []
    n_e2e = min(args.steps, 3)
    barrier()
    for _ in range(n_e2e):
        flush.zero_()

        def e2e_step():
            s.C.copy_(costs_h, non_blocking=True)
            s.alpha.copy_(alpha_h, non_blocking=True)
            it, _ = step()
            u_h.copy_(s.u, non_blocking=True)
            return it

        ms, it = _timed(e2e_step)
        e2e_times.append(ms)
    barrier()
    e2e_ms = job_max_ms(e2e_times, world, dev) / n_e2e
    e2e_value = H * W * L * iters * world / (e2e_ms / 1000.0)
    h2d = costs_h.numel() * costs_h.element_size() + alpha_h.numel() * 4
    d2h = u_h.numel() * 4

    # --- the fused iteration, back to back: float16 (phase one), float32 (two) -------
    def kernel_ms(storage):
        q = cmf.default_params(FLAGSHIP, L, storage=storage, costs=COSTS)
        k = cmf.alloc_potts(inst, q)
        cmf.cmf_init_potts(k)
        cmf.cmf_iterate_potts(k, 20)
        flush.zero_()
        ms, _ = _timed(lambda: cmf.cmf_iterate_potts(k, 50))
        del k
        torch.cuda.empty_cache()
        return ms / 50

    ms16, ms32 = kernel_ms(1), kernel_ms(0)
    t16, t32 = ms16 * it16, ms32 * (iters - it16)
    storage_dom = 1 if t16 >= t32 else 0
    launch_ms = ms16 if storage_dom == 1 else ms32
    # algorithmic bytes of the dominant instantiation: for float32 every field
    # in 4 bytes (u, q_i, p_i, p_s read and written, costs and alpha read:
    # 16 x 36 + 8 + 4 = 588 B/px); for the float16 phase q_i and p_i in 2 bytes
    # with u and p_s in 4 (396 B/px) -- rounding either of those two to 16
    # bits stalls this workload's gap at 3e-2 and 4e-4, above the target, so
    # the 16-bit count of every field (296 B/px) is reported beside it
    algo_px = algorithmic_bytes_per_px("potts", L, storage_dom, True, "f32")
    design_px = algorithmic_bytes_per_px("potts", L, storage_dom, True,
                                         {0: "f32", 2: "f16"}[COSTS])
    achieved = algo_px * H * W / (launch_ms / 1000.0) / 1e9
    name = "k_potts_strip<__half>" if storage_dom == 1 else "k_potts_strip<float>"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": _traffic("paper_2004_11227_gb300/csrc/cmf_potts_strip.cu", name),
                "kernel": name, "peak_kind": peak_kind,
                "algorithmic_bytes_per_px": algo_px,
                "algorithmic_bytes_per_launch": algo_px * H * W, "launch_ms": launch_ms,
                "design_bytes_per_px": design_px,
                "time_share_in_solve": {"float16_phase": t16 / (t16 + t32),
                                        "float32_phase": t32 / (t16 + t32)},
                "float16_kernel": {"launch_ms": ms16, "bytes_per_px_16bit": BYTES_PER_PX_16BIT,
                                   "frac_16bit_count": BYTES_PER_PX_16BIT * H * W / ms16 / 1e6 / peak,
                                   "design_bytes_per_px": algorithmic_bytes_per_px(
                                       "potts", L, 1, True, {0: "f32", 2: "f16"}[COSTS]),
                                   "frac_design": algorithmic_bytes_per_px(
                                       "potts", L, 1, True, {0: "f32", 2: "f16"}[COSTS]) *
                                   H * W / ms16 / 1e6 / peak},
                "float32_kernel": {"launch_ms": ms32,
                                   "frac": algorithmic_bytes_per_px("potts", L, 0, True, "f32") *
                                   H * W / ms32 / 1e6 / peak},
                "note": "launch time = 50 back-to-back iterations / 50 (one w-to-u pass per "
                        "call included); the dominant instantiation by time in the solve"}

    side = {}
    if rank == 0 and not args.skip_side:
        side["potts16_float32_flows"] = potts16_other_forms(cmf, inst, flush)
        side["potts16_tuned_step"] = tuned_step(cmf, inst, flush)
        side["oracle_check"] = oracle_checks(cmf, s, inst, flush)
        del s
        torch.cuda.empty_cache()
        side["potts4_2048"] = potts4_workload(cmf, synth, flush, peak)
        side["binary_1024"] = binary_workload(cmf, synth, flush, peak)
        side["batch_workload"] = batch_workload(cmf, synth, flush)
        side["batch_workload"]["tuned"] = batch_tuned(cmf, synth, flush)
        side["oracle_speed"] = oracle_speed()

    if rank == 0:
        c5 = side.get("oracle_speed", {}).get("potts L=16 4096x4096", {})
        if c5:
            rate, used = c5["all_threads"]["px_label_it_per_s"], c5["all_threads"]["threads"]
            sample = (f"{c5['all_threads']['iterations']} rpADMMII iterations of the full "
                      f"4096x4096x16 workload, FP64 C oracle, {used} threads "
                      f"({c5['all_threads']['s']} s)")
        else:
            rate, dt, used = oracle_rate(inst, FLAGSHIP, 1, 0)
            sample = (f"1 rpADMMII iteration of the full 4096x4096x16 workload, FP64 C oracle, "
                      f"{used} threads ({dt:.1f} s)")
        f32 = side.get("potts16_float32_flows", {})
        line = {
            "metric": "pixel*label*iterations/s", "value": value, "unit": "px*label*it/s",
            "n_gpus": world, "steps": args.steps, "warmup": warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H, "W": W, "L": L, "algo": "rpADMMII fused",
                       "flow_storage": "float16 q_i, p_i until the gap stalls (switch gap "
                                       "1.5e-4 with the stall test), then float32; p_s, u "
                                       "float32",
                       "check_every": CHECK_EVERY, "tol_gap": TOL,
                       "l2": "inputs and state (several GB) far larger than L2; 256 MB flush "
                             "before every timed step",
                       "parallelism": f"replicas x{world}"},
            "time_to_gap_ms": {"two_phase_fused": round(float(np.median(times)), 1),
                               "iterations": iters, "iterations_float16_phase": it16,
                               "final_gap_max": max(gaps),
                               **{k: v["time_to_gap_ms"] for k, v in f32.items()},
                               **({"speedup_two_phase_vs_float32_fused": round(
                                   f32["float32_fused"]["time_to_gap_ms"] /
                                   float(np.median(times)), 3),
                                   "speedup_two_phase_vs_plain_float32": round(
                                   f32["float32_plain"]["time_to_gap_ms"] /
                                   float(np.median(times)), 3)} if f32 else {})},
            "roofline": roofline,
            "cpu_baseline": {"value": rate, "unit": "px*label*it/s", "cores": used,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": e2e_value, "unit": "px*label*it/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            **side,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
