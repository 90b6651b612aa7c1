#!/usr/bin/env python3
"""Benchmark of the FVLBM time step (arXiv 1812.00394, Part II) on GB300.

Default workload: the uneven batched sweep -- 48 instances (32 laminar Delaunay cavities of
10k-40k triangles at Re 100-3200, 4 turbulent backward-facing steps of ~80k hybrid cells, 12
turbulent NACA 0012 C-meshes of 50k-200k cells at 0-12 degrees), advanced together by one
handle of the CUDA library (every launch of a step covers all instances, CUDA-graph replayed).
A "step" is one full time step of every instance (SST where enabled, three IMEX stages, final
update).  The metric is Mcell-steps/s of the FP32 deviation-storage path; the plain FP64 path
is timed on the same workload beside it, and both are compared with the FP64 CPU oracle.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torch.distributed.run: the one sweep is split across the ranks, its
instances balanced by cell count (strong scaling; instances never exchange data inside a
step), and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mcell-steps/s FP32/batched vs plain FP64 at stated L2 error; % HBM roofline"
UNIT = "Mcell-steps/s"
L2_BYTES = 129e6
# Algorithmic HBM bytes per cell-step of the whole step (minimal fused design: 114 state
# words plus 84 B of neighbour indices; +34 words with k-omega SST), per storage precision.
STEP_BYTES = {("f32", False): 540.0, ("f32", True): 676.0, ("f64", False): 996.0, ("f64", True): 1268.0}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:  # noqa: BLE001
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- workload
def make_workload(name: str):
    from paper_1812_00394_gb300 import meshgen as mg
    if name == "sweep":
        return mg.batched_sweep(seed=5)
    if name == "sweep_small":  # the sweep's kinds in small (7 instances), for counter captures
        return mg.batched_sweep(seed=5, n_cavity=4, n_bfs=1, n_naca=2)
    if name == "delaunay40k":
        return [mg.cavity_delaunay(re=1000.0, z=5.0, seed=2)]
    if name == "cavity64":
        return [mg.cavity_quad(64, re=400.0, seed=1)]
    raise ValueError(name)


def host_cores() -> int:
    """Cores this process may run on (the machine's host cores available to the oracle)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # not Linux
        return os.cpu_count() or 1


def _sample_indices(cases):
    """One instance of each kind (first cavity, first BFS, first NACA) for oracle checks."""
    picks, seen = [], set()
    for i, c in enumerate(cases):
        kind = c.name.split("_")[0].rstrip("0123456789")
        if kind not in seen:
            seen.add(kind)
            picks.append(i)
    return picks


# ----------------------------------------------------------------------------- reference arm
def cpu_oracle_rate(cases, budget_s: float, max_steps: int = 50, threads: int = 1):
    """Time the FP64 oracle, as it stands, on a bounded sample: each sampled instance is
    stepped until about budget_s / n_samples seconds are spent, with its per-cell loops on
    `threads` threads.  Returns (Mcell-steps/s, desc)."""
    from oracle import oracle as orc
    from oracle.oracle import Oracle
    orc.set_threads(threads)
    picks = _sample_indices(cases)
    cell_steps, secs, desc = 0, 0.0, []
    for i in picks:
        o = Oracle(cases[i])
        n, t0 = 0, time.perf_counter()
        while n < max_steps and time.perf_counter() - t0 < budget_s / len(picks):
            o.step(1)
            n += 1
        dt = time.perf_counter() - t0
        cell_steps += n * cases[i].mesh.n_cells
        secs += dt
        desc.append(f"{cases[i].name} x {n} steps")
    return cell_steps / secs / 1e6, "; ".join(desc)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cases = make_workload(args.workload)
    picks = _sample_indices(cases)
    from oracle import oracle as orc
    from oracle.oracle import Oracle
    cores = host_cores()
    orc.set_threads(cores)          # the oracle's per-cell loops on every host core
    oracles = [Oracle(cases[i]) for i in picks]
    # the first warm-up step times each sampled instance; the largest are dropped until the
    # remaining steps fit the time budget (one instance stays)
    cost = []
    for o in oracles:
        t0 = time.perf_counter()
        o.step(1)
        cost.append(time.perf_counter() - t0)
    keep = list(range(len(picks)))
    rest = args.steps + max(args.warmup - 1, 0)
    while len(keep) > 1 and rest * sum(cost[j] for j in keep) > args.ref_budget:
        keep.remove(max(keep, key=lambda j: cost[j]))
    picks = [picks[j] for j in keep]
    oracles = [oracles[j] for j in keep]
    cells = sum(cases[i].mesh.n_cells for i in picks)
    for _ in range(args.warmup - 1):
        for o in oracles:
            o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for o in oracles:
            o.step(1)
    el = time.perf_counter() - t0
    value = cells * args.steps / el / 1e6
    sample = (f"each step = one FP64 oracle time step of {len(picks)} instances of the sweep "
              f"({', '.join(cases[i].name for i in picks)}; {cells} cells), per-cell loops on "
              f"{cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": _workload_desc(args.workload), "instances": len(cases),
                   "cells": sum(c.mesh.n_cells for c in cases), "sample_cells": cells,
                   "precision": "fp64 CPU oracle (a bounded sample of the workload per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "host_nproc": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ----------------------------------------------------------------------------- our arm
def _time_steps(torch, solver, stream, steps, dist, world):
    """K steps bracketed by barrier + synchronize; CUDA events on the handle's stream."""
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    solver.step(steps)
    stop.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    return max_over_ranks(torch, dist, world, start.elapsed_time(stop), device="cuda")


def max_over_ranks(torch, dist, world: int, value: float, device: str = "cuda") -> float:
    """The slowest rank's time (all ranks get it); a no-op for one rank.  Inside a step the
    ranks exchange nothing: the sweep's instances are sharded by rank."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(torch, dist, world: int, value, device: str = "cuda"):
    """The sum over ranks of a number or an array (per-rank parts of a sweep-wide total); a
    no-op for one rank."""
    if world <= 1:
        return value
    scalar = np.ndim(value) == 0
    t = torch.tensor(np.atleast_1d(np.asarray(value, np.float64)), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = t.cpu().numpy()
    return float(out[0]) if scalar else out


def shard_of(cases, world: int, rank: int):
    """This rank's share of the sweep (cell-balanced, see paper_1812_00394_gb300.shard)."""
    from paper_1812_00394_gb300.shard import assign_instances
    return [cases[i] for i in assign_instances([c.mesh.n_cells for c in cases], world)[rank]]


def aggregate_rate(cells_all_ranks: float, steps: int, ms_max: float) -> float:
    """Whole-job Mcell-steps/s: the cells all ranks advanced over the slowest rank's time."""
    return cells_all_ranks * steps / (ms_max * 1e-3) / 1e6


def _vel(fields):
    return np.concatenate([fields["u"], fields["v"]])


def run_ours(args):
    import torch
    from paper_1812_00394_gb300 import fvlbm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()

    t_setup = time.perf_counter()
    sweep = make_workload(args.workload)          # the same sweep on every rank
    cases = shard_of(sweep, world, rank)          # this rank's instances
    total_cells = sum(c.mesh.n_cells for c in cases)
    sst_cells = sum(c.mesh.n_cells for c in cases if c.sst)
    cells_job = sum(c.mesh.n_cells for c in sweep)
    fvlbm.load()

    results = {}
    solvers = {}
    for prec, tag in ((fvlbm.FVLBM_FP32_DEV, "f32"), (fvlbm.FVLBM_FP64, "f64")):
        with torch.cuda.stream(stream):
            s = fvlbm.Solver(cases, precision=prec, device=dev, stream=stream.cuda_stream)
            s.step(args.warmup)
            tuned = s.autotune(3)            # kernel configuration chosen by measurement
            torch.cuda.synchronize()
            with ClockSampler(dev) as clk:
                ms = _time_steps(torch, s, stream, args.steps, dist, world)
            results[tag] = {"ms": ms, "clocks": clk.summary(), "autotune": tuned}
        solvers[tag] = s
    # the explicit Euler comparison scheme (Sec. 3.1 / 4.1) on the same workload, FP32: cost per
    # step (its stable dt is < 2 tau, the IMEX one is not limited by tau)
    with torch.cuda.stream(stream):
        se = fvlbm.Solver(cases, precision=fvlbm.FVLBM_FP32_DEV, device=dev,
                          stream=stream.cuda_stream, scheme=fvlbm.SCHEME_EULER)
        se.step(args.warmup)
        ms_euler = _time_steps(torch, se, stream, args.steps, dist, world)
        se.close()
    setup_s = time.perf_counter() - t_setup

    ms32 = results["f32"]["ms"]
    value = aggregate_rate(cells_job, args.steps, ms32)
    ms64 = results["f64"]["ms"]
    value64 = aggregate_rate(cells_job, args.steps, ms64)

    # FP32 against FP64 (both GPU) after the same warmup + timed steps, on every cell of the
    # sweep: per kind of instance (sums of squares over all ranks) and C_D, C_L of every airfoil
    s32, s64 = solvers["f32"], solvers["f64"]
    kinds = ("cavity", "bfs", "naca")
    sq = np.zeros(2 * len(kinds))
    force_err = np.zeros(2)
    for i, c in enumerate(cases):
        k = kinds.index(c.name.split("_")[0].rstrip("0123456789"))
        a, b = _vel(s32.fields(i)), _vel(s64.fields(i))
        sq[2 * k] += float(np.sum((a - b) ** 2))
        sq[2 * k + 1] += float(np.sum(b ** 2))
        if c.name.startswith("naca"):
            f32, f64 = s32.forces(i), s64.forces(i)
            force_err[0] = max(force_err[0], abs(f32["cd"] - f64["cd"]) / abs(f64["cd"]))
            force_err[1] = max(force_err[1], abs(f32["cl"] - f64["cl"]) / max(abs(f64["cl"]), 1e-3))
    sq = sum_over_ranks(torch, dist, world, sq)
    force_err = [max_over_ranks(torch, dist, world, float(x)) for x in force_err]
    err_kind = {}
    for k, kind in enumerate(kinds):
        if sq[2 * k + 1] > 0:
            err_kind[f"fp32_vs_fp64_gpu_velocity_rel_l2[{kind}]"] = float(np.sqrt(sq[2 * k] / sq[2 * k + 1]))
    l2_32_64 = float(np.sqrt(sq[0::2].sum() / sq[1::2].sum()))
    err_kind["fp32_vs_fp64_gpu_cd_max_rel"] = float(force_err[0])
    err_kind["fp32_vs_fp64_gpu_cl_max_rel"] = float(force_err[1])
    err_kind["fp32_vs_fp64_after_steps"] = args.warmup + args.steps
    err_kind["fp32_within_target"] = bool(
        all(v <= 1e-4 for kk, v in err_kind.items() if kk.startswith("fp32_vs_fp64_gpu_velocity"))
        and force_err[0] <= 5e-3 and force_err[1] <= 5e-3)
    err_kind["target"] = "velocity rel L2 <= 1e-4 per kind of instance; C_D, C_L each <= 0.5 %"

    # per-kernel device times (CUDA events on the handle's stream) for the roofline
    with torch.cuda.stream(stream):
        prof = s32.profile_kernels(max(4, min(args.steps, 20)))
    kname, kstat = max(prof.items(), key=lambda kv: kv[1]["ms"])
    per_launch_ms = kstat["ms"] / kstat["launches"]
    hbm, peak_kind = _peaks()
    lam_cells = total_cells - sst_cells
    face_value = results["f32"]["autotune"][0] == "facevalue"
    kbytes = _kernel_bytes(kname, "f32", total_cells, sst_cells, face_value)
    achieved = kbytes / (per_launch_ms * 1e-3) / 1e9
    step_bytes = lam_cells * STEP_BYTES[("f32", False)] + sst_cells * STEP_BYTES[("f32", True)]
    step_gbs = step_bytes / (ms32 / args.steps * 1e-3) / 1e9
    lps = s32.footprint()[1]
    dev_bytes = s32.footprint()[0]
    traffic, traffic_src = _ncu_traffic(kname, args.workload, world, face_value)

    # errors against the FP64 CPU oracle on sampled instances (fresh short runs)
    err = {}
    if rank == 0 and not args.no_oracle_check:
        err = _oracle_errors(cases, fvlbm, dev, stream, torch, nsteps=args.check_steps)

    # end to end through the C ABI with pinned host buffers: upload f, one step, read u, v;
    # pipelined (async calls) for the headline, synchronous calls for context
    e2e = _e2e(torch, fvlbm, s32, stream, args, world, dist, cells_job, pipelined=True, f32_io=True)
    e2e_f64 = _e2e(torch, fvlbm, s32, stream, args, world, dist, cells_job, pipelined=True)
    e2e_sync = _e2e(torch, fvlbm, s32, stream, args, world, dist, cells_job, pipelined=False)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate1, sample1 = cpu_oracle_rate(cases, args.cpu_budget / 2, threads=1)
        rate_n, sample_n = cpu_oracle_rate(cases, args.cpu_budget / 2, threads=cores)
        cpu = {"value": rate_n, "unit": UNIT, "cores": cores, "host_nproc": cores, "kind": "oracle",
               "sample": sample_n + f" (FP64 CPU oracle, per-cell loops on {cores} threads, this host)",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": sample1 + " (FP64 CPU oracle, one thread, this host)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": _workload_desc(args.workload), "instances": len(sweep),
                       "cells": cells_job, "cells_rank0": total_cells, "sst_cells_rank0": sst_cells,
                       "precision": "fp32 f-w*rho0 deviation storage, fp32 arithmetic, fp64 reductions",
                       "l2": f"inputs larger than L2 (device working set {dev_bytes / 1e6:.0f} MB > 129 MB); no flush",
                       "parallelism": f"{world} process(es), one per GPU; the sweep's instances split "
                                      f"across them by cell count"},
            "fp64_plain": {"value": value64, "unit": UNIT, "ms_per_step": ms64 / args.steps,
                           "speedup_fp32_over_fp64": value / value64,
                           "roofline": _fp64_roofline(fvlbm, dev, total_cells, sst_cells,
                                                      ms64 / args.steps, args.workload,
                                                      results["f64"]["autotune"][0])},
            "explicit_euler_fp32": {"ms_per_step": ms_euler / args.steps,
                                    "imex_over_euler_cost_per_step": ms32 / ms_euler,
                                    "note": "comparison scheme of Sec. 4.1: stable only for dt < 2 tau"},
            "error": {"fp32_vs_fp64_gpu_velocity_rel_l2": l2_32_64, **err_kind, **err},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                         "traffic_source": traffic_src, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": kbytes,
                         "avg_launch_ms": per_launch_ms},
            "step_roofline": {"bytes_per_cell_step": step_bytes / total_cells,
                              "achieved": step_gbs, "peak": hbm, "unit": "GB/s",
                              "frac": step_gbs / hbm, "peak_kind": peak_kind},
            "autotune": {"fp32": {"chosen": results["f32"]["autotune"][0],
                                  "ms_per_step": results["f32"]["autotune"][1]},
                         "fp64": {"chosen": results["f64"]["autotune"][0],
                                  "ms_per_step": results["f64"]["autotune"][1]}},
            "kernels": {k: _kernel_line(k, v, total_cells, sst_cells, face_value, hbm)
                        for k, v in prof.items()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_f64_io": e2e_f64,
            "e2e_sync": e2e_sync,
            "clocks": results["f32"]["clocks"],
            "clocks_fp64": results["f64"]["clocks"],
            "gpu_launches": lps * args.steps,
            "setup_s": setup_s,
        }
        print(json.dumps(line))
    for s in solvers.values():
        s.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def _workload_desc(name):
    return {"sweep": "batched sweep: 48 instances (32 laminar Delaunay cavities 10k-40k cells "
                     "Re 100-3200, 4 SST backward-facing steps ~80k cells, 12 SST NACA0012 "
                     "C-meshes 50k-200k cells alpha 0-12 deg), CFL 0.5 each",
            "delaunay40k": "laminar lid-driven cavity Re 1000, seeded Delaunay ~40k triangles, dt = 5 tau",
            "cavity64": "laminar lid-driven cavity Re 400, 64x64 quads, CFL 0.5",
            "sweep_small": "the batched sweep's kinds in small: 4 cavities, 1 SST backward-facing "
                           "step, 2 SST NACA0012 C-meshes"}[name]


PROFILE_SUMMARY = {False: "k_fused_stage_fp32_sweep.md", True: "k_fused_fv_fp32_sweep.md"}


def kernel_source_sha256() -> str:
    """SHA-256 over the sources of the stage kernels (fvlbm_kernels.cu, fvlbm_fused_fv.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("fvlbm_kernels.cu", "fvlbm_fused_fv.cuh"):
        with open(os.path.join(ROOT, "paper_1812_00394_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _ncu_traffic(kname, workload, world, face_value=False):
    """(DRAM bytes read + written per launch of kernel `kname`, where the figure comes from).
    The figure is read from the committed ncu summary of the default sweep under profiles/,
    and only while the kernel sources hash to the value that summary records (the capture was
    taken on these sources); otherwise (None, reason)."""
    import re
    if workload != "sweep":
        return None, "no ncu capture for this workload"
    fname = PROFILE_SUMMARY[bool(face_value)]
    try:
        sha = kernel_source_sha256()
        with open(os.path.join(ROOT, "profiles", fname)) as fh:
            txt = fh.read()
    except OSError:
        return None, f"profiles/{fname} not found"
    m = re.search(r"kernel_source_sha256=([0-9a-f]{64})((?: \w+=\d+)+)", txt)
    if not m or m.group(1) != sha:
        return None, f"profiles/{fname} was captured on other kernel sources"
    vals = dict(kv.split("=") for kv in m.group(2).split())
    if kname not in vals:
        return None, f"profiles/{fname} has no figure for {kname}"
    return float(vals[kname]), f"ncu capture committed in profiles/{fname} (kernel sources sha256 {sha[:16]}...)"


def _fp64_roofline(fvlbm, dev, cells, sst_cells, ms_per_step, workload, config):
    """The FP64 path against the FP64 pipe: FP64 flops per step (from the committed ncu count of
    the two-pass kernels' DADD, DMUL and DFMA instructions, per cell and per SST cell, valid
    while the kernel sources hash to the recorded value) over the measured FMA peak."""
    import re
    try:
        peak = fvlbm.fvlbm_fp64_peak(dev)
    except Exception as e:  # noqa: BLE001 -- reported, not fatal
        return {"bound": "alu", "pipe": "fp64", "peak": None, "error": str(e)}
    out = {"bound": "alu", "pipe": "fp64", "peak": peak, "unit": "TFLOP/s",
           "peak_kind": "measured FP64 FMA rate (fvlbm_fp64_peak)", "achieved": None, "frac": None}
    if workload != "sweep" or config != "twopass":
        out["source"] = "flop counts are for the two-pass kernels on the sweep only"
        return out
    try:
        with open(os.path.join(ROOT, "profiles", "k_flux_stage_fp64_sweep.md")) as fh:
            txt = fh.read()
    except OSError:
        out["source"] = "profiles/k_flux_stage_fp64_sweep.md not found"
        return out
    m = re.search(r"kernel_source_sha256=([0-9a-f]{64}) fp64_flops_per_cell=([0-9.e+]+) "
                  r"fp64_flops_per_sst_cell=([0-9.e+]+)", txt)
    if not m or m.group(1) != kernel_source_sha256():
        out["source"] = "profiles/k_flux_stage_fp64_sweep.md was counted on other kernel sources"
        return out
    flops = cells * float(m.group(2)) + sst_cells * float(m.group(3))
    out.update(flops_per_step=flops, achieved=flops / (ms_per_step * 1e-3) / 1e12,
               source="ncu instruction counts committed in profiles/k_flux_stage_fp64_sweep.md")
    out["frac"] = out["achieved"] / peak
    return out


def _kernel_line(kname, v, cells, sst_cells, face_value, hbm):
    """Average launch time of one kernel and, where its algorithmic bytes are defined, its
    achieved GB/s and fraction of the measured HBM peak."""
    ms = v["ms"] / v["launches"]
    out = {"avg_ms": ms, "launches": v["launches"]}
    try:
        b = _kernel_bytes(kname, "f32", cells, sst_cells, face_value)
    except KeyError:
        return out
    gbs = b / (ms * 1e-3) / 1e9
    out.update(algorithmic_bytes=b, achieved_gbs=gbs, frac=gbs / hbm)
    return out


def _kernel_bytes(kname, prec, cells, sst_cells, face_value=False):
    """Algorithmic bytes of one launch of each kernel: its per-cell state reads and writes
    counted once (neighbour values assumed reused from cache), neighbour indices 4 B each
    (3.5 per cell), geometry not counted (recomputable).  With the face-value stages the SST
    update writes no f^(1) (stage 1 relaxes f^n itself)."""
    w = 4 if prec == "f32" else 8
    idx = 14.0
    if face_value and kname == "sst_update":
        return sst_cells * ((3 + 3 + 12 + 1 + 4) * w + idx)
    words = {
        "stage1": 9 + 1 + 9,                       # f^n, tau -> f^(1)
        "grad_f": 9 + 18,                          # f^(J) -> gradient
        "flux_stage1": 9 + 18 + 9 + 1 + 27,        # f1, g, f^n, tau -> f2, B, C
        "flux_stage2": 9 + 18 + 18 + 1 + 18,       # f2, g, B, C, tau -> f3, C
        "flux_stage3": 9 + 18 + 9 + 1 + 9 + 3,     # f3, g, C, tau -> f^{n+1}, macros
        "sst_grad": 3 + 2 + 1 + 12 + 1,
        "sst_update": 3 + 3 + 12 + 1 + 4 + 9 + 9,  # + f^n -> f^(1) (fused path)
        "fused_stage1": 9 + 1 + 27,                # f^n, tau -> f2, B, C (gradient in smem)
        "fused_stage2": 9 + 18 + 1 + 18,           # f2, B, C, tau -> f3, C
        "fused_stage3": 9 + 9 + 1 + 12,            # f3, C, tau -> f^{n+1}, macros
    }[kname]
    n = sst_cells if kname.startswith("sst") else cells
    return n * (words * w + idx)


def _oracle_errors(cases, fvlbm, dev, stream, torch, nsteps):
    from oracle.oracle import Oracle
    out = {}
    worst_vel, worst_force = 0.0, 0.0
    for i in _sample_indices(cases):
        c = cases[i]
        o = Oracle(c)
        o.step(nsteps)
        fo = o.fields()
        for prec, tag in ((fvlbm.FVLBM_FP32_DEV, "f32"), (fvlbm.FVLBM_FP64, "f64")):
            with torch.cuda.stream(stream):
                s = fvlbm.Solver(c, precision=prec, device=dev, stream=stream.cuda_stream)
                s.step(nsteps)
                fg = s.fields()
                fr = s.forces()
                s.close()
            e = float(np.linalg.norm(_vel(fg) - _vel(fo)) / np.linalg.norm(_vel(fo)))
            out[f"{tag}_vs_oracle_velocity_rel_l2[{c.name}]"] = e
            if tag == "f32":
                worst_vel = max(worst_vel, e)
                if c.name.startswith("naca"):
                    ofr = o.forces()
                    sc = math.hypot(ofr["cd"], ofr["cl"])
                    worst_force = max(worst_force, abs(fr["cd"] - ofr["cd"]) / sc,
                                      abs(fr["cl"] - ofr["cl"]) / sc)
    out["oracle_check_steps"] = nsteps
    out["f32_worst_velocity_rel_l2"] = worst_vel
    out["f32_worst_cd_cl_rel"] = worst_force
    return out


def _e2e(torch, fvlbm, solver, stream, args, world, dist, cells_job, pipelined=True, f32_io=False):
    """Same metric through the public API with host buffers: per step, an upload of the whole
    state (all instances, FVLBM_ALL_INSTANCES) from pinned host memory, one fvlbm_step, and a
    read of u and v back to pinned host memory.  pipelined=True uses fvlbm_set_f_async /
    fvlbm_get_fields_async (transfers on the copy engines overlap the steps, two host buffers
    per direction, one fvlbm_wait at the end); pipelined=False the synchronous calls.
    f32_io=True uploads the state in the FP32 deviation format of the FP32 path
    (fvlbm_set_fdev_f32_async: f - w rho0 as float, half the bytes of double f)."""
    import ctypes as C
    total = fvlbm.fvlbm_info(solver.h, -1)[0]
    lib = fvlbm.load()
    vp = C.c_void_p
    if f32_io:
        host_f = [torch.empty((total, 9), dtype=torch.float32, pin_memory=True).numpy() for _ in range(2)]
        for hf in host_f:
            if lib.fvlbm_get_fdev_f32(solver.h, -1, hf.ctypes.data_as(vp)):
                raise RuntimeError("fvlbm_get_fdev_f32 failed")
    else:
        host_f = [torch.empty((total, 9), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        for hf in host_f:
            hf[:] = fvlbm.fvlbm_get_f(solver.h, -1)
    u = [torch.empty(total, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    v = [torch.empty(total, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    k = args.steps  # the same step count as the device-timed region

    def check(rc, what):
        if rc:
            raise fvlbm.FvlbmError(rc, what)

    def one_step(j):
        b = j % 2
        if pipelined:
            if f32_io:
                check(lib.fvlbm_set_fdev_f32_async(solver.h, -1, host_f[b].ctypes.data_as(vp)),
                      "fvlbm_set_fdev_f32_async")
            else:
                check(lib.fvlbm_set_f_async(solver.h, -1, host_f[b].ctypes.data_as(vp)), "fvlbm_set_f_async")
            solver.step(1)
            check(lib.fvlbm_get_fields_async(solver.h, -1, None, u[b].ctypes.data_as(vp),
                                             v[b].ctypes.data_as(vp), None, None, None),
                  "fvlbm_get_fields_async")
        else:
            check(lib.fvlbm_set_f(solver.h, -1, host_f[b].ctypes.data_as(vp)), "fvlbm_set_f")
            solver.step(1)
            check(lib.fvlbm_get_fields(solver.h, -1, None, u[b].ctypes.data_as(vp),
                                       v[b].ctypes.data_as(vp), None, None, None), "fvlbm_get_fields")
    with torch.cuda.stream(stream):
        one_step(0)
        one_step(1)  # both staging slots sized before the timed region
        check(lib.fvlbm_wait(solver.h), "fvlbm_wait")
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for j in range(k):
            one_step(j)
        check(lib.fvlbm_wait(solver.h), "fvlbm_wait")
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
    total_job = cells_job
    if world > 1:
        el = max_over_ranks(torch, dist, world, el, device="cuda")
    io = "pipelined (async calls, copy engines)" if pipelined else "synchronous calls"
    io += "; state uploaded as FP32 deviations f - w rho0" if f32_io else "; state uploaded as FP64 f"
    return {"value": total_job / (el / k) / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": int(total * 9 * (4 if f32_io else 8)),
            "d2h_bytes_per_step": int(total * 2 * 8),
            "steps": k, "ms_per_step": el / k * 1e3, "io": io}


def run_profile_mode(args):
    """Minimal run for ncu: one solver, warmup + steps, nothing else (launch list / capture)."""
    import torch
    from paper_1812_00394_gb300 import fvlbm
    torch.cuda.set_device(0)
    cases = make_workload(args.workload)
    prec = fvlbm.FVLBM_FP32_DEV if args.precision == "fp32" else fvlbm.FVLBM_FP64
    s = fvlbm.Solver(cases, precision=prec, device=0, kernel_path=args.kernel_path)
    s.step(args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(args.steps)
    st = s.step(0, stats=False)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    nbytes, lps = s.footprint()
    print(json.dumps({"mode": "profile", "workload": args.workload, "precision": args.precision,
                      "kernel_path": args.kernel_path, "device_bytes": nbytes,
                      "cells": sum(c.mesh.n_cells for c in cases), "launches_per_step": lps,
                      "warmup": args.warmup, "steps": args.steps, "wall_s": el, "st": st}))
    s.close()
    return 0


def run_adjoint_mode(args):
    """Cost of the discrete adjoint (fvlbm_adjoint, FP64) against the FP64 primal step it
    differentiates, on the NACA 0012 C-mesh (k-omega SST, Re_c = 6e6, alpha = 4 degrees, or
    laminar at Re_c = 2000) or a 256 x 256 lid-driven cavity.  Per-step costs are marginal: (time at 3S steps - time at S steps) / 2S, so
    allocation and set-up drop out.  Not a bench line of the step; prints one JSON object."""
    import dataclasses
    import torch
    from paper_1812_00394_gb300 import fvlbm, meshgen as mg
    torch.cuda.set_device(0)
    if args.adjoint_case == "naca_sst":
        case = mg.naca0012_cmesh(n_target=args.adjoint_cells, alpha_deg=4.0)
    elif args.adjoint_case == "naca_laminar":
        case = dataclasses.replace(mg.naca0012_cmesh(n_target=args.adjoint_cells, re_c=2000.0,
                                                     alpha_deg=4.0), sst=False)
    else:
        case = mg.cavity_quad(256, re=1000.0)
    s = fvlbm.Solver(case, precision=fvlbm.FVLBM_FP64, device=0, kernel_path=1)
    s.step(args.warmup)
    s.adjoint(2, 1.0, 0.0)
    n1 = max(1, args.steps)
    t = {}
    for n in (n1, 3 * n1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(n)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s.adjoint(n, 1.0, 0.0)
        t2 = time.perf_counter()
        s.adjoint(n, 1.0, 0.0, shape=True)
        t3 = time.perf_counter()
        t[n] = (t1 - t0, t2 - t1, t3 - t2)
    d = 2 * n1
    fwd, adj, shp = ((t[3 * n1][q] - t[n1][q]) / d * 1e3 for q in range(3))
    print(json.dumps({"mode": "adjoint", "case": args.adjoint_case, "cells": case.mesh.n_cells,
                      "steps": [n1, 3 * n1], "fwd_fp64_ms_per_step": fwd,
                      "adjoint_ms_per_step": adj, "adjoint_with_shape_ms_per_step": shp,
                      "adjoint_over_fwd": adj / fwd,
                      "shape_setup_s": t[n1][2] - n1 * shp / 1e3}))
    s.close()
    return 0


def run_config_mode(args):
    """The per-configuration runs (not bench lines; one JSON object per run): the 64 x 64
    cavity in FP64 over its 2,000 steps against the oracle; the 40k-triangle Delaunay cavity at
    dt = 5 tau and 50 tau in FP32 and FP64 until the residual falls below 1e-8 (at most 20,000
    steps), with the residual every 1,000 steps; the backward-facing step and a NACA 0012
    C-mesh (k-omega SST) in FP32 against FP64 after the same steps.  Time per step from the
    wall clock around graph-replayed steps (synchronised)."""
    import torch
    from paper_1812_00394_gb300 import fvlbm, meshgen as mg
    torch.cuda.set_device(0)
    FP32, FP64 = fvlbm.FVLBM_FP32_DEV, fvlbm.FVLBM_FP64

    def vel(fl):
        return np.concatenate([fl["u"], fl["v"]])

    def run(case, prec, steps, every, tol=0.0):
        s = fvlbm.Solver(case, precision=prec, device=0)
        tuned = s.autotune(3)[0]
        hist, done, el = [], 0, 0.0
        while done < steps:
            n = min(every, steps - done)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = s.step(n, stats=True)
            el += time.perf_counter() - t0
            done += n
            hist.append([done, st["residual"]])
            if st["diverged"] or (tol > 0 and st["residual"] < tol):
                break
        out = {"steps": done, "ms_per_step": el / done * 1e3, "residual": hist[-1][1],
               "residual_every": hist, "diverged": int(st["diverged"]), "config": tuned}
        return s, out

    res = []
    # configs[0]: 64 x 64 quad cavity, Re 400, FP64, 2,000 steps, against the oracle
    from oracle import oracle as orc
    from oracle.oracle import Oracle
    orc.set_threads(host_cores())
    c0 = mg.cavity_quad(64, re=400.0, seed=1)
    s, out = run(c0, FP64, 2000, 500)
    o = Oracle(c0)
    o.step(2000)
    fo, fg = o.get_f(), s.get_f()
    out.update(name="cavity64_re400_fp64", cells=c0.mesh.n_cells,
               fp64_vs_oracle_f_rel_max=float(np.abs(fg - fo).max() / np.abs(fo).max()),
               oracle_residual=o.residual())
    s.close()
    res.append(out)
    # configs[1]: 40k Delaunay cavity, Re 1000, dt = 5 tau and 50 tau, to residual 1e-8
    for z in (5.0, 50.0):
        case = mg.cavity_delaunay(re=1000.0, z=z, seed=2)
        runs = {}
        for prec, tag in ((FP32, "fp32"), (FP64, "fp64")):
            s, out = run(case, prec, args.converge_steps, 1000, tol=1e-8)
            runs[tag] = (s, out)
        a, b = runs["fp32"][0].fields(), runs["fp64"][0].fields()
        same = runs["fp32"][1]["steps"] == runs["fp64"][1]["steps"]
        import dataclasses
        dt_cfl1 = fvlbm.check_case(dataclasses.replace(case, dt=0.0, cfl=1.0))[1]
        for tag in ("fp32", "fp64"):
            out = runs[tag][1]
            out.update(name=f"delaunay_re1000_z{z:g}_{tag}", cells=case.mesh.n_cells,
                       dt_over_tau=z, dt=runs[tag][0].dt(), convective_cfl=runs[tag][0].dt() / dt_cfl1)
            if same:
                out["fp32_vs_fp64_velocity_rel_l2"] = float(np.linalg.norm(vel(a) - vel(b)) /
                                                            np.linalg.norm(vel(b)))
            res.append(out)
            runs[tag][0].close()
    # configs[2], configs[3]: SST backward-facing step and NACA 0012 C-mesh, FP32 vs FP64
    for case, name in ((mg.bfs_hybrid(n_target=80000), "bfs80k_sst"),
                       (mg.naca0012_cmesh(n_target=200000, alpha_deg=4.0), "naca200k_sst_a4")):
        s32, o32 = run(case, FP32, args.sst_steps, 1000)
        s64, o64 = run(case, FP64, args.sst_steps, 1000)
        f32, f64 = s32.fields(), s64.fields()
        fr32, fr64 = s32.forces(), s64.forces()
        o32.update(name=name + "_fp32", cells=case.mesh.n_cells,
                   fp32_vs_fp64_velocity_rel_l2=float(np.linalg.norm(vel(f32) - vel(f64)) /
                                                      np.linalg.norm(vel(f64))),
                   fp32_vs_fp64_nut_rel_l2=float(np.linalg.norm(f32["nut"] - f64["nut"]) /
                                                 np.linalg.norm(f64["nut"])),
                   fp32_vs_fp64_cd_rel=abs(fr32["cd"] - fr64["cd"]) / abs(fr64["cd"]),
                   fp32_vs_fp64_cl_rel=abs(fr32["cl"] - fr64["cl"]) / max(abs(fr64["cl"]), 1e-30),
                   fp64_ms_per_step=o64["ms_per_step"])
        res.append(o32)
        s32.close()
        s64.close()
    for r in res:
        print(json.dumps(r), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "sweep_small", "delaunay40k", "cavity64"])
    ap.add_argument("--check-steps", type=int, default=5)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds the reference arm's steps may take; it samples fewer instances "
                         "to stay within it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config-mode", action="store_true",
                    help="the per-configuration runs (cavity 64 against the oracle, the Delaunay "
                         "cavity to residual 1e-8, the SST cases FP32 vs FP64); not a bench line")
    ap.add_argument("--converge-steps", type=int, default=300000)
    ap.add_argument("--sst-steps", type=int, default=2000)
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--profile-mode", action="store_true",
                    help="only build the workload and run warmup + steps (for ncu)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--kernel-path", type=int, default=0, choices=[0, 1, 2],
                    help="profile mode: 0 fused stage kernels, 1 two-pass kernels, 2 fused "
                         "stage kernels in the face-value form")
    ap.add_argument("--adjoint-mode", action="store_true",
                    help="time the FP64 laminar adjoint against its primal step (not a bench line)")
    ap.add_argument("--adjoint-case", default="naca_laminar",
                    choices=["naca_laminar", "naca_sst", "cavity256"])
    ap.add_argument("--adjoint-cells", type=int, default=200000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_mode:
        return run_profile_mode(args)
    if args.config_mode:
        return run_config_mode(args)
    if args.adjoint_mode:
        return run_adjoint_mode(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
