#!/usr/bin/env python
"""Benchmark of the WCSPH particle-interaction pass on GB300.

Metric: particle-steps/s (fluid + boundary particles x steps / s), one step
being the whole pass: pair interaction (Eqs. 3-8), adaptive dt (Eq. 15),
Verlet update with rebinning (Eqs. 9-14), neighbour structure and sorted
gather.

Headline `value`: the mixed FP32/FP64 form on the largest single-GPU workload,
the wall-impact dam break at dp = 0.0025 m (1.6 x 0.6 x 0.6 m tank, 0.6 x 0.6 x
0.3 m column, about 8.1 M particles).  Also reported: the FP64 form on the same
case, the 0.9 M-particle obstacle case at dp = 0.01 m in both forms (with the
FP64 pair kernel's roofline), the symplectic integrator, the paper's own
parameters at its Case 1 resolution, the gate-released dam break, the batched
alpha sweep (64 instances in one set of launches) against the same instances
run one after another, the measured FP32 and FP64 FMA peaks that the rooflines
use, the end-to-end rate through the C ABI with host buffers, and the FP64 CPU
oracle timed on this host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one rank per GPU) every rank advances its own replica of
the case and its own shard of the sweep: weak scaling, no collective on the
data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "WCSPH particle-steps/s: mixed FP32 vs FP64 on one GB300; batched α-sweep speedup"
UNIT = "particle-steps/s"

# Algorithmic work of one evaluated pair (Eqs. 3-7 with Eq. 5's c_i and the
# Eq. 15 maximum): 80 flop, the per-pair figure of the method's operation count
# (relative position and velocity 6, |r|^2 5, |r| 2, kernel gradient 6,
# u . r 5, continuity 4, delta term 6, pressure term 5, viscosity about 20,
# scaling 3, accumulation 6, plus the densities' reciprocals and the running
# maximum).  It is the same for both forms and does not shrink when a kernel
# folds constants.  The mixed kernel's own instruction-level count (FMA = 2,
# other FP32 operations 1) is reported beside it: 42 per evaluated pair, +4 for
# a fluid-fluid pair (delta term), +12 for an approaching pair (viscosity).
FLOPS_PER_PAIR = 80
FLOPS_PAIR_BASE, FLOPS_PAIR_DELTA, FLOPS_PAIR_VISC = 42, 4, 12
L2_FLUSH_BYTES = 256 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="wall_impact_dp0.0025")
    ap.add_argument("--second", default="dambreak_obstacle_dp0.01",
                    help="second workload, timed in both forms (with the FP64 pair kernel's roofline)")
    ap.add_argument("--skip", default="",
                    help="comma list of: fp64,second,symplectic,paper,gate,lists,batch,mps,cpu,e2e,profile,peak")
    ap.add_argument("--series", type=float, default=0.0,
                    help="instead of timing: run the workload (mixed form, adaptive dt) for this many seconds of "
                         "physical time and print its probe series every --every seconds")
    ap.add_argument("--every", type=float, default=0.05)
    ap.add_argument("--pair-passes", type=int, default=0,
                    help="instead of timing: run this many pair passes (sph_derivatives seam, no update) of the "
                         "workload in --precision, the launch an ncu capture of the pair kernel selects")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--list-skin", type=float, default=0.0,
                    help="with --pair-passes: mixed form with neighbour lists of skin s = LIST_SKIN h")
    ap.add_argument("--accuracy-dir", default="",
                    help="with --accuracy: write each probe series there as soon as it is complete")
    ap.add_argument("--accuracy-from", default="",
                    help="compare the probe series that --accuracy-dir wrote (no GPU)")
    ap.add_argument("--pair-symmetric", action="store_true",
                    help="with --pair-passes --precision fp64 or --accuracy: the FP64 form evaluates each pair once")
    ap.add_argument("--accuracy", type=float, default=0.0,
                    help="instead of timing: run both forms for this many seconds of physical time and "
                         "report the mixed form's probe errors against the FP64 form")
    return ap.parse_args(argv)


# ---------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(backend):
    import torch.distributed as dist

    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank, world):
    """Contiguous, near-equal shard of a list for one rank."""
    n = len(items)
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return items[lo:hi]


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, f in enumerate(flags) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- our arm
def timed_steps(sim, steps, flush_buf, torch):
    """K single steps, each after an L2 flush, timed with CUDA events on the
    library's stream; returns the summed device time in seconds."""
    stream = sim.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush_buf.zero_()
        ev[k][0].record(stream)
        sim.step(0.0, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / 1e3


def cpu_baseline_sample(case, second, steps=2):
    """The FP64 oracle as it stands: full steps of the whole case on all host
    cores, and one full step of the second (smaller) case on one thread."""
    import oracle

    cores = oracle.set_threads(os.cpu_count() or 1)
    oc = oracle.make_case(case.tank, case.column, case.obstacle, dp=case.dp, h=case.h, c0=case.c0,
                          rho0=case.rho0, alpha=case.alpha)
    st = oracle.scene(oc)
    t0 = time.perf_counter()
    oracle.run(oc, st, steps)
    dt = time.perf_counter() - t0
    n = st.n
    del st
    o2 = oracle.make_case(second.tank, second.column, second.obstacle, dp=second.dp, h=second.h, c0=second.c0,
                          rho0=second.rho0, alpha=second.alpha)
    s2 = oracle.scene(o2)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.run(o2, s2, 1)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full FP64 oracle steps of the {case.name} case ({n} particles), "
                      f"adaptive dt, OpenMP gather over particles",
            "single_thread": {"value": s2.n / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"1 full step of the {second.name} case ({s2.n} particles) on one thread"}}


def hbm_peak_gbs():
    """The measured copy bandwidth of the GB300s (MEASURED_PEAKS.json,
    written by the machine's setup), or None."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def measured_peaks(sph, torch, local):
    """FP32 and FP64 FMA throughput measured on this GPU (sph_alu_peak), with
    the SM clock sampled while they run."""
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream().cuda_stream
    f32 = sph.alu_peak(sph.MIXED, 150, stream)
    f64 = sph.alu_peak(sph.FP64, 150, stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    return {"fp32_tflops": round(f32 / 1e12, 3), "fp64_tflops": round(f64 / 1e12, 3),
            "how": "sph_alu_peak: independent FMA chains (FP32: best of scalar and packed FP32x2) on every SM, "
                   "FMA = 2 flop, fastest of 3 launches of about 150 ms",
            "clocks": clk}


def pair_roofline(sim, precision, peak_tflops, kernel, traffic):
    """Roofline of the pair kernel on the handle's current state: algorithmic
    flop per launch (FLOPS_PER_PAIR x evaluated pairs) over the mean launch time
    of 50 profiled steps (CUDA events on the library's stream)."""
    sim.set_profiling(True)
    sim.step(0.0, 50)
    phases = sim.phase_times()
    sim.set_profiling(False)
    stats = sim.pair_stats()
    pair_ms, pair_n = phases["pair"]
    pair_s = pair_ms / 1e3 / max(pair_n, 1)
    flops = FLOPS_PER_PAIR * stats["evaluated"]
    achieved = flops / pair_s / 1e12
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak_tflops, 4), "traffic": traffic, "kernel": kernel,
            "pair_launch_ms": round(pair_s * 1e3, 4),
            "peak_source": ("measured FP32" if precision == 1 else "measured FP64")
                           + " FMA throughput (sph_alu_peak, this run)",
            "flops_per_launch": flops, "flops_per_pair": FLOPS_PER_PAIR, "pairs_per_launch": stats["evaluated"]}
    if precision == 1:
        src = (FLOPS_PAIR_BASE * stats["evaluated"] + FLOPS_PAIR_DELTA * stats["fluid_fluid"]
               + FLOPS_PAIR_VISC * stats["approaching"])
        roof["source_counted"] = {"flops_per_launch": src, "tflops": round(src / pair_s / 1e12, 3),
                                  "frac": round(src / pair_s / 1e12 / peak_tflops, 4)}
    phase = {k: round(v[0] / max(v[1], 1), 4) for k, v in phases.items()}
    return roof, phase, stats


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    dist_init("nccl" if world > 1 else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2306_01959_gb300 import sph, workloads as wl

    skip = set(filter(None, args.skip.split(",")))
    case = wl.by_name(args.workload)
    second = wl.by_name(args.second)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    peaks = None if "peak" in skip else measured_peaks(sph, torch, local)
    peak32 = peaks["fp32_tflops"] if peaks else float("nan")
    peak64 = peaks["fp64_tflops"] if peaks else float("nan")

    # ---- mixed form on the headline workload
    sim = sph.Simulation(case, precision=sph.MIXED, use_graph=1, graph_steps=1)
    best_shape = sim.autotune(2)
    npart = sim.n
    sim.step(0.0, args.warmup)
    sim.sync()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    torch.cuda.profiler.start()  # brackets the timed region for an external profiler (no-op otherwise)
    dev_s = timed_steps(sim, args.steps, flush, torch)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    sim.sync()
    dev_s = max_over_ranks(dev_s)
    total_particles = sum_over_ranks(npart)
    value = total_particles * args.steps / dev_s
    launches = sim.launches_per_step() * args.steps

    # steady state without flushes, multi-step graphs (context)
    sim16 = sph.Simulation(case, precision=sph.MIXED, use_graph=1, graph_steps=16,
                           pair_warps=int(best_shape[0]), pair_ctas_per_sm=int(best_shape[1]),
                           pair_group=int(best_shape[2]))
    sim16.step(0.0, 32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim16.stream)
    sim16.step(0.0, 256)
    e1.record(sim16.stream)
    torch.cuda.synchronize()
    steady_ms = e0.elapsed_time(e1) / 256
    sim16.close()

    roof = phases = stats = None
    if "profile" not in skip:
        roof, phases, stats = pair_roofline(sim, sph.MIXED, peak32, "k_pair_mixed",
                                            recorded_traffic("pair_mixed", case.name))

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if "e2e" not in skip:
        pts = torch.tensor(case.pressure_xyz, dtype=torch.float64).pin_memory().numpy()
        xy = torch.tensor(case.wave_xy, dtype=torch.float64).pin_memory().numpy()
        ke = max(20, min(200, args.steps // 5))
        sim.step(0.0, 2)
        sim.sync()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            sim.step(0.0, 1)
            sim.probe_pressure(pts)
            sim.probe_wave_height(xy)
            if case.obstacle is not None:
                sim.probe_force()
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": total_particles * ke / te, "unit": UNIT,
               "h2d_bytes_per_step": int(8 + pts.nbytes + xy.nbytes),
               "d2h_bytes_per_step": int(8 * (len(pts) + len(xy)) + (24 if case.obstacle is not None else 0)),
               "steps": ke, "calls": "sph_step(dt=0, 1) + pressure and wave-height probes per step"
                                     + (" + force probe" if case.obstacle is not None else "")}
    sim.close()

    # ---- FP64 form on the headline workload
    fp64 = None
    if "fp64" not in skip:
        sim64 = sph.Simulation(case, precision=sph.FP64, use_graph=1, graph_steps=1)
        sim64.step(0.0, 2)
        sim64.sync()
        k64 = max(3, min(10, args.steps // 100))
        s64 = max_over_ranks(timed_steps(sim64, k64, flush, torch))
        fp64 = {"workload": case.name, "value": sum_over_ranks(sim64.n) * k64 / s64,
                "ms_per_step": round(s64 / k64 * 1e3, 3), "steps": k64}
        sim64.close()
        # each pair once, partners' shares by FP64 atomics (opt-in: run-to-run
        # differences in the last bits)
        sims64 = sph.Simulation(case, precision=sph.FP64, use_graph=1, graph_steps=1, pair_symmetric=1)
        sims64.step(0.0, 2)
        sims64.sync()
        ss64 = max_over_ranks(timed_steps(sims64, k64, flush, torch))
        fp64["symmetric"] = {"value": sum_over_ranks(sims64.n) * k64 / ss64,
                             "ms_per_step": round(ss64 / k64 * 1e3, 3), "steps": k64}
        sims64.close()

    # ---- second workload (0.9 M particles) in both forms, FP64 pair roofline
    sec = None
    if "second" not in skip:
        sec = {"workload": second.name}
        for name, prec, kw in (("mixed", sph.MIXED, {}), ("fp64", sph.FP64, {}),
                               ("fp64_symmetric", sph.FP64, {"pair_symmetric": 1})):
            s2 = sph.Simulation(second, precision=prec, use_graph=1, graph_steps=1, **kw)
            shp = s2.autotune(2) if prec == sph.MIXED else None
            s2.step(0.0, 3)
            s2.sync()
            k2 = max(3, min(100 if prec == sph.MIXED else 20, args.steps // 10))
            t2 = max_over_ranks(timed_steps(s2, k2, flush, torch))
            entry = {"particles": int(s2.n), "value": sum_over_ranks(s2.n) * k2 / t2,
                     "ms_per_step": round(t2 / k2 * 1e3, 4), "steps": k2}
            if shp:
                entry["pair_launch_shape"] = list(shp)
            if "profile" not in skip:
                r2, ph2, _ = pair_roofline(s2, prec, peak32 if prec == sph.MIXED else peak64,
                                           "k_pair_mixed" if prec == sph.MIXED else "k_pair_fp64",
                                           None if kw else
                                           recorded_traffic("pair_mixed" if prec == sph.MIXED else "pair_fp64",
                                                            second.name))
                if kw:
                    r2["note"] = ("pairs counted once each (the pass evaluates every interacting pair once and "
                                  "hands the partner its share); the ordered passes count both orders")
                entry["roofline"] = r2
                entry["phase_ms_per_step"] = ph2
            sec[name] = entry
            s2.close()
        sec["speedup_mixed_vs_fp64"] = round(sec["mixed"]["value"] / sec["fp64"]["value"], 2)
        sec["speedup_fp64_symmetric_vs_fp64"] = round(sec["fp64_symmetric"]["value"] / sec["fp64"]["value"], 2)

    # ---- symplectic predictor-corrector (two pair passes per step), mixed form
    sym = None
    if "symplectic" not in skip:
        sims = sph.Simulation(case, precision=sph.MIXED, integrator=sph.SYMPLECTIC, use_graph=1, graph_steps=1,
                              pair_warps=int(best_shape[0]), pair_ctas_per_sm=int(best_shape[1]),
                              pair_group=int(best_shape[2]))
        sims.step(0.0, 3)
        sims.sync()
        ks = max(10, min(50, args.steps // 5))
        ss = max_over_ranks(timed_steps(sims, ks, flush, torch))
        sym = {"workload": case.name, "value": sum_over_ranks(sims.n) * ks / ss,
               "ms_per_step": round(ss / ks * 1e3, 4), "steps": ks, "pair_passes_per_step": 2,
               "launches_per_step": sims.launches_per_step()}
        sims.close()

    # ---- the paper's own parameters (h = 1.5 dp, c0 = 20 sqrt(g H_W)) at its
    # Case 1 resolution, for a like-for-like line beside its K40m timing
    paper = None
    if "paper" not in skip:
        pc = wl.paper_case1()
        simp = sph.Simulation(pc, precision=sph.MIXED, use_graph=1, graph_steps=1)
        shp = simp.autotune(2)
        simp.step(0.0, 3)
        simp.sync()
        kp = max(10, min(100, args.steps // 5))
        sp = max_over_ranks(timed_steps(simp, kp, flush, torch))
        paper = {"workload": pc.name, "particles": int(simp.n), "h_over_dp": 1.5, "c0": round(pc.c0, 4),
                 "value": sum_over_ranks(simp.n) * kp / sp, "ms_per_step": round(sp / kp * 1e3, 4), "steps": kp,
                 "pair_launch_shape": list(shp),
                 "paper_k40m_context": {"value": 1.98e7, "unit": UNIT,
                                        "note": "whole DualSPHysics solver on a Tesla K40m, Table 1, derived"}}
        simp.close()

    # ---- the gate-released dam break (Case 2 shapes), mixed form
    gate = None
    if "gate" not in skip:
        gc = wl.gate_dambreak()
        simg = sph.Simulation(gc, precision=sph.MIXED, use_graph=1, graph_steps=1)
        shg = simg.autotune(2)
        simg.step(0.0, 3)
        simg.sync()
        kg = max(10, min(100, args.steps // 5))
        sg = max_over_ranks(timed_steps(simg, kg, flush, torch))
        gate = {"workload": gc.name, "particles": int(simg.n), "gate_speed": gc.gate_velocity[2],
                "value": sum_over_ranks(simg.n) * kg / sg, "ms_per_step": round(sg / kg * 1e3, 4), "steps": kg,
                "pair_launch_shape": list(shg)}
        simg.close()

    # ---- neighbour lists with a skin (opt-in) on the headline workload, against
    # the per-step sweep timed above
    lists = None
    if "lists" not in skip:
        lists = {"workload": case.name}
        for skin in (0.15, 0.3):
            siml = sph.Simulation(case, precision=sph.MIXED, use_graph=1, graph_steps=1, list_skin=skin)
            siml.step(0.0, 3)
            siml.sync()
            siml.list_stats()
            kl = max(10, min(60, args.steps // 5))
            sl_ = max_over_ranks(timed_steps(siml, kl, flush, torch))
            lists[f"skin_{skin}h"] = {"value": sum_over_ranks(siml.n) * kl / sl_,
                                      "ms_per_step": round(sl_ / kl * 1e3, 4), "steps": kl,
                                      "list_stats": siml.list_stats()}
            siml.close()

    # ---- batched alpha sweep vs the same instances one after another
    batch = None
    if "batch" not in skip:
        batch = run_batch(args, sph, wl, torch, rank, world)

    # ---- the MPS step (Section 2.3) on the paper's Case 1 tank shape
    mps_line = None
    if "mps" not in skip:
        mps_line = run_mps(args, wl, torch, hbm_peak_gbs())

    cpu = None
    if rank == 0 and world == 1 and "cpu" not in skip:
        cpu = cpu_baseline_sample(case, second)

    if rank == 0:
        cnt = sph.Simulation(case, precision=sph.MIXED).counts()
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dev_s / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": case.name, "particles": int(npart), "fluid": int(cnt[0]),
                       "boundary": int(cnt[1] + cnt[2]), "precision": "mixed FP32 pair / FP64 position+dt",
                       "dt": "adaptive (Eq. 15)", "integrator": "Verlet, first-order step every 40",
                       "l2": "256 MB L2 flush before every timed step (not timed)",
                       "launch": "one CUDA-graph launch per step", "parallelism": f"replicas x{world}",
                       "pair_launch_shape": list(best_shape)},
            "gpu_launches": launches, "wall_s_timed_region": round(t_wall, 3),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "measured_peaks": peaks,
            "fp64": fp64, "speedup_mixed_vs_fp64": round(value / fp64["value"], 2) if fp64 else None,
            "second_workload": sec, "symplectic": sym, "paper_parameters": paper, "gate_dambreak": gate,
            "batched_alpha_sweep": batch, "mps": mps_line, "neighbour_lists": lists,
            "steady_state_graph16_ms_per_step": round(steady_ms, 4),
            "phase_ms_per_step": phases, "pair_stats": stats,
        }
        print(json.dumps(line))


def run_batch(args, sph, wl, torch, rank, world):
    """The 64-instance alpha sweep for its 1,000 steps: one handle for all
    instances in one persistent launch, the same handle with per-phase launches
    replayed from CUDA graphs, and the 64 instances as handles run one after
    another (per-phase launches from graphs)."""
    cases = shard(wl.alpha_sweep(64, seed=2306), rank, world)
    kb = 1000
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    simp = sph.Simulation(cases, precision=sph.MIXED, batch=True, persistent=1)
    simp.step(0.0, 10)
    simp.sync()
    e0.record(simp.stream)
    simp.step(0.0, kb)
    e1.record(simp.stream)
    torch.cuda.synchronize()
    simp.sync()
    tp = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    simp.close()
    simb = sph.Simulation(cases, precision=sph.MIXED, batch=True, use_graph=1, graph_steps=10)
    simb.step(0.0, 10)
    simb.sync()
    e0.record(simb.stream)
    simb.step(0.0, kb)
    e1.record(simb.stream)
    torch.cuda.synchronize()
    tb = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    nb = simb.n
    simb.close()
    singles = [sph.Simulation(c, precision=sph.MIXED, use_graph=1, graph_steps=10) for c in cases]
    for s in singles:
        s.step(0.0, 10)
    torch.cuda.synchronize()
    e0.record(singles[0].stream)
    for s in singles:
        s.step(0.0, kb)
    e1.record(singles[0].stream)
    torch.cuda.synchronize()
    ts = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    for s in singles:
        s.close()
    return {"instances": 64, "particles": int(sum_over_ranks(nb)), "steps": kb,
            "value": sum_over_ranks(nb) * kb / tp, "launches": "one persistent cooperative launch for all steps",
            "per_phase_graph_value": sum_over_ranks(nb) * kb / tb,
            "sequential_value": sum_over_ranks(nb) * kb / ts, "speedup": round(ts / tp, 3),
            "speedup_per_phase_graph": round(ts / tb, 3)}


def run_mps(args, wl, torch, peak_hbm=None):
    """The MPS step (prediction, number density, free surface, Eq. 23 assembled
    and solved by CG to 1e-6, gradient, correction) on the paper's Case 1 tank
    shape at l0 = 0.0075 m with its fixed dt of 3e-4 s, timed over steps that
    each wait for their solve."""
    from paper_2306_01959_gb300 import mps

    c = wl.mps_case1()
    tank = mps.Tank(c.tank, c.column, c.dp, wl.MPS_CASE1_DT)
    tank.step(3)
    km = max(5, min(20, args.steps // 10))
    its = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(tank.stream)
    for _ in range(km):
        tank.step(1)
        its.append(tank.last_solve()[0])
    e1.record(tank.stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev = e0.elapsed_time(e1) / 1e3
    tank.set_profiling(True)
    its3 = 0
    for _ in range(3):
        tank.step(1)
        its3 += tank.last_solve()[0]
    phases = {k: round(v / 3, 3) for k, v in tank.phase_times().items()}
    tank.set_profiling(False)
    rows, nnz = tank.system_size()
    n = tank.n
    tank.close()
    # CG iteration against the HBM roofline: the stored entries (8 B value + 4 B
    # column) and per row the entry count (4 B) and twelve 8-byte vector
    # accesses (SpMV: diag, p, q; update: x, r read and written, p, q; new
    # direction: r, p read and written); the gathers of p count once (p is held
    # in L2)
    cg_roof = None
    if peak_hbm and its3 > 0:
        per_it = 12 * nnz + rows * (4 + 12 * 8)
        t_it = phases["cg"] / 1e3 / (its3 / 3)
        cg_roof = {"bound": "hbm", "achieved": round(per_it / t_it / 1e9, 1), "peak": peak_hbm, "unit": "GB/s",
                   "frac": round(per_it / t_it / 1e9 / peak_hbm, 4), "traffic": None,
                   "bytes_per_iteration": int(per_it), "rows": rows, "stored_entries": nnz,
                   "ms_per_iteration": round(t_it * 1e3, 4),
                   "note": "CG iteration (SpMV, two dot products, updates; five launches) timed by phase events"}
    return {"workload": c.name, "particles": int(n), "fluid": int(tank.counts[0]), "dt": wl.MPS_CASE1_DT,
            "value": n * km / dev, "unit": UNIT, "ms_per_step": round(dev / km * 1e3, 3), "steps": km,
            "wall_value": n * km / wall, "cg_iterations_per_step": round(float(np.mean(its)), 1),
            "phase_ms_per_step": phases, "cg_roofline": cg_roof,
            "cg_tol": 1e-6, "paper_mps_cpu_context": {"value": 2.0e5, "unit": UNIT,
                                                      "note": "the paper's in-house MPS on 20 Xeon cores, Table 1"}}


def recorded_traffic(kernel, workload):
    """DRAM bytes per pair launch from the committed ncu summary of that
    kernel on that workload, or None when the kernel's source changed since the
    counters were taken."""
    import hashlib

    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    m = hashlib.sha256()
    for ext in (".cu", ".cuh"):  # the kernel's launcher and, where it has one, its body
        src = os.path.join(ROOT, "paper_2306_01959_gb300", "csrc", kernel + ext)
        if os.path.exists(src):
            m.update(open(src, "rb").read())
    h = m.hexdigest()[:16]
    ent = rec.get(workload)
    if not ent or ent.get("source_sha256_16") != h:
        return None
    return ent.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle as it stands, on the host cores: full oracle steps
    (neighbour structure, Eqs. 3-8, Eq. 15, Eqs. 9-14) of the same workload.
    When K full steps would not end within about two minutes, fewer are timed
    (at least 2) and the rate is over those; the warm-up is one step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2306_01959_gb300 import workloads as wl

    case = wl.by_name(args.workload)
    cores = oracle.set_threads(os.cpu_count() or 1)
    oc = oracle.make_case(case.tank, case.column, case.obstacle, dp=case.dp, h=case.h, c0=case.c0,
                          rho0=case.rho0, alpha=case.alpha)
    st = oracle.scene(oc)
    t0 = time.perf_counter()
    oracle.run(oc, st, 1)  # warm-up step, also the estimate of one step's time
    t_one = time.perf_counter() - t0
    budget_s = 120.0
    k = max(2, min(args.steps, int(budget_s / max(t_one, 1e-9))))
    t0 = time.perf_counter()
    oracle.run(oc, st, k)
    dt = time.perf_counter() - t0
    value = st.n * k / dt
    desc = (f"{k} full FP64 oracle steps of the {case.name} case ({st.n} particles) after one warm-up step, "
            f"adaptive dt, OpenMP gather over particles")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "steps_timed": k, "warmup": args.warmup, "ms_per_step": round(dt / k * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case.name, "particles": int(st.n)},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def accuracy_errors(series, workload, physical_time):
    """Mixed vs FP64 and the control, per time window, from the probe series
    (dicts name -> rows of (t, wave heights, pressures)) that are present."""
    from paper_2306_01959_gb300 import workloads as wl

    case = wl.by_name(workload)
    hc = case.column[2]
    pref = 1000.0 * 9.81 * hc

    def errs(a, b, upto):
        n = min(len(a), len(b))
        idx = [i for i in range(n) if a[i][0] <= upto + 1e-9]
        if not idx:
            return None
        w = max(float(np.max(np.abs(np.asarray(a[i][1]) - np.asarray(b[i][1])))) for i in idx) / hc
        p = max(float(np.max(np.abs(np.asarray(a[i][2]) - np.asarray(b[i][2])))) for i in idx) / pref
        return {"wave_over_Hc": round(w, 5), "pressure_over_rho0_g_Hc": round(p, 5)}

    windows = [round(0.1 * k, 1) for k in range(1, int(round(physical_time * 10)) + 1)]
    out = {"workload": workload, "physical_time_s": physical_time,
           "series": {k: {"samples": len(v), "t_end": round(float(v[-1][0]), 5) if v else None}
                      for k, v in series.items()}}
    if "fp64" in series and "mixed" in series:
        out["mixed_vs_fp64"] = {str(t): errs(series["mixed"], series["fp64"], t) for t in windows}
    if "mixed_nudged" in series and "mixed" in series:
        out["mixed_vs_mixed_nudged_1nm"] = {str(t): errs(series["mixed_nudged"], series["mixed"], t) for t in windows}
    return out


def run_accuracy(args):
    """Mixed vs FP64 on the same case: probe series every 0.01 s of physical
    time; errors reported per time window.  Control: the mixed form against
    itself with one fluid particle moved by 1 nm, which shows how fast any
    rounding-level difference is amplified by the flow itself.  With
    --accuracy-dir each series is written there as soon as it is complete
    (mixed, then FP64, then the control), so that a run cut short keeps what
    it finished; --accuracy-from compares such files without a GPU."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2306_01959_gb300 import sph, workloads as wl

    case = wl.by_name(args.workload)
    pts = np.array(case.pressure_xyz)
    xy = np.array(case.wave_xy)
    t0 = time.perf_counter()

    def series(prec, nudge=False):
        kw = {"pair_symmetric": 1} if (prec == sph.FP64 and args.pair_symmetric) else {}
        sim = sph.Simulation(case, precision=prec, **kw)
        if nudge:
            g = sim.get_state()
            g["r"][0, 0] += 1e-9
            sim.set_state(g["r"], g["u"], g["rho"], g["uprev"], g["rhoprev"], g["step"])
        rows = []
        while True:
            sim.step(0.0, 10)
            tcur = sim.time()[0]
            if tcur >= 0.01 * (len(rows) + 1):
                rows.append((float(tcur), sim.probe_wave_height(xy).tolist(), sim.probe_pressure(pts).tolist()))
                if tcur >= args.accuracy:
                    break
        sim.sync()
        nsteps = int(sim.get_state()["step"])
        sim.close()
        torch.cuda.synchronize()
        name = "fp64" if prec == sph.FP64 else ("mixed_nudged" if nudge else "mixed")
        info = {"series": name, "steps": nsteps, "t": round(rows[-1][0], 5),
                "wall_s": round(time.perf_counter() - t0, 1)}
        print(json.dumps(info), file=sys.stderr, flush=True)
        if args.accuracy_dir:
            os.makedirs(args.accuracy_dir, exist_ok=True)
            with open(os.path.join(args.accuracy_dir, f"accuracy_{case.name}_{name}.json"), "w") as f:
                json.dump({"workload": case.name, "physical_time_s": args.accuracy, "info": info,
                           "fp64_reference": ("each pair once (pair_symmetric)" if args.pair_symmetric
                                              else "each ordered pair") if prec == sph.FP64 else None,
                           "rows": rows}, f)
        return rows

    ser = {}
    ser["mixed"] = series(sph.MIXED)
    ser["fp64"] = series(sph.FP64)
    ser["mixed_nudged"] = series(sph.MIXED, nudge=True)
    out = accuracy_errors(ser, case.name, args.accuracy)
    out["fp64_reference"] = "each pair once (pair_symmetric)" if args.pair_symmetric else "each ordered pair"
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    print(json.dumps(out))


def run_accuracy_from(args):
    """The comparison of run_accuracy from the series files it wrote."""
    ser, wlname, ptime, ref = {}, None, None, None
    for name in ("mixed", "fp64", "mixed_nudged"):
        hits = [f for f in os.listdir(args.accuracy_from) if f.startswith("accuracy_") and f.endswith(f"_{name}.json")
                and (name != "mixed" or not f.endswith("_mixed_nudged.json"))]
        if not hits:
            continue
        d = json.load(open(os.path.join(args.accuracy_from, sorted(hits)[0])))
        ser[name] = d["rows"]
        wlname, ptime = d["workload"], d["physical_time_s"]
        ref = d.get("fp64_reference") or ref
    if not ser:
        raise SystemExit("no accuracy series in " + args.accuracy_from)
    out = accuracy_errors(ser, wlname, ptime)
    out["fp64_reference"] = ref
    print(json.dumps(out))


def run_series(args):
    """The workload advanced for args.series seconds of physical time (mixed
    form, adaptive dt, CUDA graphs of 16 steps): wave heights, Eq. 33 pressures,
    the obstacle force, mass and energies every args.every seconds."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2306_01959_gb300 import sph, workloads as wl

    case = wl.by_name(args.workload)
    pts = np.array(case.pressure_xyz)
    xy = np.array(case.wave_xy)
    sim = sph.Simulation(case, precision=sph.MIXED, use_graph=1, graph_steps=16)
    shape = sim.autotune(2)
    t0 = time.perf_counter()
    rows = []
    steps = 0
    target = 0.0
    while True:
        tcur = float(sim.time()[0])
        if tcur >= target - 1e-12:
            d = sim.diagnostics()
            rows.append({"t": round(tcur, 6), "step": steps, "wave_height": np.round(sim.probe_wave_height(xy), 5).tolist(),
                         "pressure": np.round(sim.probe_pressure(pts), 2).tolist(),
                         "force": np.round(sim.probe_force(), 3).tolist() if case.obstacle is not None else None,
                         "mass": d[0], "e_kin": round(d[5], 4), "e_pot": round(d[6], 4), "e_int": round(d[7], 4),
                         "out_of_domain": int(d[8])})
            target += args.every
            if tcur >= args.series:
                break
        sim.step(0.0, 16)
        steps += 16
    sim.sync()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    print(json.dumps({"workload": case.name, "particles": int(sim.n), "h": case.h, "c0": case.c0, "dp": case.dp,
                      "precision": "mixed", "integrator": "Verlet, first-order step every 40", "dt": "adaptive (Eq. 15)",
                      "physical_time_s": args.series, "steps": steps, "wall_s": round(wall, 1),
                      "particle_steps_per_s": round(sim.n * steps / wall, 1), "pair_launch_shape": list(shape),
                      "wave_xy": case.wave_xy, "pressure_xyz": case.pressure_xyz, "series": rows}))
    sim.close()


def run_pair_passes(args):
    """A handle of the workload and args.pair_passes pair passes on its initial
    state (the case an ncu capture of one pair launch is taken on)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2306_01959_gb300 import sph, workloads as wl

    case = wl.by_name(args.workload)
    prec = sph.MIXED if args.precision == "mixed" else sph.FP64
    kw = {"list_skin": args.list_skin} if args.list_skin > 0 else {}
    if args.pair_symmetric:
        kw["pair_symmetric"] = 1
    sim = sph.Simulation(case, precision=prec, **kw)
    ms = []
    for _ in range(args.pair_passes):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.derivatives()
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms.append(round(e0.elapsed_time(e1), 3))
    print(json.dumps({"workload": case.name, "particles": int(sim.n), "precision": args.precision,
                      "list_skin": args.list_skin, "pair_symmetric": bool(args.pair_symmetric),
                      "pair_passes": args.pair_passes,
                      "ms_per_pass_with_readback": ms}))
    sim.close()


def main(argv=None):
    args = parse_args(argv)
    if args.pair_passes > 0:
        run_pair_passes(args)
        return
    if args.series > 0.0:
        run_series(args)
        return
    if args.accuracy_from:
        run_accuracy_from(args)
        return
    if args.accuracy > 0.0:
        run_accuracy(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
