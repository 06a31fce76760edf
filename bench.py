#!/usr/bin/env python
"""Benchmark of the WCSPH particle-interaction pass on GB300.

Metric: particle-steps/s (fluid + boundary particles x steps / s) of the
single dam break with a box obstacle at dp = 0.01 m (3.2 x 1.0 x 1.0 m tank,
1.2 x 1.0 x 0.55 m column, about 0.9 M particles), one step being the whole
pass: pair interaction (Eqs. 3-8), adaptive dt (Eq. 15), Verlet update with
rebinning (Eqs. 9-14), neighbour structure and sorted gather.

Headline `value`: the mixed FP32/FP64 form.  Also reported: the FP64 form on
the same case, the batched alpha sweep (64 instances in one set of launches)
against the same 64 instances run one after another, the pair kernel's
roofline fraction, the end-to-end rate through the C ABI with host buffers,
and the FP64 CPU oracle timed on this host.

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

# FP32 operations of one evaluated pair in the mixed pair kernel, counted from
# its source (pair_term_f): FMA counts 2; add, multiply, min/max and MUFU
# operations count 1.  Every evaluated pair costs 42: relative position and
# velocity 6, |r|^2 5, |r| 3, m F 5, u . r 5, 1/rho_j 2, continuity 2, mu / h 3,
# pressure term 4, accumulation 6, max 1.  A fluid-fluid pair adds 4 (delta
# term) and an approaching pair 12 (c_j 6, switch and scale 2, mean density 3,
# the pressure term's multiply becoming an FMA 1).  The kernel counts both
# classes, so the total is the exact algorithmic work of a launch.
FLOPS_PAIR_BASE, FLOPS_PAIR_DELTA, FLOPS_PAIR_VISC = 42, 4, 12
# FP32 peak from the unit counts and the maximum SM clock: 152 SMs x 128 FP32
# lanes x 2 flop per FMA x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="dambreak_obstacle_dp0.01")
    ap.add_argument("--skip", default="", help="comma list of: fp64,symplectic,paper,gate,batch,cpu,e2e,profile")
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


def cpu_baseline_sample(case, steps=2):
    """The FP64 oracle as it stands, full steps of the whole case on all host cores."""
    import oracle

    cores = oracle.set_threads(os.cpu_count() or 1)
    oc = oracle.make_case(case.tank, case.column, case.obstacle, dp=case.dp, h=case.h, c0=case.c0,
                          rho0=case.rho0, alpha=case.alpha)
    st = oracle.scene(oc)
    t0 = time.perf_counter()
    oracle.run(oc, st, steps)
    dt = time.perf_counter() - t0
    # the same oracle on one thread, one further full step
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.run(oc, st, 1)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": st.n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full FP64 oracle steps of the {case.name} case ({st.n} particles), "
                      f"adaptive dt, OpenMP gather over particles",
            "single_thread": {"value": st.n / dt1, "unit": UNIT, "cores": 1,
                              "sample": "1 further full step of the same case on one thread"}}


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
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {}

    # ---- mixed form: headline
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
    sim16 = sph.Simulation(case, precision=sph.MIXED, use_graph=1, graph_steps=16)
    sim16.autotune(2)
    sim16.step(0.0, 32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim16.stream)
    sim16.step(0.0, 256)
    e1.record(sim16.stream)
    torch.cuda.synchronize()
    steady_ms = e0.elapsed_time(e1) / 256
    sim16.close()

    # ---- pair-kernel roofline: CUDA events around every phase (eager launches)
    roof = None
    phases = None
    stats = None
    if "profile" not in skip:
        sim.set_profiling(True)
        sim.step(0.0, 50)
        phases = sim.phase_times()
        sim.set_profiling(False)
        stats = sim.pair_stats()
        pair_ms, pair_n = phases["pair"]
        pair_s = pair_ms / 1e3 / max(pair_n, 1)
        flops = (FLOPS_PAIR_BASE * stats["evaluated"] + FLOPS_PAIR_DELTA * stats["fluid_fluid"]
                 + FLOPS_PAIR_VISC * stats["approaching"])
        achieved = flops / pair_s / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(FP32_PEAK_TFLOPS, 2),
                "unit": "TFLOP/s", "frac": round(achieved / FP32_PEAK_TFLOPS, 4), "traffic": recorded_traffic(),
                "kernel": "k_pair_mixed", "pair_launch_ms": round(pair_s * 1e3, 4),
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)",
                "flops_per_launch": flops, "pairs_per_launch": stats["evaluated"],
                "flops_per_pair": round(flops / max(stats["evaluated"], 1), 2)}

    # ---- FP64 form on the same case
    fp64 = None
    if "fp64" not in skip:
        sim64 = sph.Simulation(case, precision=sph.FP64, use_graph=1, graph_steps=1)
        sim64.step(0.0, 2)
        sim64.sync()
        k64 = max(3, min(20, args.steps // 50))
        s64 = max_over_ranks(timed_steps(sim64, k64, flush, torch))
        fp64 = {"value": sum_over_ranks(sim64.n) * k64 / s64, "ms_per_step": round(s64 / k64 * 1e3, 3),
                "steps": k64}
        sim64.close()

    # ---- symplectic predictor-corrector (two pair passes per step), mixed form
    sym = None
    if "symplectic" not in skip:
        sims = sph.Simulation(case, precision=sph.MIXED, integrator=sph.SYMPLECTIC, use_graph=1, graph_steps=1,
                              pair_warps=int(best_shape[0]), pair_ctas_per_sm=int(best_shape[1]),
                              pair_group=int(best_shape[2]))
        sims.step(0.0, 3)
        sims.sync()
        ks = max(10, min(200, args.steps // 5))
        ss = max_over_ranks(timed_steps(sims, ks, flush, torch))
        sym = {"value": sum_over_ranks(sims.n) * ks / ss, "ms_per_step": round(ss / ks * 1e3, 4), "steps": ks,
               "pair_passes_per_step": 2, "launches_per_step": sims.launches_per_step()}
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
        kp = max(10, min(200, args.steps // 5))
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
        kg = max(10, min(200, args.steps // 5))
        sg = max_over_ranks(timed_steps(simg, kg, flush, torch))
        gate = {"workload": gc.name, "particles": int(simg.n), "gate_speed": gc.gate_velocity[2],
                "value": sum_over_ranks(simg.n) * kg / sg, "ms_per_step": round(sg / kg * 1e3, 4), "steps": kg,
                "pair_launch_shape": list(shg)}
        simg.close()

    # ---- batched alpha sweep vs the same instances one after another
    batch = None
    if "batch" not in skip:
        cases = shard(wl.alpha_sweep(64, seed=2306), rank, world)
        kb = max(10, min(200, args.steps // 5))
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
        batch = {"instances": 64, "particles": int(sum_over_ranks(nb)), "steps": kb,
                 "value": sum_over_ranks(nb) * kb / tb, "sequential_value": sum_over_ranks(nb) * kb / ts,
                 "speedup": round(ts / tb, 3)}

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
               "steps": ke, "calls": "sph_step(dt=0, 1) + pressure, wave-height and force probes per step"}
    sim.close()

    cpu = None
    if rank == 0 and world == 1 and "cpu" not in skip:
        cpu = cpu_baseline_sample(case)

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
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "fp64": fp64, "speedup_mixed_vs_fp64": round(value / fp64["value"], 2) if fp64 else None,
            "symplectic": sym, "paper_parameters": paper, "gate_dambreak": gate,
            "batched_alpha_sweep": batch, "steady_state_graph16_ms_per_step": round(steady_ms, 4),
            "phase_ms_per_step": {k: round(v[0] / max(v[1], 1), 4) for k, v in phases.items()} if phases else None,
            "pair_stats": stats,
        }
        print(json.dumps(line))


def recorded_traffic():
    """DRAM bytes per pair launch from the committed ncu summary, or None when
    the pair kernel source changed since the counters were taken."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "pair_mixed_traffic.json")
    src = os.path.join(ROOT, "paper_2306_01959_gb300", "csrc", "pair_mixed.cu")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != h:
        return None
    return rec.get("dram_bytes_per_launch")


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle as it stands on the host cores: each step is one
    pair pass over a fixed sample of particles of the same workload (the
    oracle's own neighbour structure rebuilt every step)."""
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
    rng = np.random.Generator(np.random.PCG64(1))
    sample = np.sort(rng.choice(st.n, size=min(st.n, 4096), replace=False)).astype(np.int64)
    for _ in range(max(args.warmup, 1)):
        oracle.derivatives_subset(oc, st, sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.derivatives_subset(oc, st, sample)
    dt = time.perf_counter() - t0
    value = len(sample) * args.steps / dt
    desc = (f"oracle pair pass (Eqs. 3-8, neighbour structure rebuilt) over {len(sample)} sampled particles of "
            f"the {case.name} case ({st.n} particles) per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case.name, "particles": int(st.n)},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_accuracy(args):
    """Mixed vs FP64 on the same case: probe series every 0.01 s of physical
    time; errors reported per time window.  Control: the mixed form against
    itself with one fluid particle moved by 1 nm, which shows how fast any
    rounding-level difference is amplified by the flow itself."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2306_01959_gb300 import sph, workloads as wl

    case = wl.by_name(args.workload)
    pts = np.array(case.pressure_xyz)
    xy = np.array(case.wave_xy)
    t0 = time.perf_counter()

    def series(prec, nudge=False):
        sim = sph.Simulation(case, precision=prec)
        if nudge:
            g = sim.get_state()
            g["r"][0, 0] += 1e-9
            sim.set_state(g["r"], g["u"], g["rho"], g["uprev"], g["rhoprev"], g["step"])
        rows = []
        while True:
            sim.step(0.0, 10)
            tcur = sim.time()[0]
            if tcur >= 0.01 * (len(rows) + 1):
                rows.append((tcur, sim.probe_wave_height(xy), sim.probe_pressure(pts)))
                if tcur >= args.accuracy:
                    break
        sim.sync()
        sim.close()
        torch.cuda.synchronize()
        return rows

    ref = series(sph.FP64)
    mix = series(sph.MIXED)
    ctl = series(sph.MIXED, nudge=True)
    hc = case.column[2]
    pref = 1000.0 * 9.81 * hc

    def errs(a, b, upto):
        n = min(len(a), len(b))
        idx = [i for i in range(n) if a[i][0] <= upto + 1e-9]
        if not idx:
            return None
        w = max(float(np.max(np.abs(a[i][1] - b[i][1]))) for i in idx) / hc
        p = max(float(np.max(np.abs(a[i][2] - b[i][2]))) for i in idx) / pref
        return {"wave_over_Hc": round(w, 5), "pressure_over_rho0_g_Hc": round(p, 5)}

    windows = [round(0.1 * k, 1) for k in range(1, int(round(args.accuracy * 10)) + 1)]
    print(json.dumps({"workload": case.name, "physical_time_s": args.accuracy, "samples": min(len(ref), len(mix)),
                      "mixed_vs_fp64": {str(t): errs(mix, ref, t) for t in windows},
                      "mixed_vs_mixed_nudged_1nm": {str(t): errs(ctl, mix, t) for t in windows},
                      "wall_s": round(time.perf_counter() - t0, 1)}))


def main(argv=None):
    args = parse_args(argv)
    if args.accuracy > 0.0:
        run_accuracy(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
