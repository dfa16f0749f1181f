#!/usr/bin/env python3
"""Benchmark of the GF-BD reaction-diffusion step on GB300.

Default workload: 3D reversible A+B<->C with a radiation boundary condition, periodic cube
L = 2.55 um (10 uM), N_A = N_B = 1e5, sigma = 0.005 um, D = 1 (C: 0.5) um^2/s, ka = 0.02 um^3/s,
kd = 10 /s, dt = 1e-5 s (tau = 0.8), started from the mass-action equilibrium composition.
One "step" = one pass of the whole step (decays, displacements, binning, cell sweep with p_enc,
conflict resolution, pair resolution, products, compaction, observables) for every particle.

Timing: W warm-up steps, then K steps as two-step CUDA-graph launches, each bracketed by CUDA
events on the library's stream; the L2 cache is flushed (512 MiB write) between timed launches,
outside the events.  Multi-GPU (torchrun): every rank runs an independent replica with its own seed
("replicas only", weak scaling); value = all ranks' particle-steps / the slowest rank's time.

``--impl reference`` times the plain CPU FP64 oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

KERNELS_PER_STEP = 7           # kernels of one step with separate launches: prepare, scan (cells),
                               # scatter, sweep, matching (trivial pairs, rounds, resolution), angle
                               # pass (exact directions only), compaction (scan + placement)
# the fused launch runs the same stages as phases of one cooperative kernel (the matching as two)
KERNEL_OF_PHASE = {"ph_prepare": "k_prepare", "ph_scan_cells": "k_scan_cells", "ph_scatter_cells": "k_scatter_cells",
                   "ph_sweep": "k_sweep", "ph_angles": "k_angles", "ph_compact": "k_compact"}
L2_FLUSH_BYTES = 512 << 20


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--dt", type=float, default=1e-5)
    ap.add_argument("--n-each", type=int, default=100_000)
    ap.add_argument("--step-launch", default="auto", choices=["auto", "fused", "separate"],
                    help="one cooperative launch per step, one launch per kernel, or the autotuner's pick")
    ap.add_argument("--angle", default="free_step", choices=["free_step", "exact"],
                    help="direction of a resampled pair: the free step's (the step as specified) or "
                         "drawn from the full propagator (measured beside it in any case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip FP64 comparison, pair-prob batch, e2e")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the ensemble, network and membrane context measurements")
    return ap.parse_args(argv)


def box_edge(args):
    """Box edge keeping the 10 uM concentration of the L = 2.55 um, 1e5 + 1e5 system."""
    return 2.55 * (args.n_each / 100_000) ** (1.0 / 3.0)


def workload(args, seed=1, angle=None):
    system = W.reversible_3d(dt=args.dt, seed=seed, n_each=args.n_each, L=box_edge(args), equilibrium_start=True)
    system.angle = angle or args.angle
    return system


def workload_name(args):
    return (f"3D A+B<->C radiation BC, L={box_edge(args):.3g} um (10 uM), N_A=N_B={args.n_each:.0e} "
            f"(mass-action start), sigma=0.005, D=1/1/0.5, ka=0.02, kd=10, dt={args.dt:g}, "
            f"pair direction: {args.angle}")


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# roofline bookkeeping
# ------------------------------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_per_launch(kernel, precision, n):
    """DRAM bytes per launch of `kernel` from one ncu capture (profiles/traffic.json), scaled to n
    particles by the particles of the captured workload (the traffic of these kernels grows in
    proportion to the particles they move); None when no capture of the current kernel exists."""
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        tj = json.load(f)
    rec = tj.get(f"{kernel}:{precision}")
    if not isinstance(rec, dict) or rec.get("bytes") is None or not rec.get("particles"):
        return None
    return rec["bytes"] * n / rec["particles"]


def algorithmic_bytes(kernel, precision, w):
    """Per-launch algorithmic bytes of a step kernel: the data the stage must read and write once
    (w: particles n, binned particles nb, cells, fired pairs, accepted pairs, decays per step).
    v = bytes of one position record (x, y, z, species/id bits)."""
    v = 16 if precision == "mixed" else 32
    n, nb, cells = w["n"], w["nb"], w["cells"]
    fired, acc, dec = w["fired"], w["accepted"], w["decays"]
    table = {
        # read position + id; write end position, status, cell, slot; one cell counter per binned
        "k_prepare": n * (2 * v + 16) + 4 * nb,
        # read the cell counts, write the cell starts, clear the counts
        "k_scan_cells": 12 * cells,
        # read cell, slot, both positions, id, cell start; write both sorted positions + index
        "k_scatter_cells": nb * (4 * v + 20),
        # both positions of every binned particle once, the cell starts once, the fired records
        "k_sweep": nb * 2 * v + 4 * cells + fired * 52,
        # trivial pairs: fired records and both degrees, accepted / conflict lists (48 B per fired
        # pair); then degrees cleared, and per accepted pair or decay: record, state, 2x2 positions
        # read, 2 positions + statuses written (conflict rounds add re-reads of the conflict pairs)
        "k_match_resolve": fired * (48 + 16) + (acc + dec) * (48 + 6 * v),
        # one 160-B job per resolved pair or decay pair left to it; write two positions (only
        # when directions come from the full propagator)
        "k_angles": (acc + dec) * (160 + 2 * v) if w.get("angles") else 0,
        # read status, end position, id; write position + id (the scan stays on chip)
        "k_compact": n * (2 * v + 12),
    }
    table["k_step_fused"] = sum(table.values())      # the whole step in one launch
    # the fused launch's two matching phases split the matching kernel's bytes
    table["ph_match_trivial"] = fired * 48
    table["ph_match_resolve"] = table["k_match_resolve"] - fired * 48
    kernel = KERNEL_OF_PHASE.get(kernel, kernel)     # a phase of the fused launch = its stage's kernel
    if kernel not in table:
        raise KeyError(f"no algorithmic byte count for step kernel {kernel}")
    return table[kernel]


# ------------------------------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample
# ------------------------------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (x86: /proc/cpuinfo; Arm: lscpu), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def _oracle_rate(O, system, seconds, openmp, max_steps=None):
    """Particle-steps/s of the oracle stepping `system` for about `seconds` (or max_steps)."""
    st = O.init_state(system)
    ps = steps = 0
    t0 = time.perf_counter()
    while True:
        n = st.n
        st, _ = O.step(system, st, openmp=openmp)
        ps += n
        steps += 1
        if max_steps is not None and steps >= max_steps:
            break
        if max_steps is None and time.perf_counter() - t0 >= seconds and steps >= 2:
            break
    return ps / (time.perf_counter() - t0), steps


def oracle_sample(args, seconds, seed=1):
    """The CPU baseline: the FP64 oracle, single-threaded and (OpenMP build, pair loop on all
    threads, same results) on all host cores, on bounded samples of the workloads."""
    import oracle as O

    O.build()
    # Same density, time step and chemistry; a smaller box so that the O(N^2) oracle fits the
    # time budget.  Rate reported per particle-step.
    n_each = 4000
    L = box_edge(args) * (n_each / args.n_each) ** (1 / 3)
    system = W.reversible_3d(dt=args.dt, seed=seed, n_each=n_each, L=L, equilibrium_start=True)
    system.angle = args.angle
    v1, steps = _oracle_rate(O, system, seconds, openmp=False)
    out = {"value": v1, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
           "sample": f"{steps} oracle steps of the same system in a sub-box L={L:.3f} um with "
                     f"N_A=N_B={n_each} (same 10 uM density, dt, chemistry); O(N^2) candidate "
                     f"search, single thread (the O(N^2) search makes the per-particle cost grow "
                     f"with the box, so the full-size system would run slower per particle)",
           "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    threads = O.threads(True) if O.lib(True) is not None else 1
    if threads > 1:
        vall, steps_all = _oracle_rate(O, system, seconds / 3, openmp=True)
        out["all_cores"] = {"value": vall, "unit": "particle-steps/s", "cores": threads,
                            "sample": f"{steps_all} steps of the same sub-box, OpenMP build (pair loop on all threads)"}
    # the irreversible A+B->C workload in full (2000 A + 2000 B... 1000 + 1000, 2000 steps) and the
    # first 64 replicas of the ensemble, on all cores when the OpenMP build exists
    omp = threads > 1
    irr = W.irreversible_3d(seed=seed)
    irr.angle = args.angle
    v0, n0 = _oracle_rate(O, irr, 0.0, openmp=omp, max_steps=2000)
    out["irreversible_3d_full"] = {"value": v0, "unit": "particle-steps/s", "cores": threads, "steps": n0,
                                   "sample": "3D A+B->C, 1000 + 1000 in L = 1 um, dt = 1e-5, all 2000 steps"}
    ens = W.ensemble_3d()
    ens.angle = args.angle
    reps = ens.replica_list()[:64]
    t0 = time.perf_counter()
    ps = 0
    for r, rep in enumerate(reps):
        sysr = W.System(**{**ens.__dict__, "L": rep.L, "n_init": list(rep.n_init), "replicas": None})
        st = O.init_state(sysr)
        st2, _ = O.step(sysr, st, openmp=omp)
        ps += st.n
    el = time.perf_counter() - t0
    out["ensemble_3d_64_replicas"] = {"value": ps / el, "unit": "particle-steps/s", "cores": threads,
                                      "sample": "one step of each of the first 64 of the 4096 replicas "
                                                f"({ps} particles); the whole ensemble's rate extrapolates "
                                                "per replica"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    # bounded per-step samples: each timed "step" is one oracle step of the sub-box sample
    import oracle as O

    O.build()
    n_each = 4000
    L = box_edge(args) * (n_each / args.n_each) ** (1 / 3)
    system = W.reversible_3d(dt=args.dt, seed=1, n_each=n_each, L=L, equilibrium_start=True)
    system.angle = args.angle
    st = O.init_state(system)
    for _ in range(max(args.warmup, 0) and min(args.warmup, 3)):
        st, _ = O.step(system, st)
    steps = min(args.steps, 40)
    ps = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        ps += st.n
        st, _ = O.step(system, st)
    el = time.perf_counter() - t0
    v = ps / el
    line = {"impl": "reference", "metric": "particle-steps/s", "value": v, "unit": "particle-steps/s",
            "n_gpus": world, "steps": steps, "warmup": min(args.warmup, 3), "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args) + " -- oracle on a bounded sub-box sample"},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{steps} steps, sub-box L={L:.3f} um, N_A=N_B={n_each} at the same density"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def timed_graph_run(sim, torch, flush, steps):
    """K steps as two-step graph launches, each between CUDA events on the library's stream."""
    launches = steps // 2
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(launches)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(launches)]
    s = sim.stream
    for k in range(launches):
        with torch.cuda.stream(s):
            flush.add_(1)                      # L2 flush, outside the timed events
        s.synchronize()                        # finished before the timed launch starts
        with torch.cuda.stream(s):
            starts[k].record(s)
        sim.run(2)
        with torch.cuda.stream(s):
            ends[k].record(s)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / 1e3, 2 * launches


def reduce_over_ranks(dist, torch, elapsed, ps_local, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's time and the particle-steps of
    all ranks (each rank runs its own independent system)."""
    if dist is None:
        return elapsed, float(ps_local)
    tt = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    pt = torch.tensor([float(ps_local)], dtype=torch.float64, device=device)
    dist.all_reduce(pt)
    return float(tt.item()), float(pt.item())


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1107_0270_gb300 as pkg

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    system = workload(args, seed=1 + rank)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    sim = pkg.Simulation(system, precision=args.precision, cell_factor="tune", step_launch=args.step_launch)
    layout = sim.info()
    sim.run(max(args.warmup, 3))
    sim.sync()
    obs0 = sim.observables()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with ClockSampler(local_rank) as clk:
        elapsed, steps_done = timed_graph_run(sim, torch, flush, args.steps)
    barrier()
    obs1 = sim.observables()
    ps_local = obs1["stats"]["particle_steps"] - obs0["stats"]["particle_steps"]
    cand_local = obs1["stats"]["candidates"] - obs0["stats"]["candidates"]
    t_max, ps_total = reduce_over_ranks(dist, torch, elapsed, ps_local, "cuda")
    value = ps_total / t_max

    extras = {}
    if rank == 0:
        # per-kernel times of single (non-graph) steps, CUDA events on the library's stream
        ker = {}
        nsamp = 20
        n_now = sim.num_particles()
        for _ in range(nsamp):
            flush.add_(1)
            torch.cuda.synchronize()
            for name, ms in sim.timed_step():
                ker.setdefault(name, []).append(ms)
        ker_avg = {k: sum(v) / len(v) for k, v in ker.items()}
        fused = "k_step_fused" in ker_avg
        # with the fused launch the step is ONE kernel (its phases are reported beside it)
        phases = {k: v for k, v in ker_avg.items() if k != "k_step_fused"}
        step_ms = ker_avg["k_step_fused"] if fused else sum(ker_avg.values())
        dominant = "k_step_fused" if fused else max(ker_avg, key=lambda k: ker_avg[k])
        st = sim.get_state()
        d_stats = {k: obs1["stats"][k] - obs0["stats"][k] for k in obs1["stats"]}
        per = max(steps_done, 1)
        work = {"n": n_now, "nb": int(np.sum(np.isin(st["species"], [0, 1]))), "cells": layout["cells"],
                "fired": d_stats["fired"] / per, "accepted": d_stats["matched"] / per,
                "decays": d_stats["decays"] / per, "angles": args.angle == "exact"}
        cand_per_step = cand_local / per
        peak, peak_kind = measured_peaks()
        ab = algorithmic_bytes(dominant, args.precision, work)
        achieved = ab / (ker_avg[dominant] * 1e-3) / 1e9
        traffic = traffic_per_launch(dominant, args.precision, work["n"])
        extras["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                              "frac": achieved / peak, "traffic": traffic, "kernel": dominant,
                              "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({peak_kind})",
                              "algorithmic_bytes_per_launch": ab, "kernel_ms": ker_avg[dominant],
                              "share": ker_avg[dominant] / step_ms}
        step_bytes = sum(algorithmic_bytes(k, args.precision, work) for k in phases)
        step_graph_ms = 1e3 * t_max / per
        extras["step_roofline"] = {"bound": "hbm", "algorithmic_bytes_per_step": step_bytes,
                                   "ms_per_step": step_graph_ms,
                                   "achieved": step_bytes / (step_graph_ms * 1e-3) / 1e9, "peak": peak,
                                   "unit": "GB/s",
                                   "frac": step_bytes / (step_graph_ms * 1e-3) / 1e9 / peak,
                                   "work_per_step": {k: round(float(v), 1) for k, v in work.items()}}
        extras["kernel_ms"] = {k: round(v, 5) for k, v in ker_avg.items()}
        extras["phase_roofline"] = {
            k: {"ms": round(v, 5), "algorithmic_bytes": algorithmic_bytes(k, args.precision, work),
                "frac": algorithmic_bytes(k, args.precision, work) / max(v * 1e-3, 1e-12) / 1e9 / peak}
            for k, v in phases.items()}
        sweep_ms = ker_avg.get("ph_sweep", ker_avg.get("k_sweep"))
        extras["sweep_pair_prob_evals_per_s"] = cand_per_step / (sweep_ms * 1e-3)
        extras["candidates_per_step"] = cand_per_step
        if not args.no_extras:
            extras.update(extra_measurements(args, torch, pkg, flush, sim))
    sim.close()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    clocks = clk.summary()
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": steps_done, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t_max / steps_done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "precision": args.precision, "angle": args.angle,
                   "particles": int(obs1["counts"].sum()), "timing": "2-step CUDA graph launches, events on the library stream",
                   "l2": "flushed (512 MiB write) between timed graph launches",
                   "parallelism": f"replicas x{world} (one independent system per GPU)"},
        "gpu_launches": steps_done // 2 if layout.get("fused")
        else (KERNELS_PER_STEP - (args.angle != "exact")) * steps_done,
        "layout": layout,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
    }
    line.update(extras)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(args, args.cpu_sample_seconds)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def extra_measurements(args, torch, pkg, flush, sim_main):
    out = {}
    # FP64 step on the same workload
    if args.precision == "mixed":
        sim64 = pkg.Simulation(workload(args), precision="fp64", cell_factor="tune")
        sim64.run(max(args.warmup, 3))
        sim64.sync()
        o0 = sim64.observables()
        el, nst = timed_graph_run(sim64, torch, flush, min(args.steps, 1000))
        o1 = sim64.observables()
        out["fp64"] = {"value": (o1["stats"]["particle_steps"] - o0["stats"]["particle_steps"]) / el,
                       "unit": "particle-steps/s", "steps": nst, "ms_per_step": 1e3 * el / nst}
        sim64.close()
    # standalone pair-probability batch (p_enc only) on 2^25 candidate-shaped pairs (> L2)
    system = workload(args)
    pr = system.pairs[0]
    Drel = system.D[pr.s1] + system.D[pr.s2]
    r0n, rn = W.pair_samples(1 << 20, pr.sigma, Drel, system.dt, seed=11)
    reps = 32
    r0 = torch.tensor(np.tile(r0n, reps), device="cuda")
    r = torch.tensor(np.tile(rn, reps), device="cuda")
    res = {}
    for prec in ("mixed", "fp64"):
        sim = pkg.Simulation(workload(args, seed=2), precision=prec)
        pe = torch.empty_like(r0)
        for _ in range(3):
            sim.pair_probs(r0, r, out=(pe, None))
        torch.cuda.synchronize()
        times = []
        for _ in range(10):
            flush.add_(1)
            torch.cuda.synchronize()           # the flush has finished before the timed launch
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(sim.stream):
                sim.stream.wait_stream(torch.cuda.current_stream())
                a.record(sim.stream)
            sim.pair_probs(r0, r, out=(pe, None))
            with torch.cuda.stream(sim.stream):
                b.record(sim.stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) * 1e-3)
        t = statistics.median(times)
        gbs = r0.numel() * 24 / t / 1e9
        peak, _ = measured_peaks()
        res[prec] = {"evals_per_s": r0.numel() / t, "gbs": gbs, "pairs": r0.numel(),
                     # 24 B per pair against the measured HBM copy rate; the FP64 batch is bound by
                     # the FP64 pipe instead (profiles/k_pair_probs_fp64_2e25pairs.md)
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                  "frac": gbs / peak}}
        sim.close()
    # error of the mixed probabilities at scale: the 2^20 distinct pairs of the batch, mixed against
    # the FP64 GPU values (which match the oracle to 1e-12)
    ru0, ru = torch.tensor(r0n, device="cuda"), torch.tensor(rn, device="cuda")
    vals = {}
    for prec in ("mixed", "fp64"):
        sim = pkg.Simulation(workload(args, seed=2), precision=prec)
        pe, pre = sim.pair_probs(ru0, ru)
        sim.sync()
        vals[prec] = (pe.cpu().numpy(), pre.cpu().numpy())
        sim.close()
    d_enc = np.abs(vals["mixed"][0] - vals["fp64"][0])
    d_reac = np.abs(vals["mixed"][1] - vals["fp64"][1])
    res["mixed_max_abs_error"] = {"p_enc": float(d_enc.max()), "p_reac": float(d_reac.max()),
                                  "pairs": int(d_enc.size), "target": 2e-6}
    out["pair_prob_evals_per_s"] = res
    out["first_passage"] = fpt_measurement(args, torch, pkg, flush)
    # the other time steps of the same configuration, mixed and FP64 (device-timed graph launches)
    sweep = {}
    for dt in (1e-6, 1e-4):
        for prec in ("mixed", "fp64"):
            system = W.reversible_3d(dt=dt, seed=1, n_each=args.n_each, L=box_edge(args), equilibrium_start=True)
            system.angle = args.angle
            sim = pkg.Simulation(system, precision=prec)
            sim.run(4)
            sim.sync()
            o0 = sim.observables()
            el, nst = timed_graph_run(sim, torch, flush, 200)
            o1 = sim.observables()
            sweep[f"dt={dt:g}:{prec}"] = {
                "value": (o1["stats"]["particle_steps"] - o0["stats"]["particle_steps"]) / el,
                "unit": "particle-steps/s", "ms_per_step": 1e3 * el / nst,
                "candidates_per_step": (o1["stats"]["candidates"] - o0["stats"]["candidates"]) / nst}
            sim.close()
    out["dt_sweep"] = sweep
    out["exact_angles"] = exact_angle_measurement(args, torch, pkg, flush)
    if not args.no_workloads:
        out["workloads"] = other_workloads(torch, pkg, flush, args.angle)
    # end to end through the C ABI with host buffers: per step, upload the state from page-locked
    # host memory (rd_set_state), one step, read the resulting state (positions, species, ids,
    # next ids) back into page-locked host memory (rd_get_state).  The headline is one system, so
    # the per-particle replica array, which the ABI makes optional for it, is not moved.
    sim = pkg.Simulation(workload(args, seed=3), precision=args.precision)
    sim.run(4)
    cap = 2 * sim.num_particles() + 1024

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()

    bufs = [{"x": pinned((cap, 3), torch.float64), "species": pinned(cap, torch.int32),
             "ids": pinned(cap, torch.int32).view(np.uint32),
             "next_id": pinned(1, torch.int32).view(np.uint32)} for _ in range(2)]
    st = sim.get_state(out=bufs[0])

    def e2e_step(st, k):
        sim.set_state(st["x"], st["species"], st["ids"], st["replica"], st["next_id"], st["step"])
        sim.step()
        return sim.get_state(out=bufs[(k + 1) % 2])

    for k in range(3):
        st = e2e_step(st, k)
    # five blocks of 20 steps, host wall clock; the median block is reported (host jitter)
    rates, h2d, d2h, n_e2e = [], 0, 0, 0
    for _ in range(5):
        t0 = time.perf_counter()
        ps = 0
        for k in range(20):
            n = st["ids"].shape[0]
            st = e2e_step(st, k)
            ps += n
            h2d += n * (24 + 4 + 4) + 4
            d2h += st["ids"].shape[0] * (24 + 4 + 4) + 4
            n_e2e += 1
        rates.append(ps / (time.perf_counter() - t0))
    binding_rate = statistics.median(rates)
    # the same three calls made on the C ABI directly (what a C caller does): pointers and
    # by-reference outputs prepared once, so the host's share per step is the three calls alone
    import ctypes as C

    lib, h = pkg._lib(), sim._h
    ptrs = [(b["x"].ctypes.data_as(C.POINTER(C.c_double)), b["species"].ctypes.data_as(C.POINTER(C.c_int32)),
             b["ids"].ctypes.data_as(C.POINTER(C.c_uint32)), b["next_id"].ctypes.data_as(C.POINTER(C.c_uint32)))
            for b in bufs]
    n_io, step_io = C.c_int64(), C.c_int64()
    n_ref, step_ref = C.byref(n_io), C.byref(step_io)
    n_cur, step_cur = int(st["ids"].shape[0]), int(st["step"])
    if st["ids"].ctypes.data != bufs[0]["ids"].ctypes.data:     # the state must sit in buffer 0
        for key in ("x", "species", "ids"):
            bufs[0][key][:n_cur] = st[key]
        bufs[0]["next_id"][:] = st["next_id"]

    def capi_step(k, n, step):
        xa, spa, ida, nxa = ptrs[k % 2]
        xb, spb, idb, nxb = ptrs[(k + 1) % 2]
        rc = lib.rd_set_state(h, n, xa, spa, ida, None, nxa, step)
        if rc == 0:
            rc = lib.rd_step(h)
        if rc == 0:
            n_io.value = cap
            rc = lib.rd_get_state(h, n_ref, xb, spb, idb, None, nxb, step_ref)
        if rc != 0:
            raise pkg.RDError(rc, "C-ABI end-to-end step")
        return n_io.value, step_io.value

    for k in range(4):                                            # even count: the state is back in buffer 0
        n_cur, step_cur = capi_step(k, n_cur, step_cur)
    rates, h2d, d2h, n_e2e = [], 0, 0, 0
    for _ in range(5):
        t0 = time.perf_counter()
        ps = 0
        for k in range(20):
            n_in = n_cur
            n_cur, step_cur = capi_step(k, n_cur, step_cur)
            ps += n_in
            h2d += n_in * (24 + 4 + 4) + 4
            d2h += n_cur * (24 + 4 + 4) + 4
            n_e2e += 1
        rates.append(ps / (time.perf_counter() - t0))
    out["e2e"] = {"value": statistics.median(rates), "unit": "particle-steps/s", "h2d_bytes_per_step": h2d // n_e2e,
                  "d2h_bytes_per_step": d2h // n_e2e,
                  "path": "rd_set_state (page-locked host arrays: positions, species, ids, next id) + rd_step "
                          "+ rd_get_state (the same arrays back), per step, called on the C ABI with "
                          "pointers prepared once",
                  "binding_value": binding_rate,
                  "binding_path": "the same three calls through the Python binding's Simulation.set_state / "
                                  "step / get_state"}
    sim.close()
    return out


def fpt_measurement(args, torch, pkg, flush, levels=10):
    """First-passage refinement (rd_first_passage) of 2^20 encountered pairs of the headline rule,
    FP64 and FP32 (mixed handle), device-timed, with the oracle on a sample of the same pairs beside it."""
    import fpt_bench

    system = workload(args, seed=2)
    r0e, re, distinct = fpt_bench.encountered_pairs(pkg, torch, system, 1 << 20)
    res = {"distinct_pairs": distinct}
    for prec in ("fp64", "mixed"):
        res[prec] = fpt_bench.time_refinement(pkg, torch, system, r0e, re, levels, flush=flush, precision=prec)
    # CPU baseline: the oracle on a bounded sample of the same pairs, one host thread
    import oracle as O

    pr = system.pairs[0]
    m = 2000
    Drel = system.D[pr.s1] + system.D[pr.s2]
    tau = Drel * system.dt / pr.sigma ** 2
    a0, a1 = r0e[:m].cpu().numpy() / pr.sigma, re[:m].cpu().numpy() / pr.sigma
    t0 = time.perf_counter()
    O.fpt_refine_batch(system.dim, a0, a1, tau, levels, system.seed, np.arange(m, dtype=np.uint64))
    res["cpu_baseline"] = {"value": m / (time.perf_counter() - t0), "unit": "pairs/s", "cores": 1,
                           "kind": "oracle", "sample": f"the first {m} of the same pairs"}
    return res


def exact_angle_measurement(args, torch, pkg, flush):
    """The headline workload with every resampled pair's direction drawn from the full propagator
    (the angle pass), both precisions: rate and the angle pass's share of the step."""
    res = {}
    for prec, steps in (("mixed", 40), ("fp64", 20)):
        sim = pkg.Simulation(workload(args, seed=1, angle="exact"), precision=prec)
        sim.run(4)
        sim.sync()
        o0 = sim.observables()
        el, nst = timed_graph_run(sim, torch, flush, steps)
        o1 = sim.observables()
        ker = {}
        for _ in range(4):
            for kname, ms in sim.timed_step():
                ker[kname] = ker.get(kname, 0.0) + ms / 4
        ang = ker.get("ph_angles", ker.get("k_angles", 0.0))
        res[prec] = {"value": (o1["stats"]["particle_steps"] - o0["stats"]["particle_steps"]) / el,
                     "unit": "particle-steps/s", "ms_per_step": 1e3 * el / nst,
                     "angle_pass_ms": round(ang, 5),
                     "jobs_per_step": (o1["stats"]["resampled"] - o0["stats"]["resampled"]) / nst,
                     "fallbacks": o1["stats"]["angle_fallback"] - o0["stats"]["angle_fallback"]}
        sim.close()
    return res


def other_workloads(torch, pkg, flush, angle="free_step"):
    """The other experiment shapes at full size (mixed precision), timed like the headline."""
    cases = [
        ("ensemble_3d", "4096 independent 3D A+B<->C replicas, N per species log-uniform in [64, 8192], "
                        "1-20 uM, dt=1e-5", lambda: W.ensemble_3d(), 40),
        ("network_3d", "5-species 3D network, 1e7 particles in L=20 um, dt=1e-5", lambda: W.network_3d(dt=1e-5), 20),
        ("membrane_2d", "2D A+B<->C (+C+C reflective), 2e5+2e5 in L=10 um, dt=1e-4 (tau=0.8, Weber tables)",
         lambda: W.membrane_2d(), 40),
    ]
    res = {}
    for name, desc, make, steps in cases:
        try:
            t0 = time.perf_counter()
            system = make()
            system.angle = angle
            sim = pkg.Simulation(system, precision="mixed")
            init_s = time.perf_counter() - t0
            sim.run(4)
            sim.sync()
            o0 = sim.observables()
            el, nst = timed_graph_run(sim, torch, flush, steps)
            o1 = sim.observables()
            ker = {}
            for _ in range(4):
                for kname, ms in sim.timed_step():
                    ker[kname] = ker.get(kname, 0.0) + ms / 4
            ps = o1["stats"]["particle_steps"] - o0["stats"]["particle_steps"]
            res[name] = {"workload": desc, "value": ps / el, "unit": "particle-steps/s", "steps": nst,
                         "ms_per_step": 1e3 * el / nst, "particles": int(o1["counts"].sum()),
                         "init_s": round(init_s, 2), "layout": sim.info(),
                         "kernel_ms": {k: round(v, 5) for k, v in ker.items()}}
            sim.close()
        except Exception as exc:  # report, do not hide
            res[name] = {"workload": desc, "error": str(exc)[:200]}
        torch.cuda.empty_cache()
    return res


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
