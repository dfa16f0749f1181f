"""Throughput of the first-passage refinement (rd_first_passage) on encountered pairs.

Encountered pairs are made the way a step makes them: candidate-shaped pairs of the reversible 3D
system (start separations uniform in the cut-off shell, free end points) kept with probability
p_enc, evaluated by the library itself before any timing.  ``python -m
fpt_bench --pairs N --levels K`` prints one JSON line; the benchmark calls
the same functions.
"""
from __future__ import annotations

import argparse
import json
import statistics


def encountered_pairs(pkg, torch, system, n, seed=11):
    """n encountered pairs (device float64 tensors r0, r; the distinct ones repeated) and the
    number of distinct pairs."""
    import workloads as W

    pr = system.pairs[0]
    Drel = system.D[pr.s1] + system.D[pr.s2]
    r0n, rn = W.pair_samples(n, pr.sigma, Drel, system.dt, seed=seed)
    sim = pkg.Simulation(system, precision="fp64")
    r0c, rc = torch.tensor(r0n, device="cuda"), torch.tensor(rn, device="cuda")
    pe, _ = sim.pair_probs(r0c, rc)
    sim.sync()
    sim.close()
    gen = torch.Generator(device="cuda").manual_seed(5)
    keep = torch.rand(pe.shape, device="cuda", dtype=torch.float64, generator=gen) < pe
    r0e, re = r0c[keep], rc[keep]
    distinct = int(r0e.numel())
    reps = -(-n // max(1, distinct))
    return r0e.repeat(reps)[:n].contiguous(), re.repeat(reps)[:n].contiguous(), distinct


def time_refinement(pkg, torch, system, r0e, re, levels, reps=5, warmup=3, flush=None, precision="fp64"):
    """Median device time of rd_first_passage over `reps` launches (CUDA events on the handle's
    stream; the L2 is overwritten between launches when `flush` is given).  precision "mixed"
    selects the FP32 evaluation (3D)."""
    sim = pkg.Simulation(system, precision=precision)
    n = r0e.numel()
    streams = torch.arange(n, dtype=torch.int64, device="cuda")
    for _ in range(warmup):
        g = sim.first_passage(r0e, re, streams, levels)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        if flush is not None:
            flush.add_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(sim.stream):
            sim.stream.wait_stream(torch.cuda.current_stream())
            a.record(sim.stream)
        g = sim.first_passage(r0e, re, streams, levels)
        with torch.cuda.stream(sim.stream):
            b.record(sim.stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b) * 1e-3)
    t = statistics.median(times)
    att = g["attempts"].double()
    out = {"pairs": n, "levels": levels, "ms": 1e3 * t, "pairs_per_s": n / t,
           "attempts_per_s": float(att.sum().item()) / t, "mean_attempts": float(att.mean().item()),
           "max_attempts": int(att.max().item()), "over_attempt_bound": int((g["bin"] < 0).sum().item()),
           # pairs and their draws by the draw count at which the work moves to wider search tiers
           "draw_tiers": [{"over": lo, "pairs": int((att > lo).sum().item()),
                           "draws": float(att[att > lo].sum().item())} for lo in (256, 4352, 32768)]}
    sim.close()
    return out


def main(argv=None):
    import torch

    import paper_1107_0270_gb300 as pkg
    import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=1 << 20)
    ap.add_argument("--levels", type=int, default=10)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    a = ap.parse_args(argv)
    system = W.reversible_3d(seed=2)
    flush = torch.empty(512 << 18, dtype=torch.float32, device="cuda")
    r0e, re, distinct = encountered_pairs(pkg, torch, system, a.pairs)
    res = time_refinement(pkg, torch, system, r0e, re, a.levels, reps=a.reps, flush=flush, precision=a.precision)
    res["precision"] = a.precision
    res["distinct_pairs"] = distinct
    print(json.dumps(res))


if __name__ == "__main__":
    main()
