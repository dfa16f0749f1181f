"""Small, self-contained runs of single kernels for ncu captures (the summaries under profiles/
name the command).  Each case builds a system, runs a few steps (or a few pair-probability batches)
and exits; the kernel of interest is then captured with `ncu -k regex:<kernel> -s <skip> -c 1`.

  python profile_cases.py network SCALE     5-species 3D network at SCALE x 1e7 particles, mixed
  python profile_cases.py ensemble R        the first R replicas of the 4096-replica ensemble, mixed
  python profile_cases.py pairprob PREC     2^25 candidate-shaped pairs of the headline rule (PREC
                                            mixed or fp64), three batches
  python profile_cases.py headline PREC     the headline 3D A+B<->C system (1e5 + 1e5, dt = 1e-5,
                                            mass-action start), free-step directions (PREC mixed or
                                            fp64), separate kernels, six steps
  python profile_cases.py angles PREC       the same system with directions drawn from the full
                                            propagator: the angle pass runs once a step
"""
import argparse

import numpy as np

import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["network", "ensemble", "pairprob", "headline", "angles"])
    ap.add_argument("size", help="network: scale; ensemble: replicas; pairprob, headline, angles: precision")
    args = ap.parse_args()

    import torch

    import paper_1107_0270_gb300 as pkg

    if args.case in ("network", "ensemble"):
        if args.case == "network":
            system = W.network_3d(dt=1e-5, scale=float(args.size), L=20.0)
        else:
            system = W.ensemble_3d(n_replicas=int(args.size))
        system.angle = "free_step"
        sim = pkg.Simulation(system, precision="mixed", step_launch="separate")
        sim.run(4)
        for _ in range(2):
            print(dict(sim.timed_step()), flush=True)
        print("particles", sim.num_particles(), sim.info(), flush=True)
        sim.close()
        return
    system = W.reversible_3d(dt=1e-5, seed=2, n_each=100_000, L=2.55, equilibrium_start=True)
    if args.case in ("headline", "angles"):
        system.angle = "exact" if args.case == "angles" else "free_step"
        sim = pkg.Simulation(system, precision=args.size, step_launch="separate")
        sim.run(4)
        for _ in range(2):
            print(dict(sim.timed_step()), flush=True)
        print("particles", sim.num_particles(), "stats", sim.observables()["stats"], flush=True)
        sim.close()
        return
    pr = system.pairs[0]
    d_rel = system.D[pr.s1] + system.D[pr.s2]
    r0n, rn = W.pair_samples(1 << 20, pr.sigma, d_rel, system.dt, seed=11)
    r0 = torch.tensor(np.tile(r0n, 32), device="cuda")
    r = torch.tensor(np.tile(rn, 32), device="cuda")
    sim = pkg.Simulation(system, precision=args.size)
    pe = torch.empty_like(r0)
    for _ in range(3):
        sim.pair_probs(r0, r, out=(pe, None))
    torch.cuda.synchronize()
    print("pairs", r0.numel(), flush=True)
    sim.close()


if __name__ == "__main__":
    main()
