"""Host-side checks of the benchmark's bookkeeping (no GPU): every kernel that the step launches
has an algorithmic byte count, the launch count per step matches the timer marks, and the
default system is the configuration the line names."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def step_kernel_marks():
    src = open(os.path.join(ROOT, "paper_1107_0270_gb300", "csrc", "rd_kernels.cu")).read()
    body = src[src.index("static void step_impl"):]
    body = body[:body.index("\n}\n")]
    return re.findall(r'mark\("(k_[a-z_]+)"\)', body)


def test_every_step_kernel_has_algorithmic_bytes():
    marks = step_kernel_marks()
    # one timer mark after each kernel of the step (a launch that picks between two kernel
    # variants still launches one)
    assert len(marks) == len(set(marks)) == bench.KERNELS_PER_STEP
    w = {"n": 1000, "nb": 800, "cells": 500, "fired": 10, "accepted": 8, "decays": 2, "angles": True}
    for k in marks:
        for prec in ("mixed", "fp64"):
            assert bench.algorithmic_bytes(k, prec, w) > 0
    # the angle pass moves nothing when directions are the free step's (it is not launched then)
    assert bench.algorithmic_bytes("k_angles", "mixed", {**w, "angles": False}) == 0


def test_default_workload_is_the_named_configuration():
    """The benchmark's default system is the one its config line names: 3D A+B<->C with the
    radiation boundary condition, 1e5 + 1e5 particles in L = 2.55 um (10 uM), sigma 0.005,
    D = 1/1/0.5, ka 0.02, kd 10, dt 1e-5, started at the mass-action composition."""
    args = bench.parse([])
    s = bench.workload(args)
    assert (args.gpus, args.precision, args.angle) == (1, "mixed", "free_step")
    assert s.dim == 3 and abs(s.L - 2.55) < 1e-12 and s.dt == 1e-5
    assert list(s.D) == [1.0, 1.0, 0.5]
    (pr,) = s.pairs
    assert (pr.s1, pr.s2, pr.sigma, pr.bc, pr.ka, pr.product) == (0, 1, 0.005, "rad", 0.02, 2)
    (dec,) = s.decays
    assert (dec.parent, dec.kd, tuple(dec.products)) == (2, 10.0, (0, 1))
    # mass-action start: every C is one bound A+B, so A + C = B + C = 1e5
    n_a, n_b, n_c = s.n_init
    assert n_a == n_b and n_a + n_c == 100_000 and abs(n_c / 100_000 - 0.7505) < 1e-5
    name = bench.workload_name(args)
    for part in ("L=2.55 um", "N_A=N_B=1e+05", "sigma=0.005", "D=1/1/0.5", "ka=0.02", "kd=10", "dt=1e-05",
                 "free_step"):
        assert part in name
    # a scaled system keeps the concentration
    small = bench.parse(["--n-each", "12500"])
    assert abs(bench.box_edge(small) - 2.55 / 2) < 1e-12

