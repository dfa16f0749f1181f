"""Host-side checks of the benchmark's bookkeeping (no GPU): every kernel that the step launches
has an algorithmic byte count, and the launch count per step matches the timer marks."""
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
