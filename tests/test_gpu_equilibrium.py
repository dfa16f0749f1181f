"""Equilibrium of A + B <-> C at full size on the GPU (a property that holds at any size).

Started at the mass-action composition, the bound fraction must stay there: K = ka / kd with the
intrinsic constants (Section 2.2.3), so x / (N0 - x)^2 = K / V.  3D: 1e5 + 1e5 at 10 uM,
K = 0.002 um^3, f = 0.7505; 2D membrane: 2e5 + 2e5 on 100 um^2, K = 0.01 um^2, f = 0.800.  The
mean over the run (sampled every step from the device-side count history) must lie within 0.01 of
f; at these sizes the statistical error is below 0.001, so the bound is on the method's own
time-step bias."""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402


def mass_action_fraction(K, c):
    # f / (1 - f)^2 = K c, the root in (0, 1)
    a = K * c
    return ((2 * a + 1) - math.sqrt(4 * a + 1)) / (2 * a)


def run_fraction(system, precision, steps, n_each, bound_species=2):
    sim = pkg.Simulation(system, precision=precision)
    sim.run(steps)
    h = sim.count_history(0, steps + 1)
    sim.close()
    f = h[:, bound_species] / n_each
    return float(f[steps // 5:].mean())


@pytest.mark.parametrize("precision,dt,steps", [("mixed", 1e-6, 4000), ("mixed", 1e-5, 6000),
                                                ("mixed", 1e-4, 6000), ("fp64", 1e-5, 3000)])
def test_3d_bound_fraction_stays_at_mass_action(precision, dt, steps):
    f_ma = mass_action_fraction(0.02 / 10.0, 1e5 / 2.55 ** 3)
    f = run_fraction(W.reversible_3d(dt=dt, equilibrium_start=True), precision, steps, 100_000)
    assert abs(f - f_ma) < 0.01, (f, f_ma)


def test_2d_bound_fraction_stays_at_mass_action():
    f_ma = mass_action_fraction(0.01 / 1.0, 2e5 / 100.0)
    assert abs(f_ma - 0.8) < 1e-12
    # the free-step direction (the exact law is checked against the oracle in test_gpu_angle.py)
    system = W.membrane_2d(equilibrium_start=True)
    system.angle = "free_step"
    f = run_fraction(system, "mixed", 15000, 200_000)
    assert abs(f - f_ma) < 0.01, (f, f_ma)
