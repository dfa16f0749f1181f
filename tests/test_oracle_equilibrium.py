"""Pin of the whole oracle step against the equilibrium of A + B <-> C.

With the radiation boundary of intrinsic rate ka and dissociation at rate kd placing the products
at contact, the equilibrium constant is K = ka / kd (Section 2.2.3: the reversible reaction obeys
detailed balance with the intrinsic constants).  For N0 A and N0 B in a closed box of volume V,
ideal-solution statistics give the exact law of the bound count x,
    P(x) proportional to (K / V)^x / (x! ((N0 - x)!)^2),
whose mean tends to the mass-action value x / (N0 - x)^2 = K / V for large N0.  A long oracle run
started near equilibrium must reproduce that mean.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def exact_mean_bound(n0, K, V):
    logw = np.array([x * math.log(K / V) - math.lgamma(x + 1) - 2 * math.lgamma(n0 - x + 1)
                     for x in range(n0 + 1)])
    w = np.exp(logw - logw.max())
    return float((w * np.arange(n0 + 1)).sum() / w.sum())


def test_exact_law_reduces_to_mass_action():
    # large N0: x/(N0-x)^2 = K/V; at 10 uM and K = 0.002 um^3 the bound fraction is 0.7505
    n0 = 100_000
    V = 2.55 ** 3
    f = exact_mean_bound(n0, 0.02 / 10.0, V) / n0
    c = n0 / V
    f_ma = ((2 * 0.002 * c + 1) - math.sqrt(4 * 0.002 * c + 1)) / (2 * 0.002 * c)
    assert abs(f - f_ma) < 1e-4 and abs(f_ma - 0.7505) < 5e-4


@pytest.mark.slow
def test_oracle_equilibrium_bound_count():
    n0 = 150
    L = (n0 / (W.PER_UM3_PER_UM * 10.0)) ** (1.0 / 3.0)
    system = W.reversible_3d(dt=1e-4, n_each=n0, L=L, equilibrium_start=True, seed=11)
    # 30 000 oracle steps: the free-step direction keeps this within the CPU suite's budget; the
    # full-size GPU equilibrium runs (test_gpu_equilibrium) use the exact propagator direction
    system.angle = "free_step"
    st = O.init_state(system)
    xs = []
    for _ in range(30_000):
        st, _ = O.step(system, st)
        xs.append(st.counts(3)[2])
    xs = np.array(xs[1000:], float)
    batches = xs[: len(xs) // 1000 * 1000].reshape(-1, 1000).mean(axis=1)
    sd = batches.std(ddof=1) / math.sqrt(len(batches))
    expect = exact_mean_bound(n0, 0.02 / 10.0, L ** 3)
    # allowance 0.4% of the mean for the large-step (dt = 1e-4 s) bias of the many-body
    # approximation (each particle reacts at most once per step), on top of 4 standard errors
    assert abs(xs.mean() - expect) < 4 * sd + 0.004 * expect, (xs.mean(), expect, sd)
