"""Degenerate systems on the GPU against the oracle: no particles, no pair rules (diffusion and
decay only), decay into nothing until the box is empty, replicas that start empty, and a single
isolated pair."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402


def stepwise(system, steps, precision="fp64", tol=1e-12):
    sim = pkg.Simulation(system, precision=precision)
    st = O.init_state(system)
    for k in range(steps):
        sim.step()
        st, _ = O.step(system, st)
        g = sim.get_state()
        assert np.array_equal(g["ids"], st.ids), k
        assert np.array_equal(g["species"], st.species), k
        d = np.abs(g["x"] - st.x)
        d = np.minimum(d, system.L - d)
        assert d.max(initial=0.0) <= tol * system.L, k
    out = sim.observables()
    sim.close()
    return out


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_empty_system_steps(dim, precision):
    system = W.System(dim=dim, L=1.0, dt=1e-5, seed=1, D=[1.0, 1.0, 0.5], n_init=[0, 0, 0],
                      pairs=[W.PairRule(0, 1, 0.01, "rad", 0.05, 2)], decays=[W.Decay(2, 10.0, (0, 1))])
    sim = pkg.Simulation(system, precision=precision)
    sim.run(6)
    obs = sim.observables()
    assert obs["step"] == 6 and obs["counts"].sum() == 0
    assert sim.get_state()["ids"].size == 0
    sim.close()


def test_no_pair_rules_diffusion_and_decay():
    system = W.System(dim=3, L=0.8, dt=1e-4, seed=2, D=[0.5, 2.0], n_init=[300, 0], pairs=[],
                      decays=[W.Decay(0, 800.0, (1,))])
    obs = stepwise(system, 8)
    assert obs["stats"]["decays"] > 0


def test_decay_into_nothing_empties_the_box():
    system = W.System(dim=3, L=0.5, dt=1e-3, seed=3, D=[1.0], n_init=[200], pairs=[],
                      decays=[W.Decay(0, 3000.0, ())])
    obs = stepwise(system, 6)
    assert obs["counts"].sum() == 0


def test_replicas_that_start_empty():
    reps = [W.Replica(0.4, [60, 60, 0]), W.Replica(0.5, [0, 0, 0]), W.Replica(0.3, [0, 40, 0]),
            W.Replica(0.45, [50, 50, 20])]
    base = W.reversible_3d(dt=2e-5, seed=4, n_each=60, L=0.4)
    system = W.System(**{**base.__dict__, "replicas": reps})
    sim = pkg.Simulation(system, precision="fp64")
    states = [O.init_state(system, r) for r in range(len(reps))]
    for _ in range(5):
        sim.step()
        states = [O.step(system, states[r], replica=r)[0] for r in range(len(reps))]
    g = sim.get_state()
    for r in range(len(reps)):
        m = g["replica"] == r
        assert np.array_equal(g["ids"][m], states[r].ids), r
        assert np.max(np.abs(g["x"][m] - states[r].x), initial=0.0) <= 1e-12 * reps[r].L, r
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_single_isolated_pair(dim):
    if dim == 3:
        system = W.System(dim=3, L=0.2, dt=2e-5, seed=5, D=[1.0, 1.0, 0.5], n_init=[1, 1, 0],
                          pairs=[W.PairRule(0, 1, 0.02, "rad", 0.5, 2)], decays=[W.Decay(2, 50.0, (0, 1))])
    else:
        system = W.System(dim=2, L=0.2, dt=1e-4, seed=5, D=[0.1, 0.1, 0.1], n_init=[1, 1, 0],
                          pairs=[W.PairRule(0, 1, 0.02, "rad", 0.5, 2)], decays=[W.Decay(2, 50.0, (0, 1))])
    stepwise(system, 40, tol=1e-10)
