"""GPU parity on the shapes of the five workloads (scaled to sizes the oracle finishes quickly):
the irreversible 3D system's A-count trajectory, a batched ensemble of uneven replicas and the
five-species network with absorbing, reflective and radiation pairs and a unimolecular reaction
with non-interacting products."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402


def test_irreversible_count_history_matches_oracle():
    # A count per step and the survival histogram -dN_A (irreversible A + B -> C, FP64, 200 steps)
    system = W.irreversible_3d()
    sim = pkg.Simulation(system, precision="fp64")
    sim.run(200)
    hist = sim.count_history(0, 201)
    st = O.init_state(system)
    ref = [st.counts(3)]
    for _ in range(200):
        st, _ = O.step(system, st)
        ref.append(st.counts(3))
    ref = np.array(ref)
    assert np.array_equal(hist, ref)
    survival = -np.diff(hist[:, 0])
    assert survival.sum() == 1000 - hist[-1, 0] and np.all(survival >= 0)
    sim.close()


def test_uneven_ensemble_matches_oracle_per_replica():
    base = W.ensemble_3d(n_replicas=40, seed=4, n_min=24, n_max=160, c_min_uM=5.0, c_max_uM=20.0)
    system = W.System(**{**base.__dict__, "dt": 2e-5})
    sim = pkg.Simulation(system, precision="fp64")
    reps = system.replica_list()
    ostates = [O.init_state(system, r) for r in range(len(reps))]
    for _ in range(6):
        sim.step()
        ostates = [O.step(system, ostates[r], replica=r)[0] for r in range(len(reps))]
    g = sim.get_state()
    for r in range(len(reps)):
        m = g["replica"] == r
        assert np.array_equal(g["ids"][m], ostates[r].ids), r
        assert np.array_equal(g["species"][m], ostates[r].species), r
        assert np.max(np.abs(g["x"][m] - ostates[r].x), initial=0) <= 1e-12 * reps[r].L, r
        assert int(g["next_id"][r]) == ostates[r].next_id
    counts = sim.observables()["counts"]
    for r in range(len(reps)):
        assert counts[r].tolist() == ostates[r].counts(3).tolist()
    sim.close()


def test_network_stepwise_parity():
    system = W.network_3d(dt=2e-5, scale=2e-4)          # 2000 particles, L = 1.17 um
    sim = pkg.Simulation(system, precision="fp64")
    totals = {"reactions": 0, "decays": 0, "fired": 0}
    for k in range(6):
        g0 = sim.get_state()
        o_in = O.State(g0["x"].copy(), g0["species"].copy(), g0["ids"].copy(), int(g0["step"]),
                       int(g0["next_id"][0]), 0.0)
        o_out, ost = O.step(system, o_in)
        sim.step()
        g1 = sim.get_state()
        if ost["near_threshold"] == 0:
            assert np.array_equal(g1["ids"], o_out.ids), k
            assert np.array_equal(g1["species"], o_out.species), k
            d = np.abs(g1["x"] - o_out.x)
            d = np.minimum(d, system.L - d)
            assert d.max(initial=0.0) <= 1e-12 * system.L
        for key in totals:
            totals[key] += ost[key]
    assert totals["fired"] > 0
    sim.close()


def test_network_mixed_conserves_moieties():
    # A+B<->C, C+D->E, E->A+D conserve the A-moiety (A, C, E) and the D-moiety (D, E)
    system = W.network_3d(dt=1e-5, scale=2e-3)
    sim = pkg.Simulation(system, precision="mixed")
    c0 = sim.observables()["counts"][0]
    sim.run(50)
    obs = sim.observables()
    c = obs["counts"][0]
    assert c[0] + c[2] + c[4] == c0[0] + c0[2] + c0[4]
    assert c[3] + c[4] == c0[3] + c0[4]
    assert obs["stats"]["reactions"] > 0 and obs["stats"]["decays"] > 0
    sim.close()
