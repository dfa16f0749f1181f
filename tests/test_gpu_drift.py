"""GPU parity of the deterministic-force split step (drift displacement v dt before the Brownian /
reaction step) against the oracle, step by step, in 3D and 2D."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402


def drifting_3d():
    base = W.reversible_3d(n_each=400, L=(400 / (W.PER_UM3_PER_UM * 20.0)) ** (1 / 3), dt=2e-5, seed=6)
    return W.System(**{**base.__dict__, "drift": [(150.0, -40.0, 0.0), (0.0, 60.0, -90.0), (20.0, 20.0, 20.0)]})


def drifting_2d():
    base = W.membrane_2d(n_each=60, L=0.3, dt=1e-4, seed=6)
    return W.System(**{**base.__dict__, "drift": [(30.0, 0.0, 0.0), (0.0, -20.0, 0.0), (5.0, 5.0, 0.0)]})


@pytest.mark.parametrize("make", [drifting_3d, drifting_2d], ids=["3d", "2d"])
def test_drift_step_matches_oracle(make):
    system = make()
    sim = pkg.Simulation(system, precision="fp64")
    fired = 0
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
            assert d.max(initial=0.0) <= 1e-10 * system.L, k
        fired += ost["fired"]
    assert fired > 0
    sim.close()


def test_mixed_drift_conserves_and_moves():
    system = drifting_3d()
    sim = pkg.Simulation(system, precision="mixed")
    c0 = sim.observables()["counts"][0]
    sim.run(40)
    c = sim.observables()["counts"][0]
    assert c[0] + c[2] == c0[0] + c0[2] and c[1] + c[2] == c0[1] + c0[2]
    sim.close()
