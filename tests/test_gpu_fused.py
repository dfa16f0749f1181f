"""The fused step (the whole step as one cooperative launch) against the separate kernels, and the
large-size code paths forced at oracle sizes.

The fused launch runs the same device code as the separate kernels, phase by phase, with grid
barriers in place of kernel boundaries, so both must give bit-identical trajectories.  The
conflict rounds on the whole grid (taken above 2048 conflict pairs) and the rounds in global
memory (short lists otherwise go to shared memory) are forced on small systems and compared with
the oracle step by step; a dense system with more than 2048 conflict pairs in one step is compared
with the oracle directly (Section 3, "Details")."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402
from test_gpu_parity import compare_states, dense_reversible, oracle_state_from  # noqa: E402


def _systems():
    drift = W.reversible_3d(dt=1e-4, seed=4, n_each=300, L=(300 / (W.PER_UM3_PER_UM * 30.0)) ** (1 / 3))
    drift.drift = [[30.0, -10.0, 5.0], [-20.0, 0.0, 10.0], [0.0, 40.0, 0.0]]
    return {
        "reversible_3d": dense_reversible(n_each=500, conc_uM=40.0, dt=1e-4),
        "membrane_2d": W.membrane_2d(n_each=600, L=0.6, dt=1e-4),
        "ensemble_3d": W.ensemble_3d(n_replicas=40, n_min=16, n_max=256, c_min_uM=20.0, c_max_uM=60.0),
        "network_3d": W.network_3d(dt=1e-4, scale=3e-4, L=4.0),
        "drift_3d": drift,
    }


def _run(system, precision, launch, steps):
    sim = pkg.Simulation(system, precision=precision, step_launch=launch)
    assert sim.info()["fused"] == (launch == "fused")
    sim.run(steps)           # graphs: two steps per launch
    sim.step()               # and a single step
    st = sim.get_state()
    obs = sim.observables()
    hist = sim.count_history(0, obs["step"] + 1)
    sim.close()
    return st, obs, hist


@pytest.mark.parametrize("name", list(_systems()))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_launch_is_bit_identical_to_separate_kernels(name, precision):
    system = _systems()[name]
    a = _run(system, precision, "fused", 24)
    b = _run(system, precision, "separate", 24)
    assert a[1]["step"] == b[1]["step"] == 25
    for key in ("ids", "species", "replica", "next_id"):
        assert np.array_equal(a[0][key], b[0][key]), key
    assert np.array_equal(a[0]["x"], b[0]["x"])
    assert a[1]["stats"] == b[1]["stats"]
    assert np.array_equal(a[1]["counts"], b[1]["counts"])
    assert np.array_equal(a[2], b[2])
    assert a[1]["stats"]["fired"] > 0


def test_fused_phase_times_are_reported():
    sim = pkg.Simulation(dense_reversible(), precision="mixed", step_launch="fused")
    sim.run(4)
    times = dict(sim.timed_step())
    for name in ("ph_prepare", "ph_scan_cells", "ph_scatter_cells", "ph_sweep", "ph_match_trivial",
                 "ph_match_resolve", "ph_compact", "k_step_fused"):
        assert name in times and times[name] >= 0.0
    assert sum(v for k, v in times.items() if k.startswith("ph_")) <= 1.05 * times["k_step_fused"] + 0.01
    sim.close()


def _stepwise_forced(system, steps, force_paths, launch, precision="fp64"):
    sim = pkg.Simulation(system, precision=precision, step_launch=launch, force_paths=force_paths)
    rounds = 0
    for k in range(steps):
        g0 = sim.get_state()
        o_out, ost, tr = O.step(system, oracle_state_from(g0), trace=True)
        sim.step()
        g1 = sim.get_state()
        f = sim.last_fired()
        if ost["near_threshold"] == 0:
            ga = sorted(zip(f["id_a"][f["accepted"]].tolist(), f["id_b"][f["accepted"]].tolist()))
            oa = sorted(zip(tr["ida"][tr["matched"] == 1].tolist(), tr["idb"][tr["matched"] == 1].tolist()))
            assert ga == oa, f"step {k}: accepted sets differ"
            compare_states(g1, o_out, system.L)
    rounds = sim.observables()["stats"]["match_rounds"]
    sim.close()
    return rounds


@pytest.mark.parametrize("launch", ["fused", "separate"])
@pytest.mark.parametrize("force", [1, 2])
def test_forced_large_size_matching_paths_match_oracle(launch, force):
    # bit 0: rounds on the whole cooperative grid; bit 1: rounds in global memory by one block
    rounds = _stepwise_forced(dense_reversible(n_each=400, conc_uM=60.0, dt=1e-4), 5, force, launch)
    assert rounds > 0


def _conflict_pairs(f):
    ends = np.concatenate([f["id_a"], f["id_b"]])
    u, c = np.unique(ends, return_counts=True)
    multi = set(u[c > 1].tolist())
    return sum(1 for a, b in zip(f["id_a"].tolist(), f["id_b"].tolist()) if a in multi or b in multi)


@pytest.mark.parametrize("dim", [2, 3])
def test_dense_step_with_many_conflicts_matches_oracle(dim):
    # absorbing A+B->C at about half a particle per contact area: ~1e4 fired pairs, several
    # thousand of them in conflicts, matched on the whole grid; tau = 0.008 (2D small-time series)
    sigma, D = 0.005, 0.1
    dt = 0.008 * sigma ** 2 / (2 * D)
    n_each = 15000
    if dim == 2:
        L = (2 * n_each * sigma ** 2 / 0.5) ** 0.5
    else:
        L = (2 * n_each * sigma ** 3 / 0.4) ** (1 / 3)
    system = W.System(dim=dim, L=L, dt=dt, seed=21, D=[D, D, D], n_init=[n_each, n_each, 0],
                      pairs=[W.PairRule(0, 1, sigma, "abs", 0.0, 2)])
    sim = pkg.Simulation(system, precision="fp64")
    g0 = sim.get_state()
    o_out, ost = O.step(system, oracle_state_from(g0))
    sim.step()
    f = sim.last_fired()
    assert _conflict_pairs(f) > 2048
    assert ost["near_threshold"] == 0
    compare_states(sim.get_state(), o_out, L)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_capacity_compaction_matches_oracle(precision):
    # a particle capacity above 2^20 takes the compaction form of large systems (256-thread tiles,
    # separate kernels); a small system with a large capacity runs it at oracle size
    system = dense_reversible(n_each=400, conc_uM=60.0, dt=1e-4)
    system.angle = "free_step"
    sim = pkg.Simulation(system, precision=precision, step_launch="separate", capacity_factor=1400.0)
    assert sim.info()["capacity"] > (1 << 20)
    ref = pkg.Simulation(system, precision=precision, step_launch="separate")
    for k in range(4):
        g0 = sim.get_state()
        o_out, ost = O.step(system, oracle_state_from(g0))
        sim.step()
        ref.step()
        g1 = sim.get_state()
        r1 = ref.get_state()
        # the same trajectory as a handle of ordinary capacity, bit for bit
        for key in ("ids", "species", "next_id"):
            assert np.array_equal(g1[key], r1[key]), key
        assert np.array_equal(g1["x"], r1["x"])
        if precision == "fp64" and ost["near_threshold"] == 0:
            compare_states(g1, o_out, system.L)
    sim.close()
    ref.close()
