"""GPU parity of the CUDA library against the CPU oracle (through the C ABI).

Bar: integer decisions (which pairs fire, which are accepted, which react, ids, species) are
bit-exact unless a uniform draw lies within 1e-9 of its probability (counted by both sides);
positions agree within 1e-12 x L in FP64; per-pair probabilities within 1e-12 (FP64) and 2e-6
(mixed FP32 p_enc).
"""
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


def dense_reversible(n_each=500, conc_uM=40.0, dt=1e-4, seed=3):
    L = (n_each / (W.PER_UM3_PER_UM * conc_uM)) ** (1 / 3)
    return W.reversible_3d(dt=dt, seed=seed, n_each=n_each, L=L)


def oracle_state_from(st):
    return O.State(st["x"].copy(), st["species"].copy(), st["ids"].copy(), int(st["step"]),
                   int(st["next_id"][0]), 0.0)


def compare_states(g, o, L, tol=1e-12):
    assert np.array_equal(g["ids"], o.ids), "ids differ"
    assert np.array_equal(g["species"], o.species), "species differ"
    assert int(g["next_id"][0]) == o.next_id
    d = np.abs(g["x"] - o.x)
    d = np.minimum(d, L - d)             # a coordinate may wrap on one side only
    assert d.max(initial=0.0) <= tol * L, f"max position difference {d.max()}"


def stepwise(system, steps, precision="fp64", check_fired=True):
    sim = pkg.Simulation(system, precision=precision)
    L = system.L
    totals = {"fired": 0, "reactions": 0, "resampled": 0, "decays": 0}
    for k in range(steps):
        g0 = sim.get_state()
        o_in = oracle_state_from(g0)
        o_out, ost, tr = O.step(system, o_in, trace=True)
        assert len(tr["ida"]) == ost["candidates"], "oracle trace truncated"
        sim.step()
        g1 = sim.get_state()
        if check_fired:
            f = sim.last_fired()
            gf = sorted(zip(f["id_a"].tolist(), f["id_b"].tolist()))
            of = sorted(zip(tr["ida"][tr["fired"] == 1].tolist(), tr["idb"][tr["fired"] == 1].tolist()))
            if ost["near_threshold"] == 0:
                assert gf == of, f"step {k}: fired sets differ"
                ga = sorted(zip(f["id_a"][f["accepted"]].tolist(), f["id_b"][f["accepted"]].tolist()))
                oa = sorted(zip(tr["ida"][tr["matched"] == 1].tolist(), tr["idb"][tr["matched"] == 1].tolist()))
                assert ga == oa, f"step {k}: accepted sets differ"
                # p_enc of the fired pairs
                gp = dict(zip(zip(f["id_a"].tolist(), f["id_b"].tolist()), f["p_enc"].tolist()))
                op = dict(zip(zip(tr["ida"].tolist(), tr["idb"].tolist()), tr["p_enc"].tolist()))
                for key, p in gp.items():
                    assert abs(p - op[key]) <= 1e-12
        if ost["near_threshold"] == 0:
            compare_states(g1, o_out, L)
        for key in totals:
            totals[key] += ost[key]
    obs = sim.observables()
    sim.close()
    return totals, obs


def test_initial_positions_bit_exact():
    system = W.irreversible_3d()
    sim = pkg.Simulation(system, precision="fp64")
    g = sim.get_state()
    o = O.init_state(system)
    assert np.array_equal(g["ids"], o.ids)
    assert np.array_equal(g["species"], o.species)
    assert np.array_equal(g["x"], o.x)
    obs = sim.observables()
    assert obs["counts"][0].tolist() == [1000, 1000, 0]
    sim.close()


@pytest.mark.parametrize("tau", [0.006, 0.08, 0.8, 8.0])
def test_pair_probs_fp64(tau):
    sigma, D = 0.005, 2.0
    dt = tau * sigma ** 2 / D
    system = W.System(dim=3, L=1.0, dt=dt, seed=1, D=[1.0, 1.0, 0.5], n_init=[1, 1, 0],
                      pairs=[W.PairRule(0, 1, sigma, "rad", 0.02, 2)])
    r0, r = W.pair_samples(20000, sigma, D, dt, seed=int(tau * 1000))
    sim = pkg.Simulation(system, precision="fp64")
    pe, pr = sim.pair_probs(torch.tensor(r0, device="cuda"), torch.tensor(r, device="cuda"))
    pe_o, pr_o = O.pair_probs(system, r0, r)
    assert np.max(np.abs(pe.cpu().numpy() - pe_o)) <= 1e-12
    assert np.max(np.abs(pr.cpu().numpy() - pr_o)) <= 1e-12
    sim.close()


@pytest.mark.parametrize("tau", [0.006, 0.08, 0.8, 8.0])
def test_pair_probs_mixed_within_2e6(tau):
    sigma, D = 0.005, 2.0
    dt = tau * sigma ** 2 / D
    system = W.System(dim=3, L=1.0, dt=dt, seed=1, D=[1.0, 1.0, 0.5], n_init=[1, 1, 0],
                      pairs=[W.PairRule(0, 1, sigma, "rad", 0.02, 2)])
    r0, r = W.pair_samples(20000, sigma, D, dt, seed=int(tau * 1000) + 1)
    sim = pkg.Simulation(system, precision="mixed")
    pe, pr = sim.pair_probs(torch.tensor(r0, device="cuda"), torch.tensor(r, device="cuda"))
    pe_o, pr_o = O.pair_probs(system, r0, r)
    err = np.max(np.abs(pe.cpu().numpy() - pe_o))
    assert err <= 2e-6, err
    err_r = np.max(np.abs(pr.cpu().numpy() - pr_o))      # p_reac from the per-run FP32 table
    assert err_r <= 2e-6, err_r
    sim.close()


@pytest.mark.parametrize("tau", [0.08, 0.8, 8.0])
def test_resample_matches_oracle(tau):
    sigma, D = 0.005, 2.0
    dt = tau * sigma ** 2 / D
    system = W.System(dim=3, L=1.0, dt=dt, seed=1, D=[1.0, 1.0, 0.5], n_init=[1, 1, 0],
                      pairs=[W.PairRule(0, 1, sigma, "rad", 0.02, 2)])
    rng = np.random.default_rng(5)
    r0 = sigma * (1 + rng.uniform(0, 5 * math.sqrt(2 * tau), 3000))
    r0[:300] = sigma
    u = rng.uniform(1e-12, 1, 3000)
    sim = pkg.Simulation(system, precision="fp64")
    rn = sim.resample(torch.tensor(r0, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy()
    ref = np.array([O.resample3(a, b / sigma, tau) * sigma for a, b in zip(u, r0)])
    assert np.max(np.abs(rn - ref) / ref) <= 1e-12
    sim.close()


@pytest.mark.parametrize("tau", [0.08, 0.8, 8.0])
def test_mixed_resample_inverts_the_oracle_tail(tau):
    # the mixed step samples the propagator from an FP32 inverse table and one Newton step: the
    # oracle's tail at the sampled separation must give back the uniform (draws as in the step,
    # U >= 2^-24)
    sigma, D = 0.005, 2.0
    dt = tau * sigma ** 2 / D
    system = W.System(dim=3, L=1.0, dt=dt, seed=1, D=[1.0, 1.0, 0.5], n_init=[1, 1, 0],
                      pairs=[W.PairRule(0, 1, sigma, "rad", 0.02, 2)])
    rng = np.random.default_rng(6)
    r0 = sigma * (1 + rng.uniform(0, 5 * math.sqrt(2 * tau), 2000))
    r0[:200] = sigma
    u = rng.uniform(2.0 ** -24, 1, 2000)
    sim = pkg.Simulation(system, precision="mixed")
    rn = sim.resample(torch.tensor(r0, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy()
    back = np.array([O.tail3(b / sigma - 1.0, a / sigma, tau) for a, b in zip(r0, rn)])
    assert np.max(np.abs(back - u)) <= 2e-5
    sim.close()


def test_stepwise_parity_irreversible():
    totals, obs = stepwise(W.irreversible_3d(), 30)
    assert totals["fired"] > 0


def test_stepwise_parity_reversible_dense():
    totals, obs = stepwise(dense_reversible(), 25)
    assert totals["reactions"] > 0 and totals["decays"] > 0 and totals["resampled"] > 0


def test_stepwise_parity_absorbing_and_reflective():
    base = dense_reversible(n_each=400, conc_uM=60.0)
    system = W.System(**{**base.__dict__, "pairs": [W.PairRule(0, 1, 0.005, "abs", 0.0, 2),
                                                      W.PairRule(2, 2, 0.006, "ref")]})
    totals, _ = stepwise(system, 20)
    assert totals["reactions"] > 0


def test_whole_trajectory_matches():
    system = W.irreversible_3d()
    sim = pkg.Simulation(system, precision="fp64")
    o = O.init_state(system)
    first_div = None
    for k in range(60):
        o, ost = O.step(system, o)
        sim.step()
        g = sim.get_state()
        same = np.array_equal(g["ids"], o.ids) and np.max(np.abs(g["x"] - o.x), initial=0) <= 1e-9
        if not same and first_div is None:
            first_div = k
    sim.close()
    assert first_div is None, f"first divergence at step {first_div}"


def test_graph_run_equals_single_steps():
    system = dense_reversible(n_each=300)
    a = pkg.Simulation(system, precision="fp64")
    b = pkg.Simulation(system, precision="fp64")
    a.run(11)
    for _ in range(11):
        b.step()
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(sa["ids"], sb["ids"]) and np.array_equal(sa["x"], sb["x"])
    oa, ob = a.observables(), b.observables()
    assert oa["step"] == ob["step"] == 11
    assert np.array_equal(oa["counts"], ob["counts"])
    a.close()
    b.close()


def test_replicas_match_oracle_per_replica():
    base = dense_reversible(n_each=200, dt=2e-5)
    reps = [W.Replica(base.L, [200, 200, 0]), W.Replica(base.L * 1.3, [150, 120, 30]),
            W.Replica(base.L * 0.9, [90, 90, 10])]
    system = W.System(**{**base.__dict__, "replicas": reps})
    sim = pkg.Simulation(system, precision="fp64")
    g = sim.get_state()
    ostates = [O.init_state(system, r) for r in range(3)]
    for k in range(10):
        for r in range(3):
            ostates[r], _ = O.step(system, ostates[r], replica=r)
        sim.step()
    g = sim.get_state()
    for r in range(3):
        m = g["replica"] == r
        assert np.array_equal(g["ids"][m], ostates[r].ids)
        assert np.array_equal(g["species"][m], ostates[r].species)
        assert np.max(np.abs(g["x"][m] - ostates[r].x), initial=0) <= 1e-12 * reps[r].L
    sim.close()


def test_mixed_step_conserves_and_tracks_fp64():
    system = dense_reversible(n_each=2000, conc_uM=20.0, dt=1e-5)
    sim = pkg.Simulation(system, precision="mixed")
    sim.run(200)
    obs = sim.observables()
    c = obs["counts"][0]
    assert c[0] + c[2] == 2000 and c[1] + c[2] == 2000
    st = sim.get_state()
    assert np.all(np.diff(st["ids"].astype(np.int64)) > 0)
    assert np.all((st["x"] >= 0) & (st["x"] < system.L))
    sim.close()


def test_set_state_then_step_matches_oracle():
    system = dense_reversible(n_each=300)
    o = O.init_state(system)
    for _ in range(5):
        o, _ = O.step(system, o)
    sim = pkg.Simulation(system, precision="fp64")
    sim.set_state(o.x, o.species, o.ids, next_id=[o.next_id], step=o.step)
    o2, _ = O.step(system, o)
    sim.step()
    compare_states(sim.get_state(), o2, system.L)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cell_layout_and_autotune_do_not_change_results(precision):
    # every decision is keyed by particle ids, so the cell edge, the block shapes and the
    # autotuner's choice must leave the trajectory bit-identical
    system = dense_reversible(n_each=1500, conc_uM=20.0, dt=2e-5)
    states = []
    for cf, split in ((1.0, 1), (2.5, 1), (None, 0), ("tune", 0), (1.0, 2), (2.5, 2), (None, 2)):
        sim = pkg.Simulation(system, precision=precision, cell_factor=cf, sweep_split=split)
        if split == 2:
            assert sim.info()["sweep_split"] == 5
        sim.run(9)
        states.append(sim.get_state())
        sim.close()
    for st in states[1:]:
        assert np.array_equal(st["ids"], states[0]["ids"])
        assert np.array_equal(st["species"], states[0]["species"])
        assert np.array_equal(st["x"], states[0]["x"])
