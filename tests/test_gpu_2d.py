"""GPU parity of the 2D path (membrane systems, Section 4.2 of the paper) against the CPU oracle."""
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


def pair_system(tau, sigma=0.005, D=0.2, ka=0.01):
    dt = tau * sigma ** 2 / D
    return W.System(dim=2, L=1.0, dt=dt, seed=1, D=[D / 2, D / 2, 0.1], n_init=[1, 1, 0],
                    pairs=[W.PairRule(0, 1, sigma, "rad", ka, 2)])


# ka = 37.7 um^2/s gives h = 30 at D = 0.2: with tau = 0.005 (h sqrt(tau) = 2.1) p_enc still comes
# from the small-time series and p_reac from the Weber quadrature
@pytest.mark.parametrize("tau,ka", [(0.005, 0.01), (0.08, 0.01), (0.8, 0.01), (0.005, 37.7)])
def test_pair_probs_2d_fp64(tau, ka):
    system = pair_system(tau, ka=ka)
    pr = system.pairs[0]
    r0, r = W.pair_samples(400, pr.sigma, 0.2, system.dt, dim=2, seed=int(tau * 1e4))
    sim = pkg.Simulation(system, precision="fp64")
    pe, prc = sim.pair_probs(torch.tensor(r0, device="cuda"), torch.tensor(r, device="cuda"))
    pe_o, pr_o = O.pair_probs(system, r0, r)
    assert np.max(np.abs(pe.cpu().numpy() - pe_o)) <= 1e-11
    # p_reac = (g_ref - g_rad)/(g_ref - g_abs) is a ratio of two differences that both vanish far
    # from contact.  Both sides integrate each difference as one integrand (the oracle adaptively,
    # the GPU on its fixed Weber nodes), so the error of a difference is a fraction of the Weber
    # integrand's scale, ~g_free, not of the difference itself (~p_enc g_free).  The oracle's error,
    # pinned against 30-digit Laplace inversions, is <= 1e-14 p_reac / p_enc; the bound allows ten
    # times that for each side plus rounding: 1e-12 + 1e-13 / p_enc, where p_enc >= 1e-7 (a pair
    # further out fires once in 1e7 steps; below that both differences approach the integrand's
    # rounding level)
    m = pe_o >= 1e-7
    assert m.sum() > 100
    err = np.abs(prc.cpu().numpy()[m] - pr_o[m])
    assert np.all(err <= 1e-13 / pe_o[m] + 1e-12), (err.max(), (err / (1e-13 / pe_o[m] + 1e-12)).max())
    sim.close()


@pytest.mark.parametrize("tau", [0.005, 0.8])
def test_resample_2d_fp64(tau):
    system = pair_system(tau)
    sigma = system.pairs[0].sigma
    rng = np.random.default_rng(3)
    r0 = sigma * (1 + rng.uniform(0, 5 * math.sqrt(2 * tau), 40))
    r0[:5] = sigma
    u = rng.uniform(1e-6, 1, 40)
    sim = pkg.Simulation(system, precision="fp64")
    rn = sim.resample(torch.tensor(r0, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy()
    ref = np.array([O.resample2(a, b / sigma, tau) * sigma for a, b in zip(u, r0)])
    # both sides invert a quadrature of the CDF (to ~1e-13); in the tail the inversion amplifies
    # that by 1/density, so the bound is 1e-9 relative
    assert np.max(np.abs(rn - ref) / ref) <= 1e-9
    sim.close()


@pytest.mark.parametrize("tau,ka", [(0.005, 0.01), (0.08, 0.01), (0.8, 0.01), (0.005, 37.7)])
def test_pair_probs_2d_mixed_tables_within_2e6(tau, ka):
    system = pair_system(tau, ka=ka)
    pr = system.pairs[0]
    r0, r = W.pair_samples(400, pr.sigma, 0.2, system.dt, dim=2, seed=int(tau * 1e4) + 7)
    sim = pkg.Simulation(system, precision="mixed")
    pe, prc = sim.pair_probs(torch.tensor(r0, device="cuda"), torch.tensor(r, device="cuda"))
    pe_o, pr_o = O.pair_probs(system, r0, r)
    assert np.max(np.abs(pe.cpu().numpy() - pe_o)) <= 2e-6
    m = pe_o >= 1e-7
    assert np.max(np.abs(prc.cpu().numpy()[m] - pr_o[m])) <= 2e-6
    # propagator samples from the tail table: the sampled separations invert the oracle tail
    rng = np.random.default_rng(11)
    r0s = pr.sigma * (1 + rng.uniform(0, 5 * math.sqrt(2 * tau), 24))
    u = rng.uniform(0.01, 0.99, 24)
    rn = sim.resample(torch.tensor(r0s, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy()
    back = np.array([O.tail2(b / pr.sigma - 1.0, a / pr.sigma, tau) for a, b in zip(r0s, rn)])
    assert np.max(np.abs(back - u)) <= 2e-5
    sim.close()


def membrane(dt, n_each=60, L=0.3):
    return W.membrane_2d(n_each=n_each, L=L, dt=dt)


@pytest.mark.parametrize("dt,split,reach", [(1e-4, 1, 1), (1e-6, 1, 1), (1e-4, 2, 1), (1e-4, 1, 2), (1e-4, 2, 2)])
def test_stepwise_parity_2d(dt, split, reach):
    system = membrane(dt)
    sim = pkg.Simulation(system, precision="fp64", sweep_split=split, cell_reach=reach)
    assert sim.info()["reach"] == reach
    totals = {"fired": 0, "resampled": 0}
    for k in range(4):
        g0 = sim.get_state()
        o_in = O.State(g0["x"].copy(), g0["species"].copy(), g0["ids"].copy(), int(g0["step"]),
                       int(g0["next_id"][0]), 0.0)
        o_out, ost, tr = O.step(system, o_in, trace=True)
        sim.step()
        g1 = sim.get_state()
        if ost["near_threshold"] == 0:
            f = sim.last_fired()
            gf = sorted(zip(f["id_a"].tolist(), f["id_b"].tolist()))
            of = sorted(zip(tr["ida"][tr["fired"] == 1].tolist(), tr["idb"][tr["fired"] == 1].tolist()))
            assert gf == of, f"step {k}: fired sets differ"
            assert np.array_equal(g1["ids"], o_out.ids)
            assert np.array_equal(g1["species"], o_out.species)
            d = np.abs(g1["x"] - o_out.x)
            d = np.minimum(d, system.L - d)
            assert d.max(initial=0.0) <= 1e-10 * system.L
        for key in totals:
            totals[key] += ost[key]
    assert totals["fired"] > 0
    sim.close()


def test_mixed_2d_conserves():
    system = membrane(1e-4, n_each=400, L=0.8)
    sim = pkg.Simulation(system, precision="mixed")
    sim.run(20)
    c = sim.observables()["counts"][0]
    assert c[0] + c[2] == 400 and c[1] + c[2] == 400
    st = sim.get_state()
    assert np.all(st["x"][:, 2] == 0.0)
    assert np.all(np.diff(st["ids"].astype(np.int64)) > 0)
    sim.close()
