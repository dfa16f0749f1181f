"""GPU parity of the exact propagation of encountered pairs (Eq. passage_prob with the full Green's
functions of Eqs. genericGF3D / genericGF) against the CPU oracle, pair by pair through rd_propagate.

Both sides draw the length from the radial law and the angle to the start separation from the
partial-wave law given that length, with the same uniforms.  FP64: the oracle's partial-wave
integrals are converged by panel doubling to 1e-12 of D_0, the device evaluates the base panel
count (the oracle's first estimate, itself within 1e-12), and both bisect the CDF to the last bit,
so the angle differs by about 1e-12 / f; the length differs as in rd_resample (1e-12 relative in
3D, 1e-9 in 2D, both sides inverting a quadrature there).  Bound on the new separation vector:
1e-9 relative (3D), 1e-8 (2D).  FP32 (mixed handles): the angle from the rule's table, within
1e-4 in the exact law's CDF at any draw and 2e-6 at the median draw (the drawn angle's CDF value
against the uniform it came from), and |dv| <= 2e-3 (direction components) against the FP64
oracle."""
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


def pair_system(dim, tau, sigma=0.005, D=1.0, bc="rad"):
    dt = tau * sigma ** 2 / (2 * D)
    return W.System(dim=dim, L=1.0, dt=dt, seed=1, D=[D, D, 0.5], n_init=[1, 1, 0],
                    pairs=[W.PairRule(0, 1, sigma, bc, 0.02 if dim == 3 else 0.01, 2)])


def _inputs(dim, tau, n, seed):
    rng = np.random.default_rng([seed, dim, int(tau * 1000)])
    v = rng.normal(size=(n, 3))
    if dim == 2:
        v[:, 2] = 0.0
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    R0 = 1.0 + rng.uniform(0.0, 3.0 * math.sqrt(tau), n)
    R0[:4] = 1.0                      # start at contact
    r0 = v * R0[:, None]
    r0[4] = 0.0                       # zero start separation: the x axis
    u = rng.uniform(1e-6, 1.0 - 1e-6, size=(n, 4))
    return r0, u


@pytest.mark.parametrize("dim,tau", [(3, 0.08), (3, 0.8), (3, 8.0), (2, 0.8), (2, 0.08)])
def test_propagate_fp64_matches_oracle(dim, tau):
    system = pair_system(dim, tau)
    sigma = system.pairs[0].sigma
    r0, u = _inputs(dim, tau, 96, 5)
    sim = pkg.Simulation(system, precision="fp64")
    got = sim.propagate(torch.tensor(r0 * sigma, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy() / sigma
    sim.close()
    ref = np.array([O.propagate(dim, r0[k], tau, u[k, 0], u[k, 1], u[k, 2]) for k in range(len(u))])
    scale = np.linalg.norm(ref, axis=1)
    err = np.linalg.norm(got - ref, axis=1) / scale
    assert np.all(scale >= 1.0 - 1e-12)
    assert err.max() <= (1e-9 if dim == 3 else 1e-8), err.max()


@pytest.mark.parametrize("dim,tau", [(3, 0.8), (3, 0.08), (2, 0.8)])
def test_propagate_fp32_direction_within_bound(dim, tau):
    system = pair_system(dim, tau)
    sigma = system.pairs[0].sigma
    r0, u = _inputs(dim, tau, 96, 9)
    sim = pkg.Simulation(system, precision="mixed")
    got = sim.propagate(torch.tensor(r0 * sigma, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy() / sigma
    sim.close()
    ref = np.array([O.propagate(dim, r0[k], tau, u[k, 0], u[k, 1], u[k, 2]) for k in range(len(u))])
    dg = got / np.linalg.norm(got, axis=1, keepdims=True)
    dr = ref / np.linalg.norm(ref, axis=1, keepdims=True)
    # a CDF error e moves the angle by e / f(angle): up to ~1e-3 where the density is low
    assert np.abs(dg - dr).max() <= 2e-3, np.abs(dg - dr).max()
    assert np.median(np.abs(dg - dr).max(axis=1)) <= 2e-5
    # the length comes from the mixed step's table (inverts the oracle's tail to 2e-5)
    assert np.all(np.linalg.norm(got, axis=1) >= 1.0 - 1e-6)


def _angle_to(r0, got):
    """Angle between r0 and got (atan2 of the cross and dot products: accurate near 0 and pi)."""
    cr = np.linalg.norm(np.cross(r0, got), axis=1)
    return np.arctan2(cr, np.einsum("ij,ij->i", r0, got))


@pytest.mark.parametrize("dim,tau", [(3, 0.8), (3, 0.08), (3, 8.0), (2, 0.8), (2, 0.08), (2, 8.0)])
def test_tabulated_fp32_angle_law_within_bound(dim, tau):
    # mixed handles draw the angle from the rule's table (the law's CDF value under a reference law
    # with the same concentration, interpolated in (R0, R', U)): the drawn angle's CDF value under
    # the oracle's exact law, at the drawn length, must equal the uniform it came from
    system = pair_system(dim, tau)
    sigma = system.pairs[0].sigma
    rng = np.random.default_rng([17, dim, int(tau * 1000)])
    n = 160
    v = rng.normal(size=(n, 3))
    if dim == 2:
        v[:, 2] = 0.0
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    R0 = 1.0 + rng.uniform(0.0, 5.0 * math.sqrt(2 * tau), n)     # the whole candidate shell
    R0[:16] = 1.0
    r0 = v * R0[:, None]
    u = rng.uniform(1e-6, 1.0 - 1e-6, size=(n, 4))
    u[16:32, 1] = rng.uniform(0.0, 1e-3, 16)                       # the tails of the angle law
    u[32:48, 1] = 1.0 - rng.uniform(0.0, 1e-3, 16)
    sim = pkg.Simulation(system, precision="mixed")
    got = sim.propagate(torch.tensor(r0 * sigma, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy() / sigma
    sim.close()
    Rn = np.linalg.norm(got, axis=1)
    th = _angle_to(r0, got)
    err, checked = [], 0
    for k in range(n):
        U = float(np.float32(u[k, 1]))
        kappa = Rn[k] * R0[k] / (2 * tau)
        if math.ceil(kappa + 8 * math.sqrt(kappa + 1) + 14) > 127:
            continue                       # both precisions keep the free direction there
        vk = math.cos(th[k]) if dim == 3 else th[k]
        err.append(abs(O.ang_cdf(dim, vk, Rn[k], R0[k], tau) - U))
        checked += 1
    assert checked >= n // 3
    assert max(err) <= 1e-4, max(err)
    assert np.median(err) <= 2e-6, np.median(err)


def test_propagated_angles_follow_the_partial_wave_law():
    # many draws at one start separation: the cosine of the angle to r0, binned, against the
    # oracle's law integrated over the same bins (exactness of the step's direction, FP64)
    dim, tau, R0 = 3, 0.8, 1.1
    system = pair_system(dim, tau)
    sigma = system.pairs[0].sigma
    n = 8192
    rng = np.random.default_rng(3)
    r0 = np.tile([R0, 0.0, 0.0], (n, 1))
    u = rng.uniform(size=(n, 4))
    u[:, 0] = 0.5                     # one length: R' at the radial median
    sim = pkg.Simulation(system, precision="fp64")
    got = sim.propagate(torch.tensor(r0 * sigma, device="cuda"), torch.tensor(u, device="cuda")).cpu().numpy() / sigma
    sim.close()
    Rn = np.linalg.norm(got, axis=1)
    assert np.allclose(Rn, Rn[0], rtol=1e-12)
    mu = got[:, 0] / Rn
    edges = np.linspace(-1.0, 1.0, 9)
    obs, _ = np.histogram(mu, edges)
    from scipy.integrate import quad

    ex = np.array([quad(lambda v: O.ang_density(3, v, Rn[0], R0, tau), a, b)[0] for a, b in zip(edges[:-1], edges[1:])]) * n
    z = (obs - ex) / np.sqrt(np.maximum(ex, 1.0))
    assert np.abs(z).max() < 4.5, z


def test_free_step_direction_mode_is_selectable():
    system = W.reversible_3d(dt=1e-4, seed=3, n_each=300, L=(300 / (W.PER_UM3_PER_UM * 40.0)) ** (1 / 3))
    system.angle = "free_step"
    from test_gpu_parity import compare_states, oracle_state_from

    sim = pkg.Simulation(system, precision="fp64")
    for _ in range(3):
        g0 = sim.get_state()
        o_out, ost = O.step(system, oracle_state_from(g0))
        sim.step()
        if ost["near_threshold"] == 0:
            compare_states(sim.get_state(), o_out, system.L)
    assert sim.observables()["stats"]["resampled"] > 0
    sim.close()
