"""Pins of the oracle's first-passage refinement (Appendix, relation to first-passage time
algorithms): bisection of an encountered pair's step with radial-bridge midpoints and p_enc of the
two halves.

* 3D closed form.  With a = 1 and unit relative diffusion the first-passage density to the sphere
  from R0 is rho(s) = (R0 - 1) / (R0 sqrt(4 pi s^3)) exp(-(R0 - 1)^2 / 4s) and the free radial
  propagator is g(R | R', u) = (R / R') (4 pi u)^(-1/2) [exp(-(R - R')^2 / 4u) - exp(-(R + R')^2 / 4u)].
  By the strong Markov property the first contact time of the paths from R0 that end at R has the
  density rho(s) g(R | 1, tau - s) on (0, tau); its integral is p_enc(R | R0) g(R | R0, tau) (R > 1)
  or g(R | R0, tau) (R <= 1), and its mass on each of the 2^K intervals is the law of the bin the
  refinement returns.  Nothing of the bisection enters these integrals.
* Brute force in 2D and 3D: free paths of fine substeps (contact crossings inside a substep by the
  Brownian-bridge reflection probability) give the first contact substep; the refinement applied to
  the same (R0, R) pairs must give the same bin distribution.
* The direction samplers against their laws: 3D von Mises-Fisher cos(theta) against its CDF, 2D
  von Mises against scipy's.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O


def _rho3(s, R0):
    return (R0 - 1.0) / (R0 * math.sqrt(4.0 * math.pi * s ** 3)) * math.exp(-(R0 - 1.0) ** 2 / (4.0 * s))


def _g3(R, Rp, u):
    c = 1.0 / math.sqrt(4.0 * math.pi * u)
    return (R / Rp) * c * (math.exp(-(R - Rp) ** 2 / (4.0 * u)) - math.exp(-(R + Rp) ** 2 / (4.0 * u)))


def _f3(s, R0, R, tau):
    if s <= 0.0 or s >= tau:
        return 0.0
    return _rho3(s, R0) * _g3(R, 1.0, tau - s)


def _bin_probs3(R0, R, tau, K):
    edges = np.linspace(0.0, tau, 2 ** K + 1)
    mass = np.array([integrate.quad(_f3, lo, hi, args=(R0, R, tau), epsabs=0, epsrel=1e-11, limit=200)[0]
                     for lo, hi in zip(edges[:-1], edges[1:])])
    return mass


@pytest.mark.parametrize("R0,R,tau", [(1.3, 1.2, 0.5), (1.05, 1.6, 0.05), (2.2, 1.8, 0.8), (1.4, 0.8, 0.2)])
def test_first_contact_density_integrates_to_p_enc(R0, R, tau):
    total = _bin_probs3(R0, R, tau, 3).sum()
    expect = (O.p_enc3(R, R0, tau) if R > 1.0 else 1.0) * _g3(R, R0, tau)
    assert total == pytest.approx(expect, rel=1e-8)


def _oracle_bins(dim, R0, R, tau, K, n, seed=11, tau_s=0.01):
    out = O.fpt_refine_batch(dim, np.full(n, R0), np.full(n, R), tau, K, seed, np.arange(n, dtype=np.uint64),
                             tau_s=tau_s)
    assert np.all(out["bin"] < 2 ** K)
    return np.bincount(out["bin"].astype(np.int64), minlength=2 ** K), out


def _chi2_p(counts, probs):
    probs = probs / probs.sum()
    exp = counts.sum() * probs
    keep = exp >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(exp[keep], exp[~keep].sum())
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    return stats.chisquare(obs, exp * obs.sum() / exp.sum()).pvalue


@pytest.mark.parametrize("R0,R,tau", [(1.3, 1.2, 0.5), (1.05, 1.6, 0.05), (2.2, 1.8, 0.8), (1.4, 0.8, 0.2)])
def test_refined_bin_follows_closed_form_3d(R0, R, tau):
    counts, _ = _oracle_bins(3, R0, R, tau, 3, 20000)
    assert _chi2_p(counts, _bin_probs3(R0, R, tau, 3)) > 1e-3


def test_deep_refinement_follows_closed_form_3d():
    R0, R, tau, K = 1.15, 1.25, 0.3, 6
    counts, out = _oracle_bins(3, R0, R, tau, K, 30000, seed=5)
    assert _chi2_p(counts, _bin_probs3(R0, R, tau, K)) > 1e-3
    # the interval ends: R_lo = R0 exactly for bin 0, R_hi = R exactly for the last bin
    assert np.all(out["R_lo"][out["bin"] == 0] == R0)
    assert np.all(out["R_hi"][out["bin"] == 2 ** K - 1] == R)


@pytest.mark.parametrize("mistake", ["tau_doubled", "ends_swapped"])
def test_closed_form_detects_a_wrong_refinement(mistake):
    R0, R, tau = 1.05, 1.6, 0.05
    probs = _bin_probs3(R0, R, tau, 3)
    if mistake == "tau_doubled":         # bridge and p_enc on the wrong time scale
        counts, _ = _oracle_bins(3, R0, R, 2.0 * tau, 3, 20000)
    else:                                # start and end separations exchanged (time reversed)
        counts, _ = _oracle_bins(3, R, R0, tau, 3, 20000)
    assert _chi2_p(counts, probs) < 1e-6


def test_levels_zero_and_contact_at_start():
    b, lo, hi, a, _, ok = O.fpt_refine(3, 1.3, 1.4, 0.5, 0, 1, 2)
    assert (b, lo, hi, a, ok) == (0, 1.3, 1.4, 0, True)
    for dim in (2, 3):                   # starting in contact: the first contact is at t = 0
        b, lo, _, a, _, ok = O.fpt_refine(dim, 1.0, 1.4, 0.5, 5, 1, 3)
        assert ok and b == 0 and lo == 1.0 and a == 5


def test_attempt_bound_is_reported():
    # a far pair (p_enc ~ 1e-9) cannot be refined within 16 draws
    b, lo, hi, a, _, ok = O.fpt_refine(3, 4.0, 4.0, 0.3, 4, 1, 4, max_attempts=16)
    assert not ok and b == 0xFFFFFFFF and math.isnan(lo) and math.isnan(hi) and a == 16


@pytest.mark.parametrize("kappa", [0.02, 1.0, 25.0, 4e4])
def test_direction_sampler_3d(kappa):
    omc = np.array([O.fpt_direction(3, kappa, 9, k, 0)[0] for k in range(4000)])
    # cos(theta) = w has density proportional to e^{kappa w} on [-1, 1], so v = 1 - w has
    # P(v <= x) = 1 - e^{-kappa x} (1 - e^{-kappa (2 - x)}) / (1 - e^{-2 kappa})
    cdf = lambda x: 1.0 - np.exp(-kappa * np.asarray(x)) * np.expm1(-kappa * (2.0 - np.asarray(x))) / math.expm1(-2.0 * kappa)
    assert np.all((omc >= 0.0) & (omc <= 2.0))
    assert stats.kstest(omc, cdf).pvalue > 1e-3


@pytest.mark.parametrize("kappa", [0.02, 1.0, 25.0, 4e4])
def test_direction_sampler_2d(kappa):
    d = [O.fpt_direction(2, kappa, 9, k, 0) for k in range(4000)]
    th = np.array([math.atan2(sn, 1.0 - omc) for omc, sn in d])
    assert np.all(th >= 0.0)
    # |theta| of a von Mises angle: CDF 2 F(theta) - 1 on [0, pi]
    cdf = lambda x: 2.0 * stats.vonmises.cdf(np.asarray(x), kappa) - 1.0
    assert stats.kstest(th, cdf).pvalue > 1e-3
    for omc, sn in d:
        assert abs((1.0 - omc) ** 2 + sn ** 2 - 1.0) < 1e-12


def _brute_force_first_contact(dim, R0, tau, n_paths, n_sub, seed):
    rng = np.random.default_rng(seed)
    delta = tau / n_sub
    x = np.zeros((n_paths, dim))
    x[:, 0] = R0
    first = np.full(n_paths, -1)
    d_prev = np.full(n_paths, R0 - 1.0)
    sd = math.sqrt(2.0 * delta)
    for i in range(n_sub):
        x += sd * rng.standard_normal((n_paths, dim))
        d = np.sqrt(np.einsum("ij,ij->i", x, x)) - 1.0
        both_out = (d > 0.0) & (d_prev > 0.0)
        p_cross = np.where(both_out, np.exp(-np.maximum(d_prev, 0.0) * np.maximum(d, 0.0) / delta), 1.0)
        hit = (first < 0) & ((d <= 0.0) | (rng.random(n_paths) < p_cross))
        first[hit] = i
        d_prev = d
    return 1.0 + d_prev, first


def _brute_force_vs_oracle(dim, R0, tau, n_paths, tau_oracle):
    K, n_sub = 3, 256
    R, first = _brute_force_first_contact(dim, R0, tau, n_paths, n_sub, seed=[dim, 17])
    m = first >= 0
    R, first = R[m], first[m]
    bf = np.bincount(first * 2 ** K // n_sub, minlength=2 ** K)
    out = O.fpt_refine_batch(dim, np.full(R.size, R0), R, tau_oracle, K, 23, np.arange(R.size, dtype=np.uint64))
    orc = np.bincount(out["bin"].astype(np.int64), minlength=2 ** K)
    table = np.vstack([bf, orc])
    return stats.chi2_contingency(table).pvalue, table


@pytest.mark.parametrize("dim,R0,tau,n_paths", [(3, 1.3, 0.5, 40000), (2, 1.2, 0.2, 8000)])
def test_refined_bin_matches_brute_force(dim, R0, tau, n_paths):
    p, table = _brute_force_vs_oracle(dim, R0, tau, n_paths, tau)
    assert p > 1e-3, table


def test_brute_force_detects_a_wrong_refinement_2d():
    # the 2D comparison rejects the refinement run on twice the step's time scale
    p, table = _brute_force_vs_oracle(2, 1.2, 0.2, 8000, 0.4)
    assert p < 1e-6, table
