"""Pins of the oracle's encounter probability against brute-force Brownian dynamics.

p_enc(R | R0) of the radial reading (Eq. bayes1D in its radial form, Section 4.1) is the probability
that a free relative Brownian path from separation R0 that ends at R has touched the contact
sphere (circle in 2D) during the step.  Here that conditional probability is measured directly:
many free paths of the relative coordinate (D_rel = 1 in units of a, time tau = D_rel t / a^2) are
made of fine substeps, each substep's contact crossing is detected at its end points and, between
them, with the reflection-principle probability exp(-d0 d1 / delta) of a Brownian bridge crossing a
plane at distances d0, d1 (the contact surface is flat on the scale sqrt(delta) of a substep).  The
paths are free: a touch is recorded and the path goes on.  Binned by the end separation, the
touched fraction must equal the mean of the oracle's p_enc over the same paths within the binomial
error.  Nothing of the Green's-function closed forms enters the brute force.
"""
import math

import numpy as np
import pytest

import oracle as O


def _brute_force_paths(dim, R0, tau, n_paths, n_sub, seed):
    rng = np.random.default_rng(seed)
    delta = tau / n_sub
    x = np.zeros((n_paths, dim))
    x[:, 0] = R0
    touched = np.zeros(n_paths, bool)
    d_prev = np.full(n_paths, R0 - 1.0)
    sd = math.sqrt(2.0 * delta)
    for _ in range(n_sub):
        x += sd * rng.standard_normal((n_paths, dim))
        d = np.sqrt(np.einsum("ij,ij->i", x, x)) - 1.0
        inside = d <= 0.0
        both_out = (~inside) & (d_prev > 0.0)
        p_cross = np.where(both_out, np.exp(-np.maximum(d_prev, 0.0) * np.maximum(d, 0.0) / delta), 1.0)
        touched |= inside | (rng.random(n_paths) < p_cross)
        d_prev = d
    return 1.0 + d_prev, touched


def _check_bins(R, touched, p_of_R, n_bins=6):
    out = R > 1.0
    R, touched = R[out], touched[out]
    p = p_of_R(R)
    edges = np.quantile(R, np.linspace(0.0, 1.0, n_bins + 1))
    worst = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (R >= lo) & (R <= hi)
        n = m.sum()
        expect = p[m].mean()
        sd = math.sqrt(max((p[m] * (1.0 - p[m])).sum(), 1.0)) / n
        z = abs(touched[m].mean() - expect) / sd
        worst = max(worst, z)
        assert z < 4.5, (lo, hi, touched[m].mean(), expect, sd)
    return worst


@pytest.mark.parametrize("R0,tau", [(1.3, 0.5), (1.05, 0.05)])
def test_p_enc3_is_the_touching_fraction_of_free_paths(R0, tau):
    R, touched = _brute_force_paths(3, R0, tau, 100_000, 400, seed=[3, int(R0 * 100), int(tau * 1000)])
    _check_bins(R, touched, lambda r: np.array([O.p_enc3(float(v), R0, tau) for v in r]))


def _interp(fn, lo, hi, n=240):
    grid = np.linspace(lo, hi, n)
    vals = np.array([fn(float(g)) for g in grid])
    return lambda r: np.interp(r, grid, vals)


@pytest.mark.parametrize("R0,tau", [(1.2, 0.5), (1.02, 0.004)])
def test_p_enc2_is_the_touching_fraction_of_free_paths(R0, tau):
    # tau = 0.5 takes the exact Weber-integral branch, tau = 0.004 the small-time series
    R, touched = _brute_force_paths(2, R0, tau, 100_000, 400, seed=[4, int(R0 * 100), int(tau * 1000)])
    hi = float(R.max()) + 1e-9
    p_of_R = _interp(lambda r: O.p_enc2(r, R0, tau), 1.0 + 1e-9, hi)
    _check_bins(R, touched, p_of_R)


def test_brute_force_detects_a_wrong_p_enc():
    # the same statistics reject a plausible mistake: tau built from one particle's diffusion
    # constant instead of the relative one (D_rel = D_A + D_B), i.e. p_enc at tau / 2
    R0, tau = 1.3, 0.5
    R, touched = _brute_force_paths(3, R0, tau, 100_000, 400, seed=[3, 130, 500])
    with pytest.raises(AssertionError):
        _check_bins(R, touched, lambda r: np.array([O.p_enc3(float(v), R0, tau / 2) for v in r]))
