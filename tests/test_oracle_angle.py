"""Pins of the oracle's exact propagation of encountered pairs (Eq. passage_prob with the full
Green's functions of Eqs. genericGF3D / genericGF).

The new separation vector of an encountered pair is drawn from G_ref - G_abs: its length from the
radial law (the n = 0 term), its angle to the start separation, given the length, from the
partial-wave series.  Independent references here:
- the free Gaussian of Eq. (gaussian), reproduced by the same partial-wave machinery with the
  boundary terms left out (3D and 2D): pins the Bessel recurrences, the (2n+1) P_n and cos(n theta)
  weights and the quadrature;
- the closed-form radial functions of Section 4.1 (3D) and the n = 0 Weber integral (2D) against
  the n = 0 term of the series;
- the boundary conditions of every partial wave (reflective: zero radial derivative at contact);
- brute-force walks: reflected (folded at the sphere) and absorbed (killed on contact, with the
  bridge crossing probability between substeps) Brownian paths of the relative coordinate, whose
  end points (R', angle) must follow 2 pi R'^2 G_ref and 2 pi R'^2 G_abs (3D), 2 R' G (2D) bin by
  bin; a planted index mistake in the 3D boundary coefficients is rejected by the same statistic;
- the sampler inverts the CDF of the conditional density, which integrates to one.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle as O
import workloads as W


@pytest.mark.parametrize("R,R0,tau", [(1.3, 1.2, 0.8), (1.1, 1.05, 0.08), (2.4, 1.6, 0.5)])
def test_free_partial_waves_reproduce_the_3d_gaussian(R, R0, tau):
    for mu in (-0.6, 0.1, 0.7, 0.99):
        d2 = R * R + R0 * R0 - 2 * R * R0 * mu
        exact = (4 * math.pi * tau) ** -1.5 * math.exp(-d2 / (4 * tau))
        assert abs(O.gf_partial(3, "free", mu, R, R0, tau) / exact - 1) < 1e-10


@pytest.mark.parametrize("R,R0,tau", [(1.3, 1.2, 0.8), (1.1, 1.05, 0.08)])
def test_free_partial_waves_reproduce_the_2d_gaussian(R, R0, tau):
    for th in (0.1, 0.9, 2.6):
        d2 = R * R + R0 * R0 - 2 * R * R0 * math.cos(th)
        exact = math.exp(-d2 / (4 * tau)) / (4 * math.pi * tau)
        assert abs(O.gf_partial(2, "free", th, R, R0, tau) / exact - 1) < 1e-8


@pytest.mark.parametrize("R,R0,tau", [(1.3, 1.2, 0.8), (1.02, 1.1, 0.08), (1.8, 1.0, 0.3)])
def test_zeroth_wave_is_the_radial_law_3d(R, R0, tau):
    s, u = math.sqrt(tau), R + R0 - 2.0
    # g_ref - g_abs of Section 4.1 (a = 1): [2 - sqrt(4 pi tau) erfcx(s + u/2s)] e^{-u^2/4tau} / (8 pi R R0 sqrt(pi tau))
    closed = (2 - math.sqrt(4 * math.pi * tau) * O.erfcx(s + u / (2 * s))) * math.exp(-u * u / (4 * tau)) / (
        8 * math.pi * R * R0 * math.sqrt(math.pi * tau))
    D = O.ang_coeffs(3, R, R0, tau)
    assert abs((1 / (4 * math.pi)) * (2 / math.pi) * D[0] / closed - 1) < 1e-11


@pytest.mark.parametrize("R,R0,tau", [(1.3, 1.2, 0.8), (1.1, 1.05, 0.08)])
def test_zeroth_wave_is_the_radial_law_2d(R, R0, tau):
    weber = O.gbc2_weber("ref", R, R0, tau, 0.0) - O.gbc2_weber("abs", R, R0, tau, 0.0)
    D = O.ang_coeffs(2, R, R0, tau)
    assert abs(D[0] / (2 * math.pi) / weber - 1) < 1e-10


@pytest.mark.parametrize("dim", [3, 2])
def test_reflective_waves_have_zero_radial_derivative_at_contact(dim):
    R0, tau, h = 1.4, 0.5, 1e-5
    v = 0.4 if dim == 3 else 1.1
    g = [O.gf_partial(dim, "ref", v, 1.0 + k * h, R0, tau) for k in (0, 1, 2)]
    slope = (-3 * g[0] + 4 * g[1] - g[2]) / (2 * h)            # one-sided, second order
    scale = abs(g[1] - g[0]) / h + abs(g[0])
    assert abs(slope) < 1e-4 * scale
    # the absorbing function vanishes at contact, the free one does not
    assert abs(O.gf_partial(dim, "abs", v, 1.0 + 1e-12, R0, tau)) < 1e-9 * abs(g[0])


# --- brute force ------------------------------------------------------------------------------

def _walks(dim, R0, tau, n_paths, n_sub, seed, mode):
    rng = np.random.default_rng(seed)
    delta = tau / n_sub
    x = np.zeros((n_paths, dim))
    x[:, 0] = R0
    alive = np.ones(n_paths, bool)
    d_prev = np.full(n_paths, R0 - 1.0)
    sd = math.sqrt(2.0 * delta)
    for _ in range(n_sub):
        x += sd * rng.standard_normal((n_paths, dim))
        r = np.sqrt(np.einsum("ij,ij->i", x, x))
        d = r - 1.0
        if mode == "ref":
            inside = d < 0                     # fold back through the sphere along the radius
            x[inside] *= ((2.0 - r[inside]) / r[inside])[:, None]
        else:
            inside = d <= 0
            both = (~inside) & (d_prev > 0)
            pc = np.where(both, np.exp(-np.maximum(d_prev, 0) * np.maximum(d, 0) / delta), 1.0)
            alive &= ~(inside | (rng.random(n_paths) < pc))
            d_prev = d
    r = np.sqrt(np.einsum("ij,ij->i", x, x))
    v = x[:, 0] / r if dim == 3 else np.abs(np.arctan2(x[:, 1], x[:, 0]))
    return r[alive], v[alive]


def _bin_probabilities(dim, which, R0, tau, redges, vedges):
    gx, gw = np.polynomial.legendre.leggauss(16)
    P = np.zeros((len(redges) - 1, len(vedges) - 1))
    for i in range(len(redges) - 1):
        a, b = redges[i], redges[i + 1]
        for xr, wr in zip(gx, gw):
            R = 0.5 * (a + b) + 0.5 * (b - a) * xr
            D = O.ang_coeffs(dim, R, R0, tau, which)
            for j in range(len(vedges) - 1):
                c, e = vedges[j], vedges[j + 1]
                vv = 0.5 * (c + e) + 0.5 * (e - c) * gx
                if dim == 3:
                    dens = 2 * math.pi * R * R * (1 / (4 * math.pi)) * (2 / math.pi) * Lg.legval(vv, (2 * np.arange(len(D)) + 1) * D)
                else:
                    n = np.arange(1, len(D))
                    dens = 2 * R * (1 / (2 * math.pi)) * (D[0] + 2 * np.cos(np.outer(vv, n)) @ D[1:])
                P[i, j] += 0.5 * (b - a) * wr * 0.5 * (e - c) * np.sum(gw * dens)
    return P


def _z_scores(dim, which, R0, tau, n_paths=120_000, n_sub=300, seed=7):
    r, v = _walks(dim, R0, tau, n_paths, n_sub, [dim, seed, int(R0 * 100)], which)
    redges = np.quantile(r, np.linspace(0, 1, 6))
    redges[0] = min(redges[0], 1.0) if which == "ref" else redges[0]
    redges[-1] = r.max() + 1e-9
    vedges = np.linspace(-1, 1, 6) if dim == 3 else np.linspace(0, math.pi, 6)
    obs, _, _ = np.histogram2d(r, v, [redges, vedges])
    ex = _bin_probabilities(dim, which, R0, tau, redges, vedges) * n_paths
    return (obs - ex) / np.sqrt(np.maximum(ex, 1.0))


@pytest.mark.parametrize("dim,which,R0,tau", [(3, "ref", 1.3, 0.5), (3, "abs", 1.3, 0.5), (2, "ref", 1.2, 0.5)])
def test_partial_wave_laws_match_brute_force_walks(dim, which, R0, tau):
    z = _z_scores(dim, which, R0, tau)
    assert np.abs(z).max() < 4.5, np.round(z, 1)


def test_brute_force_rejects_a_wrong_bessel_derivative():
    with O.planted_fault(4):
        z = _z_scores(3, "ref", 1.3, 0.5)
    assert np.abs(z).max() > 6.0


@pytest.mark.parametrize("dim,R,R0,tau", [(3, 1.2, 1.1, 0.8), (3, 1.05, 1.02, 0.08), (2, 1.2, 1.1, 0.8)])
def test_sampler_inverts_the_conditional_law(dim, R, R0, tau):
    from scipy.integrate import quad

    lo, hi = (-1.0, 1.0) if dim == 3 else (0.0, math.pi)
    assert abs(quad(lambda v: O.ang_density(dim, v, R, R0, tau), lo, hi, limit=200, epsabs=1e-12)[0] - 1) < 1e-8
    for U in (0.05, 0.5, 0.93):
        v = O.ang_sample(dim, U, R, R0, tau)
        F = quad(lambda t: O.ang_density(dim, t, R, R0, tau), lo, v, limit=200, epsabs=1e-12)[0]
        assert abs(F - U) < 1e-8


def test_step_with_exact_angles_conserves_and_keeps_order():
    system = W.reversible_3d(n_each=200, L=(200 / (W.PER_UM3_PER_UM * 40.0)) ** (1 / 3), dt=1e-4)
    assert system.angle == "exact"
    st = O.init_state(system)
    res = 0
    for _ in range(3):
        st, stats = O.step(system, st)
        res += stats["resampled"]
        c = st.counts(3)
        assert c[0] + c[2] == 200 and c[1] + c[2] == 200
        assert np.all(np.diff(st.ids.astype(np.int64)) > 0)
    assert res > 0


def test_openmp_build_gives_the_serial_result():
    # the all-core CPU baseline runs the OpenMP build: same step, same result
    if O.lib(True) is None:
        pytest.skip("no OpenMP compiler here")
    system = W.reversible_3d(n_each=600, L=(600 / (W.PER_UM3_PER_UM * 40.0)) ** (1 / 3), dt=1e-4)
    st = O.init_state(system)
    a, sa = O.step(system, st)
    b, sb = O.step(system, st, openmp=True)
    assert sa == sb
    assert np.array_equal(a.ids, b.ids) and np.array_equal(a.species, b.species)
    assert np.array_equal(a.x, b.x)


@pytest.mark.parametrize("dim", [2, 3])
def test_angle_cdf_is_the_integral_of_the_density_and_inverts_the_sampler(dim):
    # the CDF (summed from the integrated Legendre / cosine terms) against the density (summed from
    # the terms themselves) by finite differences, its end values, and the sampler's round trip
    R, R0, tau = 1.35, 1.15, 0.5
    lo, hi = (-1.0, 1.0) if dim == 3 else (0.0, math.pi)
    assert abs(O.ang_cdf(dim, lo, R, R0, tau)) < 1e-12
    assert abs(O.ang_cdf(dim, hi, R, R0, tau) - 1.0) < 1e-12
    eps = 1e-5
    for v in np.linspace(lo + 0.05, hi - 0.05, 9):
        fd = (O.ang_cdf(dim, v + eps, R, R0, tau) - O.ang_cdf(dim, v - eps, R, R0, tau)) / (2 * eps)
        assert abs(fd - O.ang_density(dim, v, R, R0, tau)) < 1e-7
    for U in (0.02, 0.4, 0.93):
        assert abs(O.ang_cdf(dim, O.ang_sample(dim, U, R, R0, tau), R, R0, tau) - U) < 1e-12
