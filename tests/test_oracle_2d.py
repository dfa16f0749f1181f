"""Pins of the CPU oracle's 2D routines (Section 4.2 of the paper).

The oracle computes the boundary parts of the radial Green's functions either from the small-time
series of Eqs. (smallTEabs)/(smallTEabsII) (gamma_k by series arithmetic on a_k(nu)) or from the
exact n = 0 term of Eq. (genericGF) (a Weber integral).  Independent references here: the printed
gamma_1, gamma_2 of the paper; numerical Laplace inversion (Talbot, 20 digits) of the exact
Laplace-domain boundary terms Eqs. (absPert), (refPert), (radPert); the defining integral of
i^n erfc (Eq. iErf); the angle average of the free 2D Gaussian; conservation of probability.
"""
import math

import numpy as np
import pytest

import oracle as O

mp = pytest.importorskip("mpmath")
mp.mp.dps = 20
SP = math.sqrt(math.pi)
H = 0.00796        # h~2D of the membrane workload: 0.01 / (2 pi 0.2)


def gbc_laplace(bc, R, R0, tau, h=H):
    """Talbot inversion of the Laplace-domain boundary part (a = D = 1)."""
    def F(p):
        q = mp.sqrt(p)
        kk = mp.besselk(0, q * R0) * mp.besselk(0, q * R)
        if bc == "abs":
            return -(1 / (2 * mp.pi)) * mp.besseli(0, q) / mp.besselk(0, q) * kk
        if bc == "ref":
            return (1 / (2 * mp.pi)) * mp.besseli(1, q) / mp.besselk(1, q) * kk
        return (1 / (2 * mp.pi)) * (mp.besseli(1, q) - h / q * mp.besseli(0, q)) / \
            (mp.besselk(1, q) + h / q * mp.besselk(0, q)) * kk
    return float(mp.invertlaplace(F, tau, method="talbot"))


# --- series coefficients against the printed gamma_1, gamma_2 ------------------------------------

@pytest.mark.parametrize("R,R0,h", [(1.3, 1.1, 0.5), (2.0, 1.5, 0.0), (1.01, 1.7, 3.0)])
def test_gamma_matches_printed_coefficients(R, R0, h):
    g1abs = (2 * R * R0 - (R + R0)) / (8 * R * R0)
    g2abs = (9 * (R * R + R0 * R0) + 2 * R * R0 - 4 * R * R0 * (R + R0) + 4 * R * R * R0 * R0) / (128 * R * R * R0 * R0)
    g1rad = -(R * R0 * (6 + 16 * h) + R + R0) / (8 * R * R0)
    g2rad = (9 * (R * R + R0 * R0) + 2 * R * R0 + R * R0 * (R + R0) * (12 + 32 * h)
             + R * R * R0 * R0 * (36 + 192 * h + 256 * h * h)) / (128 * R * R * R0 * R0)
    assert O.gamma2(0, "abs", R, R0, h) == 1.0 and O.gamma2(0, "rad", R, R0, h) == 1.0
    assert abs(O.gamma2(1, "abs", R, R0, h) - g1abs) < 1e-15
    assert abs(O.gamma2(2, "abs", R, R0, h) - g2abs) < 1e-14
    assert abs(O.gamma2(1, "rad", R, R0, h) - g1rad) < 1e-14
    assert abs(O.gamma2(2, "rad", R, R0, h) - g2rad) < 1e-13
    # the reflective coefficients are the radiation ones at h = 0
    for k in range(1, 12):
        assert O.gamma2(k, "ref", R, R0, h) == O.gamma2(k, "rad", R, R0, 0.0)


# --- repeated integrals of erfc -------------------------------------------------------------------

def test_ierfc_low_orders_closed_forms():
    for z in [0.0, 0.3, 1.0, 2.5, 7.0]:
        assert O.ierfc_scaled(-1, z) == 2.0 / SP
        assert abs(O.ierfc_scaled(0, z) - O.erfcx(z)) < 1e-15
        # i^1 erfc(x) = e^{-x^2}/sqrt(pi) - x erfc(x)
        ref = float(1 / mp.sqrt(mp.pi) - z * mp.exp(mp.mpf(z) ** 2) * mp.erfc(z))
        assert abs(O.ierfc_scaled(1, z) - ref) <= 1e-13 * abs(ref) + 1e-16


@pytest.mark.parametrize("n", [2, 5, 11])
@pytest.mark.parametrize("z", [0.0, 0.7, 1.0, 3.0, 9.0])
def test_ierfc_against_defining_integral(n, z):
    # i^n erfc(z) = int_z^inf i^{n-1} erfc, iterated from i^0 = erfc: (2/sqrt(pi)/n!) int (t-z)^n e^{-t^2}
    ref = 2 / mp.sqrt(mp.pi) / mp.factorial(n) * mp.quad(lambda v: v ** n * mp.exp(-v * v - 2 * z * v), [0, 1, mp.inf])
    assert abs(O.ierfc_scaled(n, z) - float(ref)) <= 1e-12 * float(ref)


# --- Green's functions ----------------------------------------------------------------------------

def test_free_function_is_angle_average_of_gaussian():
    for R, R0, tau in [(1.3, 1.1, 0.8), (2.0, 1.0, 0.01), (1.05, 1.5, 0.08)]:
        f = lambda th: mp.exp(-(R * R + R0 * R0 - 2 * R * R0 * mp.cos(th)) / (4 * tau)) / (4 * mp.pi * tau)
        ref = mp.quad(f, [0, mp.pi, 2 * mp.pi]) / (2 * mp.pi)
        assert abs(O.gfree2(R, R0, tau) - float(ref)) < 1e-14 * float(ref) + 1e-300


@pytest.mark.parametrize("R,R0,tau", [(1.2, 1.05, 0.003)])
def test_small_time_series_matches_laplace_inversion(R, R0, tau):
    for bc in ("abs", "ref", "rad"):
        ref = gbc_laplace(bc, R, R0, tau)
        assert abs(O.gbc2_series(bc, R, R0, tau, H) - ref) < 1e-10 * max(1.0, abs(ref))


@pytest.mark.parametrize("R,R0,tau", [(1.3, 1.1, 0.8), (2.0, 1.5, 0.8), (1.0, 1.0, 0.3)])
def test_weber_integral_matches_laplace_inversion(R, R0, tau):
    for bc in ("abs", "ref", "rad"):
        ref = gbc_laplace(bc, R, R0, tau)
        assert abs(O.gbc2_weber(bc, R, R0, tau, H) - ref) < 1e-12 * max(1.0, abs(ref))


def test_series_fails_at_large_tau_so_weber_is_needed():
    # the asymptotic series is only a small-time tool: at tau = 0.8 it is far off
    ref = gbc_laplace("abs", 1.0001, 1.0001, 0.8)
    assert abs(O.gbc2_series("abs", 1.0001, 1.0001, 0.8, H) - ref) > 1e-2
    assert abs(O.gbc2_weber("abs", 1.0001, 1.0001, 0.8, H) - ref) < 1e-11


def test_reflective_weber_conserves_probability():
    from scipy.integrate import quad

    R0, tau = 1.2, 0.8
    g = lambda R: 2 * math.pi * R * (O.gbc2_weber("ref", R, R0, tau, 0.0) + O.gfree2(R, R0, tau))
    tot = quad(g, 1.0, 1.2, limit=200)[0] + quad(g, 1.2, 3.0, limit=200)[0] + quad(g, 3.0, 12.0, limit=200)[0]
    assert abs(tot - 1.0) < 1e-9


def test_absorbing_survival_matches_laplace_inversion():
    for R0, tau in [(1.1, 0.8), (3.0, 2.0)]:
        F = lambda p: (1 - mp.besselk(0, mp.sqrt(p) * R0) / mp.besselk(0, mp.sqrt(p))) / p
        ref = float(mp.invertlaplace(F, tau, method="talbot"))
        assert abs(O.S_abs2(R0, tau) - ref) < 1e-11


# --- probabilities and propagator -----------------------------------------------------------------

def test_p_enc2_regimes_agree_near_switch():
    for R, R0 in [(1.3, 1.1), (1.05, 1.4), (1.5, 1.5)]:
        ser = O.p_enc2(R, R0, 0.01, tau_s=0.02)
        web = O.p_enc2(R, R0, 0.01, tau_s=0.001)
        assert abs(ser - web) < 1e-9


def test_p_enc2_definition_and_limits():
    R, R0, tau = 1.3, 1.1, 0.8
    gabs = gbc_laplace("abs", R, R0, tau) + O.gfree2(R, R0, tau)
    assert abs(O.p_enc2(R, R0, tau) - (1 - gabs / O.gfree2(R, R0, tau))) < 1e-12
    assert O.p_enc2(0.9, 1.2, tau) == 1.0 and O.p_enc2(1.2, 1.0, tau) == 1.0
    # planar limit: p_enc -> exp(-(R-1)(R0-1)/tau) (Eq. 2pabs / bayes1D)
    a = 1e4
    d, d0, Dt = 1.0, 2.0, 1.0
    p = O.p_enc2(1 + d / a, 1 + d0 / a, Dt / a ** 2, tau_s=0.01)
    assert abs(p - math.exp(-d * d0 / Dt)) < 1e-4


def test_p_reac2_limits_and_small_time_asymptote():
    for tau in (0.8, 0.005):
        assert abs(O.p_reac2(1.2, 1.1, tau, 0.0)) < 1e-12
    # Section 4.2: p_reac = h 2 tau / (R + R0 - 2) + ... for small times
    R, R0, h = 1.3, 1.2, 0.2
    for tau in (1e-4, 1e-5):
        assert abs(O.p_reac2(R, R0, tau, h) / (h * 2 * tau / (R + R0 - 2)) - 1) < 0.05
    ref = gbc_laplace("ref", 1.2, 1.1, 0.8, 0.3) - gbc_laplace("rad", 1.2, 1.1, 0.8, 0.3)
    den = gbc_laplace("ref", 1.2, 1.1, 0.8, 0.3) - gbc_laplace("abs", 1.2, 1.1, 0.8, 0.3)
    assert abs(O.p_reac2(1.2, 1.1, 0.8, 0.3) - ref / den) < 1e-11


@pytest.mark.parametrize("R0,tau,tau_s", [(1.1, 0.8, 0.01), (1.0, 0.8, 0.01), (1.05, 0.005, 0.01)])
def test_tail2_against_density_quadrature(R0, tau, tau_s):
    from scipy.integrate import quad

    if tau <= tau_s:
        dens = lambda R: 2 * math.pi * R * (O.gbc2_series("ref", R, R0, tau, 0.0) - O.gbc2_series("abs", R, R0, tau, 0.0))
        top = R0 + 20 * math.sqrt(tau)
    else:
        dens = lambda R: 2 * math.pi * R * (O.gbc2_weber("ref", R, R0, tau, 0.0) - O.gbc2_weber("abs", R, R0, tau, 0.0))
        top = R0 + 12 * math.sqrt(tau) + 2
    norm = quad(dens, 1.0, top, limit=400, epsabs=1e-14)[0]
    if tau > tau_s:
        assert abs(norm - (1 - O.S_abs2(R0, tau))) < 1e-9
    assert abs(O.tail2(0.0, R0, tau, tau_s) - 1.0) < 1e-10
    for V in (0.02, 0.3, 1.0):
        t = 1 - quad(dens, 1.0, 1.0 + V, limit=400, epsabs=1e-14)[0] / norm
        assert abs(O.tail2(V, R0, tau, tau_s) - t) < 1e-9


def test_resample2_inverts_tail2():
    for R0, tau in [(1.1, 0.8), (1.3, 0.005)]:
        for U in (0.01, 0.5, 0.93):
            Rn = O.resample2(U, R0, tau)
            assert Rn >= 1.0
            assert abs(O.tail2(Rn - 1.0, R0, tau) - U) < 1e-11


def test_2d_step_conserves_and_keeps_order():
    import workloads as W

    base = W.membrane_2d(n_each=40, L=0.25, dt=2e-4)
    st = O.init_state(base)
    assert np.all(st.x[:, 2] == 0.0)
    for _ in range(2):
        st, stats = O.step(base, st)
        c = st.counts(3)
        assert c[0] + c[2] == 40 and c[1] + c[2] == 40
        assert np.all(np.diff(st.ids.astype(np.int64)) > 0)
        assert np.all(st.x[:, 2] == 0.0)


@pytest.mark.parametrize("h,tau,R,R0", [(30.0, 0.005, 1.02, 1.01), (100.0, 0.002, 1.1, 1.05)])
def test_p_reac2_of_strongly_reactive_pairs_matches_laplace_inversion(h, tau, R, R0):
    # h sqrt(tau) ~ 2-4.5: the small-time series of the radiation bracket no longer converges, so
    # p_reac switches to the exact Weber integral; against the Laplace-domain solution
    gr = gbc_laplace("ref", R, R0, tau, h)
    gd = gbc_laplace("rad", R, R0, tau, h)
    ga = gbc_laplace("abs", R, R0, tau, h)
    ref = (gr - gd) / (gr - ga)
    assert abs(O.p_reac2(R, R0, tau, h) - ref) < 1e-8, (O.p_reac2(R, R0, tau, h), ref)



def _golden_p_reac2():
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "p_reac2_laplace.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(float(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("R,R0,tau,h,ref", _golden_p_reac2())
def test_p_reac2_relative_accuracy_far_from_contact(R, R0, tau, h, ref):
    # Eq. (psurv_radII) is a ratio of two differences of Green's functions that both vanish far from
    # contact (their ratio stays O(1)); each difference is integrated as one integrand (the free
    # parts cancel, Section 4.2), so p_reac keeps its relative accuracy where p_enc is small.
    # Reference: Talbot inversions (30 digits) of the Laplace-domain differences
    # (tests/golden/make_p_reac2_laplace.py).  Measured: |dp|/p <= 1e-14 / p_enc (p_enc 0.95 .. 3e-8).
    pe = O.p_enc2(R, R0, tau)
    p = O.p_reac2(R, R0, tau, h)
    assert abs(p - ref) <= ref * (1e-13 + 1e-14 / pe), (p, ref, pe)
