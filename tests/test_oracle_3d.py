"""Pins of the CPU oracle's 3D routines against what the paper and the mathematics fix.

The radial Green's functions of Section 4.1 are typed here in mpmath only as the object under
test of the *first* group of checks: they are pinned by their defining problem (the radial
diffusion equation of Eq. (smol_bc), the boundary conditions (g_abs_bc), (g_ref_bc), (robin_bc)
and conservation of probability), and the free radial function by a numerical angular average of
the free Gaussian, Eq. (gaussian).  The oracle's closed forms (p_enc, p_reac, the propagator's tail,
survival) are then checked against quadratures of those pinned functions, against the planar 1D
limit of Eq. (2pabs)/(bayes1D), and, end to end, against the exact survival of isolated pairs.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- the paper's radial functions (Section 4.1), a = 1, tau = D t / a^2 -------------------------

def g3(bc, R, R0, tau, h=0.0):
    R, R0, tau = mp.mpf(R), mp.mpf(R0), mp.mpf(tau)
    pref = 1 / (8 * mp.pi * R * R0 * mp.sqrt(mp.pi * tau))
    u = R + R0 - 2
    e1 = mp.exp(-(R - R0) ** 2 / (4 * tau))
    e2 = mp.exp(-u ** 2 / (4 * tau))
    if bc == "abs":
        return pref * (e1 - e2)
    k = 1 + (mp.mpf(h) if bc == "rad" else 0)
    s = mp.sqrt(tau)
    return pref * (e1 + e2 - k * mp.sqrt(4 * mp.pi * tau) * mp.exp(k ** 2 * tau + u * k)
                   * mp.erfc(k * s + u / (2 * s)))


def gfree3_by_angle(R, R0, tau):
    """(1/4pi) * integral over directions of the free 3D Gaussian (4 pi tau)^(-3/2) e^{-|r-r0|^2/4tau}."""
    R, R0, tau = mp.mpf(R), mp.mpf(R0), mp.mpf(tau)
    f = lambda mu: (4 * mp.pi * tau) ** (-1.5) * mp.exp(-(R * R + R0 * R0 - 2 * R * R0 * mu) / (4 * tau))
    return mp.quad(f, [-1, 1]) / 2


POINTS = [(1.3, 1.1, 0.2, 0.199), (1.01, 1.0, 8.0, 0.159), (2.0, 1.5, 0.08, 0.159),
          (1.05, 1.2, 0.8, 5.0), (1.7, 2.2, 0.006, 0.05)]


# --- pins of the paper's functions themselves --------------------------------------------------

@pytest.mark.parametrize("bc", ["abs", "ref", "rad"])
@pytest.mark.parametrize("R,R0,tau,h", POINTS[:4])
def test_radial_g_solves_diffusion_equation(bc, R, R0, tau, h):
    # radial Laplacian in 3D: g_t = g_RR + (2/R) g_R   (Eq. smol_bc in scaled variables)
    f = lambda RR, tt: g3(bc, RR, R0, tt, h)
    gt = mp.diff(lambda tt: f(R, tt), tau)
    gR = mp.diff(lambda RR: f(RR, tau), R)
    gRR = mp.diff(lambda RR: f(RR, tau), R, 2)
    resid = gt - (gRR + 2 / mp.mpf(R) * gR)
    assert abs(resid) <= 1e-18 * (abs(gt) + abs(gRR) + 1e-30)


@pytest.mark.parametrize("R0,tau,h", [(1.1, 0.2, 0.199), (1.5, 0.8, 0.159), (2.0, 0.05, 3.0)])
def test_radial_g_boundary_conditions(R0, tau, h):
    assert abs(g3("abs", 1, R0, tau)) < mp.mpf(10) ** -25                        # Eq. (g_abs_bc)
    dref = mp.diff(lambda RR: g3("ref", RR, R0, tau), 1)
    assert abs(dref) < mp.mpf(10) ** -20 * abs(g3("ref", 1, R0, tau))              # Eq. (g_ref_bc)
    drad = mp.diff(lambda RR: g3("rad", RR, R0, tau, h), 1)
    # Eq. (robin_bc): 4 pi a^2 D dG/dr = kappa_a G  ->  dg/dR = h g at R = 1
    assert abs(drad - h * g3("rad", 1, R0, tau, h)) < mp.mpf(10) ** -20 * abs(drad)


@pytest.mark.parametrize("R0,tau", [(1.1, 0.2), (1.5, 0.8), (3.0, 0.05)])
def test_reflective_g_conserves_probability(R0, tau):
    tot = mp.quad(lambda R: 4 * mp.pi * R * R * g3("ref", R, R0, tau), [1, R0, mp.inf])
    assert abs(tot - 1) < 1e-20


# --- oracle closed forms against the pinned functions -----------------------------------------

@pytest.mark.parametrize("R,R0,tau,h", POINTS)
def test_p_enc3_is_one_minus_gabs_over_gfree(R, R0, tau, h):
    ref = 1 - g3("abs", R, R0, tau) / gfree3_by_angle(R, R0, tau)
    assert abs(O.p_enc3(R, R0, tau) - float(ref)) < 1e-14


def test_p_enc3_overlap_and_contact():
    assert O.p_enc3(0.7, 1.2, 0.2) == 1.0
    assert O.p_enc3(1.0, 1.2, 0.2) == 1.0
    assert O.p_enc3(1.4, 1.0, 0.2) == 1.0          # started at contact: met the boundary
    assert O.p_enc3(1.4, 0.9, 0.2) == 1.0          # start inside is clamped to contact


@pytest.mark.parametrize("d,d0,Dt", [(1.0, 2.0, 1.0), (0.3, 0.5, 0.2), (2.0, 2.0, 4.0)])
def test_p_enc3_planar_limit_is_1d_reflection_formula(d, d0, Dt):
    # Eq. (2pabs) and (bayes1D): with the boundary at distance d0 from the start and d from the
    # end, 1 - p_enc = f_W / free = 1 - exp(-d d0/(D t)) (variance 2 D t per coordinate).
    a = 1e5
    R, R0, tau = 1 + d / a, 1 + d0 / a, Dt / a ** 2
    x, x0, bnd = 0.0, 0.0, d0
    xend = bnd - d
    sig2 = 2 * Dt
    free = math.exp(-(xend - x0) ** 2 / (2 * sig2))
    img = math.exp(-(xend - 2 * bnd + x0) ** 2 / (2 * sig2))
    ref = 1 - (free - img) / free
    assert abs(O.p_enc3(R, R0, tau) - ref) < 1e-9


@pytest.mark.parametrize("R,R0,tau,h", POINTS)
def test_p_reac3_matches_green_function_ratio(R, R0, tau, h):
    with mp.workdps(120):   # g_ref - g_abs cancels the common exp(-(R-R0)^2/4tau) term
        ref = (g3("ref", R, R0, tau) - g3("rad", R, R0, tau, h)) / (g3("ref", R, R0, tau) - g3("abs", R, R0, tau))
    assert abs(O.p_reac3(R, R0, tau, h) - float(ref)) < 1e-13


def test_p_reac3_limits():
    # Section 2.2.3: kappa_a -> infinity gives the absorbing method (p_reac -> 1), kappa_a -> 0
    # the reflective one (p_reac -> 0).
    for R, R0, tau, _ in POINTS:
        assert O.p_reac3(R, R0, tau, 0.0) == 0.0
        assert abs(O.p_reac3(R, R0, tau, 1e12) - 1.0) < 1e-5


@pytest.mark.parametrize("R0,tau", [(1.0, 0.2), (1.1, 0.2), (1.8, 0.8), (1.2, 0.08), (1.0, 8.0)])
def test_tail3_matches_quadrature_of_propagator(R0, tau):
    dens = lambda R: 4 * mp.pi * R * R * (g3("ref", R, R0, tau) - g3("abs", R, R0, tau))
    norm = mp.quad(dens, [1, R0, mp.inf])
    # total = 1 - S_abs (the encountered fraction)
    S_abs = 1 - mp.quad(lambda R: 4 * mp.pi * R * R * (g3("ref", R, R0, tau) - g3("abs", R, R0, tau)), [1, mp.inf])
    assert abs(float(norm) - (1 - O.S_abs3(R0, tau))) < 1e-13
    assert abs(float(1 - S_abs) - float(norm)) < 1e-15
    for V in [0.0, 0.05, 0.3, 1.0, 2.5]:
        tail = mp.quad(dens, [1 + V, max(1 + V, R0) + 1e-30, mp.inf]) / norm
        assert abs(O.tail3(V, R0, tau) - float(tail)) < 1e-12


@pytest.mark.parametrize("R0,tau", [(1.0, 0.2), (1.3, 0.8), (1.05, 0.08)])
def test_resample3_inverts_tail(R0, tau):
    for U in [1e-9, 0.01, 0.3, 0.5, 0.77, 0.999999]:
        Rn = O.resample3(U, R0, tau)
        assert Rn >= 1.0
        assert abs(O.tail3(Rn - 1.0, R0, tau) - U) < 1e-13


@pytest.mark.parametrize("R0,tau,h", [(1.1, 0.2, 0.199), (1.5, 0.8, 0.159), (1.02, 0.08, 2.0)])
def test_survival_matches_quadrature(R0, tau, h):
    S_rad = mp.quad(lambda R: 4 * mp.pi * R * R * g3("rad", R, R0, tau, h), [1, R0, mp.inf])
    S_abs = mp.quad(lambda R: 4 * mp.pi * R * R * g3("abs", R, R0, tau), [1, R0, mp.inf])
    assert abs(O.S_rad3(R0, tau, h) - float(S_rad)) < 1e-13
    assert abs(O.S_abs3(R0, tau) - float(S_abs)) < 1e-13


def test_one_step_encounter_fraction_is_one_minus_S_abs():
    # integrating p_enc against the free propagator over all end points (overlaps included)
    # gives the fraction of paths that met the boundary: 1 - S_abs(tau | R0).
    R0, tau = 1.2, 0.3
    inner = mp.quad(lambda R: 4 * mp.pi * R * R * gfree3_by_angle(R, R0, tau), [0, 1])
    outer = mp.quad(lambda R: 4 * mp.pi * R * R * gfree3_by_angle(R, R0, tau) * O.p_enc3(float(R), R0, tau),
                    [1, R0, R0 + 12 * math.sqrt(tau)])
    assert abs(float(inner + outer) - (1 - O.S_abs3(R0, tau))) < 1e-10


# --- random streams ----------------------------------------------------------------------------

def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert O.philox(v[0:4], v[4:6]) == tuple(v[6:10])


def test_u52_open_interval_and_exact():
    assert O.u52(0, 0) == 0.5 * 2.0 ** -52
    assert O.u52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -52
    assert 0.0 < O.u52(0, 0) < O.u52(0xFFFFFFFF, 0xFFFFFFFF) < 1.0


def test_erfcx_against_mpmath():
    for x in np.concatenate([np.linspace(0, 6, 61), [7.5, 10, 30, 100, 1e3, 1e6], [-0.5, -2.0]]):
        ref = mp.exp(mp.mpf(x) ** 2) * mp.erfc(x)
        assert abs(O.erfcx(x) - float(ref)) <= 4e-15 * float(ref)


# --- whole step ----------------------------------------------------------------------------------

def _run(system, state, n):
    for _ in range(n):
        state, _ = O.step(system, state)
    return state


def test_displacement_moments():
    sys_ = W.System(dim=3, L=10.0, dt=1e-3, seed=5, D=[1.0], n_init=[20000], pairs=[])
    st0 = O.init_state(sys_)
    st1, _ = O.step(sys_, st0)
    d = (st1.x - st0.x + 5.0) % 10.0 - 5.0
    ell2 = 2 * 1.0 * 1e-3
    assert abs(d.mean()) < 4 * math.sqrt(ell2 / (3 * 20000))
    assert abs(d.var() / ell2 - 1) < 0.03
    # fourth moment of a normal: 3
    assert abs((d ** 4).mean() / ell2 ** 2 - 3) < 0.15


def test_init_positions_uniform_and_ordered():
    sys_ = W.irreversible_3d()
    st = O.init_state(sys_)
    assert st.n == 2000 and np.all(st.ids == np.arange(2000))
    assert np.all((st.x >= 0) & (st.x < sys_.L))
    assert abs(st.x.mean() - 0.5) < 0.02


def _isolated_pair_reaction_fraction(n_pairs, R0, steps, tau_target=0.2, h=0.199, seeds=(1,)):
    sigma, D = 0.01, 1.0
    dt = tau_target * sigma ** 2 / (2 * D)
    ka = h * 4 * math.pi * sigma * 2 * D
    reacted = 0
    total = 0
    for seed in seeds:
        sys_, pos, sp = W.isolated_pairs_3d(n_pairs, R0, sigma=sigma, D=D, ka=ka, dt=dt, seed=seed,
                                            spacing=0.2)
        # the reacted fraction of isolated pairs depends only on the radial process (the direction
        # of a resampled separation changes no later radial law), so the cheaper free-step
        # direction serves here
        sys_.angle = "free_step"
        st = O.State(pos.copy(), sp.copy(), np.arange(2 * n_pairs, dtype=np.uint32), 0, 2 * n_pairs, 0.0)
        st = _run(sys_, st, steps)
        reacted += int(np.sum(st.species == 2))
        total += n_pairs
    return reacted / total, total, dt * 2 * D / sigma ** 2, h


@pytest.mark.slow
@pytest.mark.parametrize("steps", [1, 3])
def test_isolated_pair_survival_is_exact(steps):
    # For an isolated pair the radial reading makes one step exact in distribution, so after n
    # steps the reacted fraction equals 1 - S_rad(n tau | R0) (Eq. SurvRad), up to the cut-off.
    R0 = 1.1
    frac, m, tau, h = _isolated_pair_reaction_fraction(4000, R0, steps, seeds=(1, 2, 3, 4, 5))
    S = mp.quad(lambda R: 4 * mp.pi * R * R * g3("rad", R, R0, steps * tau, h), [1, R0, mp.inf])
    p = 1 - float(S)
    sd = math.sqrt(p * (1 - p) / m)
    assert abs(frac - p) < 4 * sd, (frac, p, sd)


def test_absorbing_limit_equals_abs_decisions():
    # Section 2.2.3: radiation with kappa_a -> infinity reproduces the absorbing method.
    base = W.irreversible_3d()
    big = W.System(**{**base.__dict__, "pairs": [W.PairRule(0, 1, 0.01, "rad", 1e12, 2)]})
    ab = W.System(**{**base.__dict__, "pairs": [W.PairRule(0, 1, 0.01, "abs", 0.0, 2)]})
    s1 = O.init_state(big)
    s2 = O.init_state(ab)
    for _ in range(5):
        s1, st1 = O.step(big, s1)
        s2, st2 = O.step(ab, s2)
        assert st1["reactions"] == st2["reactions"]
        assert np.array_equal(s1.ids, s2.ids)
        assert np.allclose(s1.x, s2.x, atol=1e-12)


def test_reversible_step_conserves_and_matches():
    sys_ = W.reversible_3d(n_each=300, L=(300 / (W.PER_UM3_PER_UM * 10.0)) ** (1 / 3))
    st = O.init_state(sys_)
    for _ in range(50):
        st, stats = O.step(sys_, st, trace=False)
        c = st.counts(3)
        assert c[0] + c[2] == 300 and c[1] + c[2] == 300
        assert np.all(np.diff(st.ids.astype(np.int64)) > 0)        # array stays id-sorted
        assert stats["matched"] <= stats["fired"] <= stats["candidates"]


def test_matching_is_greedy_by_key():
    sys_ = W.reversible_3d(n_each=400, L=(400 / (W.PER_UM3_PER_UM * 30.0)) ** (1 / 3), dt=1e-4)
    st = O.init_state(sys_)
    st, stats, tr = O.step(sys_, st, trace=True)
    assert stats["candidates"] == len(tr["ida"])
    f = tr["fired"].astype(bool)
    m = tr["matched"].astype(bool)
    assert np.all(f[m])
    ids = np.concatenate([tr["ida"][m], tr["idb"][m]])
    assert len(ids) == len(np.unique(ids))                    # each particle at most once
    # every fired pair that lost has an endpoint in a matched pair
    matched_ids = set(ids.tolist())
    for a, b in zip(tr["ida"][f & ~m], tr["idb"][f & ~m]):
        assert a in matched_ids or b in matched_ids
