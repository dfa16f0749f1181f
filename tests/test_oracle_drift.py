"""Pins of the oracle's deterministic-force split step: every particle first moves by its
species' drift displacement v dt (periodic wrap), then the Brownian / reaction step runs from there
with p_enc and p_reac computed from the Brownian end points only."""
import numpy as np

import oracle as O
import workloads as W


def test_drift_alone_is_exact_translation():
    # no diffusion and no reactions: after n steps every particle sits at wrap(x + n v dt), the
    # adds done one step at a time
    v = [(3.0, -1.5, 0.25), (0.0, 2.0, -4.0)]
    system = W.System(dim=3, L=0.7, dt=1e-3, seed=3, D=[0.0, 0.0], n_init=[50, 50], pairs=[], drift=v)
    st = O.init_state(system)
    x = st.x.copy()
    sp = st.species.copy()
    for _ in range(25):
        st, stats = O.step(system, st)
        for i in range(len(x)):
            for d in range(3):
                y = x[i, d] + v[sp[i]][d] * system.dt
                if y >= system.L:
                    y -= system.L
                elif y < 0.0:
                    y += system.L
                x[i, d] = y
    assert np.array_equal(st.x, x)
    assert stats["candidates"] == 0


def test_common_drift_leaves_the_reactions_unchanged():
    # a drift shared by all species translates the whole system: relative vectors, and therefore
    # every encounter, selection and reaction decision, are those of the system without drift
    base = W.reversible_3d(n_each=300, L=(300 / (W.PER_UM3_PER_UM * 20.0)) ** (1 / 3), dt=2e-5, seed=4)
    v = (40.0, -25.0, 10.0)
    moving = W.System(**{**base.__dict__, "drift": [v, v, v]})
    a, b = O.init_state(base), O.init_state(moving)
    shift = np.zeros(3)
    total = 0
    for _ in range(30):
        a, sa = O.step(base, a)
        b, sb = O.step(moving, b)
        shift += np.array(v) * base.dt
        assert np.array_equal(a.ids, b.ids) and np.array_equal(a.species, b.species)
        assert sa["fired"] == sb["fired"] and sa["reactions"] == sb["reactions"]
        total += sa["fired"]
        d = (b.x - a.x - shift) % base.L
        d = np.minimum(d, base.L - d)
        assert d.max(initial=0.0) < 1e-12
    assert total > 0


def test_relative_drift_changes_the_encounters():
    # a drift of A relative to B is not a translation: the encounters differ from the drift-free
    # system (a sign that the split step reaches the pair statistics)
    base = W.reversible_3d(n_each=300, L=(300 / (W.PER_UM3_PER_UM * 20.0)) ** (1 / 3), dt=2e-5, seed=4)
    moving = W.System(**{**base.__dict__, "drift": [(200.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)]})
    a, b = O.init_state(base), O.init_state(moving)
    fa = fb = 0
    for _ in range(30):
        a, sa = O.step(base, a)
        b, sb = O.step(moving, b)
        fa += sa["fired"]
        fb += sb["fired"]
    assert fa != fb
