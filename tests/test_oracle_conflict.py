"""Pin of the oracle's conflict resolution against the paper's multi-candidate rule.

Section 3 ("Details"): when a particle has several encounter candidates in one step, the partner is
chosen among them with probability proportional to each candidate's encounter probability p_enc.
The oracle realises this as an exponential race: every fired pair gets the key -ln(U_sel)/p_enc and
the smallest key wins.  With one particle A and several partners B_j that interact only with A,
the only conflict is at A, so given the fired set S of a step and its p_enc values the winner is j
with probability p_j / sum_{k in S} p_k.  Summed over many independent steps, the observed wins of
each partner must match these conditional probabilities within the binomial error.

The three negative controls plant a plausible mistake in the oracle (key -ln(U) * p_enc, a
descending greedy order, the encounter draw reused as the selection draw) and check that the same
statistic rejects each of them.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

N_STEPS = 30_000
R0S = (1.02, 1.3, 1.8, 2.6)          # start separations of the four partners, in units of sigma


def _system(seed=5):
    sigma = 0.01
    # tau = D_rel dt / sigma^2 = 0.5; the cut-off sigma + 5 sqrt(2 D_rel dt) = 0.06 holds every partner
    # the winner's later propagation plays no part in the law pinned here: the free-step direction
    # (no partial-wave draw) keeps 30 000 steps fast
    return W.System(dim=3, L=1.0, dt=2.5e-5, seed=seed, D=[1.0, 1.0, 0.5], n_init=[1, 4, 0],
                    names=["A", "B", "C"], pairs=[W.PairRule(0, 1, sigma, "ref")], angle="free_step")


def _state(system):
    sigma = system.pairs[0].sigma
    c = np.array([0.5, 0.5, 0.5])
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]], float)
    x = np.vstack([c] + [c + R0 * sigma * d for R0, d in zip(R0S, dirs)])
    return O.State(x=x, species=np.array([0, 1, 1, 1, 1], np.int32), ids=np.arange(5, dtype=np.uint32),
                   step=0, next_id=5)


def _race_statistics(n_steps=N_STEPS):
    """Observed wins, expected wins and variance per partner over steps with >= 2 fired partners."""
    system = _system()
    st0 = _state(system)
    k = len(R0S)
    obs, exp, var = np.zeros(k), np.zeros(k), np.zeros(k)
    multi = 0
    for s in range(n_steps):
        st0.step = s
        _, _, tr = O.step(system, st0, trace=True)
        assert np.all(tr["ida"] == 0)            # every candidate pair involves A (id 0)
        f = tr["fired"].astype(bool)
        if f.sum() < 2:
            continue
        multi += 1
        j = tr["idb"][f].astype(int) - 1         # partner index 0..3
        p = tr["p_enc"][f]
        q = p / p.sum()
        m = tr["matched"][f].astype(bool)
        assert m.sum() == 1                      # exactly one winner at A
        obs[j[m]] += 1.0
        exp[j] += q
        var[j] += q * (1.0 - q)
    return obs, exp, var, multi


def _check(obs, exp, var, bound=4.5):
    z = (obs - exp) / np.sqrt(np.maximum(var, 1.0))
    assert np.all(np.abs(z) < bound), (obs, exp, z)
    return z


@pytest.fixture(scope="module")
def race():
    return _race_statistics()


def test_winner_frequencies_follow_p_enc(race):
    obs, exp, var, multi = race
    assert multi > 3000                           # enough steps with a real choice at A
    assert np.all(exp > 200)                      # every partner is often in the running
    _check(obs, exp, var)


def test_multi_candidate_law_is_not_uniform(race):
    # the p_enc-weighted law differs clearly from a uniform choice among the fired partners, so the
    # pin above is sensitive to the weights themselves
    obs, exp, var, multi = race
    spread = np.abs(exp / exp.sum() - 0.25).max()
    assert spread > 0.05


@pytest.mark.parametrize("fault", [1, 2, 3])
def test_planted_conflict_mistakes_are_rejected(fault):
    with O.planted_fault(fault):
        obs, exp, var, _ = _race_statistics(N_STEPS // 2)
    with pytest.raises(AssertionError):
        _check(obs, exp, var)
