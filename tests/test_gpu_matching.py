"""Conflict resolution at full size: the accepted set of every step equals the greedy matching of
the step's fired pairs in ascending (key, id_a, id_b) (Section 3: each particle takes part in at
most one reaction, the pair with the smallest exponential race key wins).  The dense 2D membrane
at tau = 0.8 puts thousands of pairs into the iterative rounds, which then run on the whole
cooperative grid; smaller membranes at the same density put hundreds there (one block, global
memory); the sparse 3D system a few (one block, shared memory)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402

SHARED_MEMORY_MAX = 256   # conflict pairs matched by one block in shared memory
SINGLE_BLOCK_MAX = 2048   # conflict pairs handled by one block (above: the cooperative grid)


def greedy_accept(f):
    """Greedy matching in ascending (key, id_a, id_b); particles are (replica, id)."""
    n = len(f["key"])
    order = np.lexsort((f["id_b"], f["id_a"], f["key"]))
    a = f["replica"].astype(np.int64) << 32 | f["id_a"].astype(np.int64)
    b = f["replica"].astype(np.int64) << 32 | f["id_b"].astype(np.int64)
    used = set()
    acc = np.zeros(n, bool)
    for k in order:
        if a[k] not in used and b[k] not in used:
            acc[k] = True
            used.add(a[k])
            used.add(b[k])
    return acc, a, b


def conflict_pairs(a, b):
    ends = np.concatenate([a, b])
    uniq, cnt = np.unique(ends, return_counts=True)
    deg = dict(zip(uniq.tolist(), cnt.tolist()))
    return sum(1 for x, y in zip(a.tolist(), b.tolist()) if deg[x] > 1 or deg[y] > 1)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_dense_2d_matching_is_greedy(precision):
    sim = pkg.Simulation(W.membrane_2d(seed=3), precision=precision)
    most = 0
    for _ in range(3):
        sim.step()
        f = sim.last_fired()
        acc, a, b = greedy_accept(f)
        assert np.array_equal(acc, f["accepted"])
        most = max(most, conflict_pairs(a, b))
    assert most > SINGLE_BLOCK_MAX        # the cooperative path ran
    sim.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sparse_3d_matching_is_greedy(precision):
    sim = pkg.Simulation(W.reversible_3d(), precision=precision)
    for _ in range(3):
        sim.step()
        f = sim.last_fired()
        acc, a, b = greedy_accept(f)
        assert np.array_equal(acc, f["accepted"])
        assert 0 < conflict_pairs(a, b) <= SHARED_MEMORY_MAX
    sim.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_mid_size_conflict_lists_are_greedy(precision):
    # membranes at the full-size density with fewer particles: at least one lands its conflict
    # list between the shared-memory and the cooperative regimes
    seen = []
    for n_each in (2000, 4000, 8000, 16000):
        L = 10.0 * (n_each / 200_000) ** 0.5
        sim = pkg.Simulation(W.membrane_2d(seed=5, n_each=n_each, L=L), precision=precision)
        for _ in range(2):
            sim.step()
            f = sim.last_fired()
            acc, a, b = greedy_accept(f)
            assert np.array_equal(acc, f["accepted"]), n_each
            seen.append(conflict_pairs(a, b))
        sim.close()
    assert any(SHARED_MEMORY_MAX < c <= SINGLE_BLOCK_MAX for c in seen), seen
