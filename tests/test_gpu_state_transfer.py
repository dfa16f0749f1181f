"""State transfer through the C ABI from and into page-locked caller arrays (asynchronous copies)
and pageable ones: both must give the same state, and a rejected state must leave the handle
untouched."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402


def pinned_buffers(cap, n_replicas):
    def pin(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()
    return {"x": pin((cap, 3), torch.float64), "species": pin(cap, torch.int32),
            "ids": pin(cap, torch.int32).view(np.uint32), "replica": pin(cap, torch.int32),
            "next_id": pin(n_replicas, torch.int32).view(np.uint32)}


def system():
    base = W.ensemble_3d(n_replicas=6, seed=8, n_min=40, n_max=200, c_min_uM=5.0, c_max_uM=20.0)
    return W.System(**{**base.__dict__, "dt": 2e-5})


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pinned_and_pageable_transfers_agree(precision):
    s = system()
    a = pkg.Simulation(s, precision=precision)
    b = pkg.Simulation(s, precision=precision)
    a.run(3)
    ref = a.get_state()                                   # pageable
    buf = pinned_buffers(2 * len(ref["ids"]) + 64, a.n_replicas)
    pin = a.get_state(out=buf)                            # page-locked, written by the device
    for k in ("x", "species", "ids", "replica", "next_id"):
        assert np.array_equal(pin[k], ref[k]), k
    # twin b loads the state from page-locked arrays, a from pageable copies; both step alike
    b.set_state(pin["x"], pin["species"], pin["ids"], pin["replica"], pin["next_id"], pin["step"])
    a.set_state(ref["x"].copy(), ref["species"].copy(), ref["ids"].copy(), ref["replica"].copy(),
                ref["next_id"].copy(), ref["step"])
    a.run(4)
    b.run(4)
    sa, sb = a.get_state(), b.get_state()
    for k in ("x", "species", "ids", "replica", "next_id"):
        assert np.array_equal(sa[k], sb[k]), k
    a.close()
    b.close()


def test_rejected_pinned_state_leaves_the_handle_untouched():
    s = system()
    sim = pkg.Simulation(s, precision="mixed")
    sim.run(2)
    before = sim.get_state()
    buf = pinned_buffers(2 * len(before["ids"]) + 64, sim.n_replicas)
    st = sim.get_state(out=buf)
    st["ids"][[0, 1]] = st["ids"][[1, 0]]                 # ids out of order inside replica 0
    with pytest.raises(pkg.RDError) as e:
        sim.set_state(st["x"], st["species"], st["ids"], st["replica"], st["next_id"], st["step"])
    assert e.value.code == 1
    after = sim.get_state()
    for k in ("x", "species", "ids", "replica", "next_id"):
        assert np.array_equal(after[k], before[k]), k
    sim.close()


def test_single_system_transfer_without_replica_array():
    # a single system needs no per-particle replica indices: omitted on both sides of the ABI,
    # the state round trip is the same as with them
    s = W.reversible_3d(dt=2e-5, seed=4, n_each=400, L=0.6)
    a = pkg.Simulation(s, precision="mixed")
    b = pkg.Simulation(s, precision="mixed")
    a.run(3)
    full = a.get_state()
    buf = pinned_buffers(2 * len(full["ids"]) + 64, 1)
    del buf["replica"]
    st = a.get_state(out=buf)
    assert st["replica"] is None
    for k in ("x", "species", "ids", "next_id"):
        assert np.array_equal(st[k], full[k]), k
    b.set_state(st["x"], st["species"], st["ids"], None, st["next_id"], st["step"])
    a.run(4)
    b.run(4)
    sa, sb = a.get_state(), b.get_state()
    for k in ("x", "species", "ids", "replica", "next_id"):
        assert np.array_equal(sa[k], sb[k]), k
    a.close()
    b.close()
