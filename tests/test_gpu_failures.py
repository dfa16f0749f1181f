"""Failure detection without a GPU fault: a list overflow and a device wait that runs out are
latched as status codes, the step that raised them leaves the state unchanged, and the handle
keeps working after the host clears the error."""
import time

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402

RD_ECAPACITY, RD_ETIMEOUT = 3, 4


def dense(n_each=2000, dt=1e-4):
    L = (n_each / (W.PER_UM3_PER_UM * 20.0)) ** (1.0 / 3.0)
    return W.reversible_3d(dt=dt, n_each=n_each, L=L, seed=7)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pair_list_overflow_is_latched_and_the_step_not_committed(precision):
    sim = pkg.Simulation(dense(), precision=precision, pair_capacity=8)
    s0 = sim.get_state()
    sim.step()
    with pytest.raises(pkg.RDError) as e:
        sim.sync()
    assert e.value.code == RD_ECAPACITY
    s1 = sim.get_state(allow_error=True)
    assert s1["status"] == RD_ECAPACITY
    assert s1["step"] == s0["step"]
    assert np.array_equal(s1["ids"], s0["ids"]) and np.array_equal(s1["x"], s0["x"])
    # the host clears the error by loading a state; the handle steps again
    sim.set_state(s0["x"], s0["species"], s0["ids"], step=s0["step"])
    sim.sync()
    sim.close()
    # the same system with room for its pairs steps normally
    ok = pkg.Simulation(dense(), precision=precision)
    ok.run(3)
    ok.sync()
    assert ok.observables()["step"] == 3
    ok.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bounded_wait_runs_out_and_the_context_stays_usable(precision):
    system = W.reversible_3d(dt=1e-5, n_each=20_000, L=2.55 * 0.2 ** (1 / 3))
    a = pkg.Simulation(system, precision=precision)
    b = pkg.Simulation(system, precision=precision)
    a.run(2)
    b.run(2)
    t0 = time.perf_counter()
    assert a.check_bounded_wait(100_000) == RD_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the probe left the state alone: both handles continue identically
    a.run(5)
    b.run(5)
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(sa["ids"], sb["ids"]) and np.array_equal(sa["x"], sb["x"])
    assert sa["step"] == 7
    a.close()
    b.close()
