"""The allocation-free step (rd_step_static) gives the same state as the handle's rd_step.

rd_step_static is for callers that cannot allocate device memory: its scratch is the library's
fixed device array.  This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1107_0270_gb300 as pkg  # noqa: E402


def _system():
    L = (300 / (W.PER_UM3_PER_UM * 40.0)) ** (1 / 3)
    return W.reversible_3d(dt=2e-5, seed=9, n_each=300, L=L)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_step_matches_handle_step_twice(precision):
    system = _system()
    sim = pkg.Simulation(system, precision=precision)
    sim.run(3)
    st = sim.get_state()
    x = torch.tensor(st["x"], device="cuda")
    sp = torch.tensor(st["species"], device="cuda")
    ids = torch.tensor(st["ids"].astype(np.int64), dtype=torch.int32, device="cuda")
    next_id, step = int(st["next_id"][0]), int(st["step"])
    tol = 1e-12 * system.L if precision == "fp64" else 0.0
    for call in range(2):
        x, sp, ids, next_id, status = pkg.step_static(system, x, sp, ids, next_id, step, precision)
        assert status == 0
        step += 1
        sim.step()
        ref = sim.get_state()
        assert ref["step"] == step
        got_ids = ids.cpu().numpy().astype(np.uint32)
        assert np.array_equal(got_ids, ref["ids"]), f"call {call}: ids differ"
        assert np.array_equal(sp.cpu().numpy(), ref["species"]), f"call {call}: species differ"
        assert next_id == int(ref["next_id"][0])
        d = np.abs(x.cpu().numpy() - ref["x"])
        assert d.max(initial=0.0) <= tol, f"call {call}: max position difference {d.max()}"
    sim.close()


def test_static_step_rejects_oversized_input():
    system = _system()
    n = 16385        # one above the documented maximum
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    sp = torch.zeros(n, dtype=torch.int32, device="cuda")
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.RDError) as e:
        pkg.step_static(system, x, sp, ids, n, 0)
    assert e.value.code == 1
