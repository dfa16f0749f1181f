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
    if precision == "mixed":
        # a mixed handle draws exact directions from its rule's table, the allocation-free call
        # (which builds no angle table) evaluates the law per pair: compare with the free-step
        # direction, where both run the same arithmetic
        system.angle = "free_step"
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


def _raw_call(system, x, sp, ids, next_id, step, precision, out_cap):
    """rd_step_static through the C ABI with output buffers prefilled with a sentinel, so that a
    test can tell whether the entry point wrote them."""
    import ctypes as C

    lib = pkg.load_library()
    cfg, rep_arr = pkg.make_config(system, precision)
    n = int(ids.numel())
    x_out = torch.full((out_cap, 3), -7.0, dtype=torch.float64, device="cuda")
    sp_out = torch.full((out_cap,), -7, dtype=torch.int32, device="cuda")
    id_out = torch.full((out_cap,), -7, dtype=torch.int32, device="cuda")
    meta = torch.full((4,), -7, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    rc = lib.rd_step_static(C.byref(cfg), C.c_void_p(s.cuda_stream), n, x.data_ptr(), sp.data_ptr(),
                            ids.data_ptr(), int(next_id), int(step), out_cap, x_out.data_ptr(), sp_out.data_ptr(),
                            id_out.data_ptr(), meta.data_ptr(), meta.data_ptr() + 8, meta.data_ptr() + 16)
    s.synchronize()
    return rc, x_out, sp_out, id_out, meta.cpu()


def test_static_step_rejects_tables_too_large_and_leaves_outputs_untouched():
    # the mixed step's FP32 tables are built in the scratch array; at dt = 1e-4 (tau = 8) those of
    # the 10 uM reversible system do not fit, so the call is refused before anything is enqueued
    system = W.reversible_3d(dt=1e-4, seed=9, n_each=5, L=2.55)
    n = 10
    x = torch.rand((n, 3), dtype=torch.float64, device="cuda") * 2.0
    sp = torch.tensor([0] * 5 + [1] * 5, dtype=torch.int32, device="cuda")
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    rc, x_out, sp_out, id_out, meta = _raw_call(system, x, sp, ids, n, 0, "mixed", 2 * n)
    assert rc == 1
    assert torch.all(x_out == -7.0) and torch.all(sp_out == -7) and torch.all(id_out == -7)
    assert torch.all(meta == -7)
    # the same system in FP64 needs no tables and runs
    rc, _, _, _, meta = _raw_call(system, x, sp, ids, n, 0, "fp64", 2 * n)
    assert rc == 0 and (int(meta[2]) & 0xFFFFFFFF) == 0   # status_out is an int32 slot


def test_static_step_pair_overflow_latches_capacity_and_keeps_the_state():
    # 4000 A and 4000 B inside a cluster smaller than the contact radius: every A-B pair overlaps
    # and fires (p_enc = 1), 1.6e7 pairs against the 65536 the scratch array holds
    system = W.reversible_3d(dt=2e-5, seed=9, n_each=4000, L=1.0)
    n = 8000
    g = torch.Generator(device="cuda").manual_seed(5)
    x = 0.5 + 0.001 * (torch.rand((n, 3), dtype=torch.float64, device="cuda", generator=g) - 0.5)
    sp = torch.tensor([0] * 4000 + [1] * 4000, dtype=torch.int32, device="cuda")
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    rc, x_out, sp_out, id_out, meta = _raw_call(system, x, sp, ids, n, 3, "fp64", 2 * n)
    assert rc == 0
    assert (int(meta[2]) & 0xFFFFFFFF) == 3        # RD_ECAPACITY in status_out (an int32 slot)
    assert int(meta[0]) == n and (int(meta[1]) & 0xFFFFFFFF) == n   # count and next id unchanged
    assert torch.equal(x_out[:n], x) and torch.equal(sp_out[:n], sp) and torch.equal(id_out[:n], ids)


def test_static_step_after_a_larger_call_matches_handle_step():
    # the array keeps the previous call's contents: a large call first, then a small system must
    # still step exactly like the handle path
    big = W.reversible_3d(dt=2e-5, seed=3, n_each=8000, L=(8000 / (W.PER_UM3_PER_UM * 40.0)) ** (1 / 3))
    simb = pkg.Simulation(big, precision="fp64")
    st = simb.get_state()
    xb = torch.tensor(st["x"], device="cuda")
    spb = torch.tensor(st["species"], device="cuda")
    idb = torch.tensor(st["ids"].astype(np.int64), dtype=torch.int32, device="cuda")
    *_, status = pkg.step_static(big, xb, spb, idb, int(st["next_id"][0]), 0, "fp64")
    assert status == 0
    simb.close()
    system = _system()
    sim = pkg.Simulation(system, precision="fp64")
    sim.run(2)
    st = sim.get_state()
    x = torch.tensor(st["x"], device="cuda")
    sp = torch.tensor(st["species"], device="cuda")
    ids = torch.tensor(st["ids"].astype(np.int64), dtype=torch.int32, device="cuda")
    x, sp, ids, next_id, status = pkg.step_static(system, x, sp, ids, int(st["next_id"][0]), int(st["step"]), "fp64")
    assert status == 0
    sim.step()
    ref = sim.get_state()
    assert np.array_equal(ids.cpu().numpy().astype(np.uint32), ref["ids"])
    assert np.array_equal(sp.cpu().numpy(), ref["species"])
    assert next_id == int(ref["next_id"][0])
    assert np.abs(x.cpu().numpy() - ref["x"]).max(initial=0.0) <= 1e-12 * system.L
    sim.close()
