"""Host-side argument checks of the Python binding (no GPU needed): the allocation-free step refuses
tensors it would otherwise hand to the library as raw device pointers."""
import pytest

torch = pytest.importorskip("torch")

import paper_1107_0270_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402


def _system():
    return W.reversible_3d(dt=2e-5, seed=9, n_each=5, L=0.2)


def test_step_static_refuses_host_tensors():
    x = torch.zeros((10, 3), dtype=torch.float64)
    sp = torch.zeros(10, dtype=torch.int32)
    ids = torch.arange(10, dtype=torch.int32)
    with pytest.raises(ValueError):
        pkg.step_static(_system(), x, sp, ids, 10, 0)


def test_make_config_carries_the_launch_options_and_the_angle_mode():
    system = _system()
    cfg, _ = pkg.make_config(system, "mixed", step_launch="separate", force_paths=3)
    assert cfg.step_launch == 2 and cfg.force_paths == 3 and cfg.angle_mode == 0
    system.angle = "free_step"
    cfg, _ = pkg.make_config(system, "fp64")
    assert cfg.angle_mode == 1 and cfg.step_launch == 0
