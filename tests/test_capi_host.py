"""CPU-side checks of the C ABI: the library builds, loads, exports every entry point that
``include/rd.h`` declares, and rejects invalid configurations before touching the GPU."""
import ctypes as C
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1107_0270_gb300 import build

    build.build()
    import paper_1107_0270_gb300 as pkg

    return pkg.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ["rd_init", "rd_step", "rd_run", "rd_observables", "rd_pair_probs", "rd_get_state",
                     "rd_set_state", "rd_free", "rd_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    import paper_1107_0270_gb300 as pkg

    assert set(pkg.EXPORTS) <= set(declared_functions())


def _init_rc(lib, system, **kw):
    import paper_1107_0270_gb300 as pkg

    cfg, keep = pkg.make_config(system, **kw)
    h = C.c_void_p()
    rc = lib.rd_init(C.byref(cfg), None, C.byref(h))
    return rc, h


@pytest.mark.parametrize("mutate", [
    lambda s: setattr(s, "dt", 0.0),
    lambda s: setattr(s, "dt", -1.0),
    lambda s: s.pairs.append(W.PairRule(0, 7, 0.01, "rad", 0.1, 2)),          # unknown species
    lambda s: s.pairs.append(W.PairRule(1, 0, 0.01, "abs", 0.0, 2)),          # duplicate pair
    lambda s: setattr(s.pairs[0], "sigma", 0.0),
    lambda s: setattr(s.pairs[0], "product", 9),
    lambda s: s.decays.append(W.Decay(2, 1.0, (0, 5))),
    lambda s: setattr(s, "L", 0.05),                                          # cut-off >= L/2
])
def test_invalid_configurations_are_rejected(lib, mutate):
    s = W.irreversible_3d()
    mutate(s)
    rc, h = _init_rc(lib, s)
    assert rc == 1 and not h.value          # RD_EINVAL, no handle


@pytest.mark.parametrize("kw,mutate", [
    ({"block_size": 300}, None),                                                 # above 256
    ({"block_size": 100}, None),                                                 # not a multiple of 32
    ({"sweep_split": 3}, None),
    ({"cell_reach": 2}, None),                                                   # reach 2 is 2D only
    ({"cell_reach": 3}, None),
    ({}, lambda s: setattr(s, "drift", [(1e6, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)])),  # > L/2 per step
    ({}, lambda s: setattr(s, "drift", [(float("nan"), 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)])),
])
def test_invalid_launch_options_are_rejected(lib, kw, mutate):
    s = W.irreversible_3d()
    if mutate:
        mutate(s)
    rc, h = _init_rc(lib, s, **kw)
    assert rc == 1 and not h.value


def test_strerror(lib):
    lib.rd_strerror.restype = C.c_char_p
    assert lib.rd_strerror(0) == b"ok"
    assert b"capacity" in lib.rd_strerror(3)
