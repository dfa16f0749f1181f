"""GB300-native Green's-function-corrected Brownian-dynamics reaction-diffusion step.

Thin ctypes binding over the C ABI of ``include/rd.h`` (library ``_lib/librd.so``).  The binding only
marshals arguments: every stage of the step runs in the library's CUDA kernels.  PyTorch provides
the device memory (its caching allocator is handed to the library) and the CUDA stream.

There is no CPU fallback: importing works without a GPU, but creating a :class:`Simulation`
raises if the compiled library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librd.so")

MAX_SPECIES, MAX_PAIRS, MAX_DECAYS = 16, 32, 16
NSTATS = 13
STAT_NAMES = ["candidates", "fired", "matched", "reactions", "resampled", "decays", "recombined",
              "near_threshold", "overlaps", "match_rounds", "particle_steps", "fired_hwm", "angle_fallback"]
BC = {"none": 0, "abs": 1, "ref": 2, "rad": 3}
PRECISION = {"fp64": 0, "mixed": 1}
STATUS = {0: "RD_OK", 1: "RD_EINVAL", 2: "RD_ENOMEM", 3: "RD_ECAPACITY", 4: "RD_ETIMEOUT",
          5: "RD_ECUDA", 6: "RD_ENOTREADY"}
# exported symbols declared in include/rd.h
EXPORTS = ["rd_init", "rd_step", "rd_run", "rd_sync", "rd_observables", "rd_get_state", "rd_set_state",
           "rd_pair_probs", "rd_resample", "rd_first_passage", "rd_last_fired", "rd_num_particles", "rd_time_kernels",
           "rd_kernel_times", "rd_free", "rd_strerror", "rd_last_cuda_error", "rd_step_static",
           "rd_info", "rd_count_history", "rd_check_bounded_wait", "rd_propagate"]


class RDError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = f"{STATUS.get(code, code)}: {_strerror(code)}"
        if what:
            msg = f"{what}: {msg}"
        if code == 5:
            msg += f" (cuda error {_lib().rd_last_cuda_error()})"
        super().__init__(msg)


class _PairRule(C.Structure):
    _fields_ = [("s1", C.c_int32), ("s2", C.c_int32), ("bc", C.c_int32), ("product", C.c_int32),
                ("sigma", C.c_double), ("ka", C.c_double)]


class _Decay(C.Structure):
    _fields_ = [("parent", C.c_int32), ("n_products", C.c_int32), ("products", C.c_int32 * 2),
                ("kd", C.c_double), ("sigma_place", C.c_double)]


class _Replica(C.Structure):
    _fields_ = [("L", C.c_double), ("n_init", C.c_int64 * MAX_SPECIES)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class _Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _RELEASE_FN), ("ctx", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("dim", C.c_int32), ("precision", C.c_int32), ("n_species", C.c_int32),
                ("n_pairs", C.c_int32), ("n_decays", C.c_int32), ("n_replicas", C.c_int32),
                ("dt", C.c_double), ("seed", C.c_uint64), ("c_cut", C.c_double), ("tau_s", C.c_double),
                ("D", C.c_double * MAX_SPECIES), ("pairs", _PairRule * MAX_PAIRS),
                ("decays", _Decay * MAX_DECAYS), ("replicas", C.POINTER(_Replica)),
                ("capacity_factor", C.c_double), ("pair_capacity", C.c_int64),
                ("cell_factor_x100", C.c_int32), ("block_size", C.c_int32),
                ("sweep_split", C.c_int32), ("cell_reach", C.c_int32),
                ("drift", (C.c_double * 3) * MAX_SPECIES),
                ("step_launch", C.c_int32), ("force_paths", C.c_int32),
                ("angle_mode", C.c_int32), ("pad_angle", C.c_int32),
                ("allocator", _Allocator)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_1107_0270_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, u32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32, C.c_double
        P = C.POINTER
        L.rd_init.argtypes = [P(_Config), vp, P(vp)]
        L.rd_step.argtypes = [vp]
        L.rd_run.argtypes = [vp, i64]
        L.rd_sync.argtypes = [vp]
        L.rd_observables.argtypes = [vp, P(i64), P(i64), P(d), P(i64)]
        L.rd_get_state.argtypes = [vp, P(i64), P(d), P(i32), P(u32), P(i32), P(u32), P(i64)]
        L.rd_set_state.argtypes = [vp, i64, P(d), P(i32), P(u32), P(i32), P(u32), i64]
        L.rd_pair_probs.argtypes = [vp, i32, vp, vp, i64, vp, vp]
        L.rd_resample.argtypes = [vp, i32, vp, vp, i64, vp]
        L.rd_first_passage.argtypes = [vp, i32, vp, vp, vp, i64, i32, C.c_uint32, vp, vp, vp, vp]
        L.rd_last_fired.argtypes = [vp, i64, P(i64), P(u32), P(u32), P(d), P(i32), P(i32), P(d)]
        L.rd_num_particles.argtypes = [vp, P(i64)]
        L.rd_time_kernels.argtypes = [vp, i32]
        L.rd_kernel_times.argtypes = [vp, i32, P(i32), C.c_char_p, P(C.c_float)]
        L.rd_step_static.argtypes = [P(_Config), vp, i64, vp, vp, vp, u32, i64, i64, vp, vp, vp, vp, vp, vp]
        L.rd_info.argtypes = [vp, P(d), i32]
        L.rd_propagate.argtypes = [vp, i32, vp, vp, i64, vp]
        L.rd_count_history.argtypes = [vp, i64, i64, P(i64)]
        L.rd_check_bounded_wait.argtypes = [vp, C.c_uint32, P(i32)]
        L.rd_free.argtypes = [vp]
        L.rd_free.restype = None
        L.rd_strerror.argtypes = [C.c_int]
        L.rd_strerror.restype = C.c_char_p
        L.rd_last_cuda_error.restype = C.c_int
        for name in EXPORTS:
            if name not in ("rd_free", "rd_strerror", "rd_last_cuda_error"):
                getattr(L, name).restype = C.c_int
        _LIB = L
    return _LIB


def load_library():
    """Load the compiled library (raises if it is missing)."""
    return _lib()


def _strerror(code: int) -> str:
    try:
        return _lib().rd_strerror(code).decode()
    except Exception:  # library not loadable
        return "unknown"


def _check(rc: int, what: str):
    if rc != 0:
        raise RDError(rc, what)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


STEP_LAUNCH = {"auto": 0, "fused": 1, "separate": 2}


def make_config(system, precision: Optional[str] = None, capacity_factor: float = 2.0,
                pair_capacity: int = 0, cell_factor=None, block_size: int = 256, sweep_split: int = 0,
                cell_reach: int = 0, step_launch: str = "auto", force_paths: int = 0):
    """Build the C configuration from a system description (see ``workloads.System``).
    cell_factor: cell edge in units of the largest cut-off; None = density-based per replica
    (about 0.25 interacting particles per cell), "tune" = timed autotuning at creation.
    sweep_split: 0 automatic, 1 one sweep thread per particle, 2 one per (particle, stencil row).
    cell_reach: 0 automatic, 1 cells of a cut-off, 2 (2D) cells of half a cut-off, two-cell stencil.
    step_launch: "auto", "fused" (the whole step as one cooperative launch) or "separate" (one
    launch per kernel); both give bit-identical results.
    force_paths: bit 0 conflict rounds on the whole grid at any size, bit 1 short conflict lists in
    global memory (test knobs for the large-size paths; results unchanged)."""
    cfg = _Config()
    cfg.dim = int(system.dim)
    cfg.precision = PRECISION[precision or system.precision]
    cfg.n_species = len(system.D)
    cfg.n_pairs = len(system.pairs)
    cfg.n_decays = len(system.decays)
    reps = system.replica_list()
    cfg.n_replicas = len(reps)
    cfg.dt = float(system.dt)
    cfg.seed = int(system.seed)
    cfg.c_cut = float(system.c_cut)
    cfg.tau_s = float(system.tau_s)
    for i, v in enumerate(system.D):
        cfg.D[i] = float(v)
    for i, p in enumerate(system.pairs):
        cfg.pairs[i] = _PairRule(p.s1, p.s2, BC[p.bc], p.product, float(p.sigma), float(p.ka))
    for i, dc in enumerate(system.decays):
        prods = list(dc.products) + [-1, -1]
        cfg.decays[i] = _Decay(dc.parent, len(dc.products), (C.c_int32 * 2)(prods[0], prods[1]),
                               float(dc.kd), float(dc.sigma_place))
    rep_arr = (_Replica * len(reps))()
    for r, rep in enumerate(reps):
        rep_arr[r].L = float(rep.L)
        for s, v in enumerate(rep.n_init):
            rep_arr[r].n_init[s] = int(v)
    cfg.replicas = C.cast(rep_arr, C.POINTER(_Replica))
    cfg.capacity_factor = float(capacity_factor)
    cfg.pair_capacity = int(pair_capacity)
    if cell_factor is None:
        cfg.cell_factor_x100 = 0
    elif cell_factor == "tune":
        cfg.cell_factor_x100 = -1
    else:
        cfg.cell_factor_x100 = int(round(float(cell_factor) * 100))
    cfg.block_size = int(block_size)
    cfg.sweep_split = int(sweep_split)
    cfg.cell_reach = int(cell_reach)
    cfg.step_launch = STEP_LAUNCH[step_launch]
    cfg.force_paths = int(force_paths)
    cfg.angle_mode = 1 if getattr(system, "angle", "exact") == "free_step" else 0
    drift = getattr(system, "drift", None)
    if drift is not None:
        for i, v in enumerate(drift):
            for d in range(3):
                cfg.drift[i][d] = float(v[d])
    return cfg, rep_arr


class Simulation:
    """One handle of the C library: a batch of replicas of a reaction-diffusion system on one GPU."""

    def __init__(self, system, precision: Optional[str] = None, device: int = 0, stream=None,
                 capacity_factor: float = 2.0, pair_capacity: int = 0, cell_factor=None,
                 block_size: int = 256, sweep_split: int = 0, cell_reach: int = 0, step_launch: str = "auto",
                 force_paths: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (there is no CPU fallback)")
        lib = _lib()
        self.system = system
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.n_species = len(system.D)
        self.n_replicas = len(system.replica_list())
        self.precision = precision or system.precision
        cfg, self._rep_arr = make_config(system, self.precision, capacity_factor, pair_capacity,
                                         cell_factor, block_size, sweep_split, cell_reach, step_launch,
                                         force_paths)
        dev = self.device.index

        def _alloc(nbytes, stream_ptr, ctx):
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream_ptr or 0)

        def _release(ptr, nbytes, stream_ptr, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = _ALLOC_FN(_alloc)
        self._release_cb = _RELEASE_FN(_release)
        cfg.allocator = _Allocator(self._alloc_cb, self._release_cb, None)
        self._cfg = cfg
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.rd_init(C.byref(cfg), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        _check(rc, "rd_init")
        self._h = h

    # -- stepping ---------------------------------------------------------------------------
    def step(self, n: int = 1):
        for _ in range(n):
            _check(_lib().rd_step(self._h), "rd_step")

    def run(self, n: int):
        _check(_lib().rd_run(self._h, int(n)), "rd_run")

    def sync(self):
        _check(_lib().rd_sync(self._h), "rd_sync")

    # -- observables and state --------------------------------------------------------------
    def observables(self):
        counts = np.zeros(self.n_replicas * self.n_species, np.int64)
        stats = np.zeros(NSTATS, np.int64)
        step = C.c_int64()
        t = C.c_double()
        rc = _lib().rd_observables(self._h, _ptr(counts, C.c_int64), C.byref(step), C.byref(t),
                                   _ptr(stats, C.c_int64))
        _check(rc, "rd_observables")
        return {"counts": counts.reshape(self.n_replicas, self.n_species), "step": step.value,
                "t": t.value, "stats": dict(zip(STAT_NAMES, stats.tolist()))}

    def check_bounded_wait(self, spin_limit: int = 100_000) -> int:
        """Run the cell scan once with a look-back wait that nothing satisfies, bounded by
        spin_limit polls; returns the status the device latched (RD_ETIMEOUT = 4 expected)."""
        st = C.c_int32()
        _check(_lib().rd_check_bounded_wait(self._h, int(spin_limit), C.byref(st)), "rd_check_bounded_wait")
        return st.value

    def count_history(self, first_step: int = 0, n_steps: Optional[int] = None):
        """Totals per species (summed over replicas) for steps first_step .. first_step+n_steps-1."""
        if n_steps is None:
            n_steps = self.observables()["step"] - first_step + 1
        out = np.zeros((max(n_steps, 1), self.n_species), np.int64)
        _check(_lib().rd_count_history(self._h, int(first_step), int(n_steps), _ptr(out, C.c_int64)),
               "rd_count_history")
        return out[:n_steps]

    def info(self):
        v = np.zeros(11)
        _check(_lib().rd_info(self._h, _ptr(v, C.c_double), 11), "rd_info")
        return {"cell_factor": abs(v[0]), "cell_rule": "density" if v[0] < 0 else "fixed",
                "cells": int(v[1]), "block": int(v[2]),
                "capacity": int(v[3]), "pair_capacity": int(v[4]), "tuned_ms_per_step": v[5],
                "r_cut_max": v[6], "sweep_split": int(v[7]), "reach": int(v[8]),
                "fused": bool(v[9]), "fused_grid": int(v[10])}

    def num_particles(self) -> int:
        n = C.c_int64()
        _check(_lib().rd_num_particles(self._h, C.byref(n)), "rd_num_particles")
        return n.value

    def get_state(self, allow_error: bool = False, out=None):
        """Current state (host copies).  allow_error: return it even when a device error
        (RD_ECAPACITY / RD_ETIMEOUT) is latched, with the code under "status".  out: optional dict
        of caller-owned arrays ("x" (m, 3) float64, "species" int32, "ids" uint32, "replica"
        int32, "next_id" uint32) with room for the current particles (e.g. page-locked buffers);
        the returned arrays are views of them.  Without a "replica" array in `out` the replica
        indices are not copied and "replica" is None (a single system needs none)."""
        if out is None:
            n = C.c_int64(self.num_particles())
            x = np.zeros((max(n.value, 1), 3))
            sp = np.zeros(max(n.value, 1), np.int32)
            ids = np.zeros(max(n.value, 1), np.uint32)
            rep = np.zeros(max(n.value, 1), np.int32)
            nxt = np.zeros(self.n_replicas, np.uint32)
        else:
            x, sp, ids, rep, nxt = out["x"], out["species"], out["ids"], out.get("replica"), out["next_id"]
            n = C.c_int64(ids.shape[0])
        step = C.c_int64()
        rc = _lib().rd_get_state(self._h, C.byref(n), _ptr(x, C.c_double), _ptr(sp, C.c_int32),
                                 _ptr(ids, C.c_uint32), _ptr(rep, C.c_int32), _ptr(nxt, C.c_uint32),
                                 C.byref(step))
        if not (allow_error and rc in (3, 4)):
            _check(rc, "rd_get_state")
        m = n.value
        return {"x": x[:m], "species": sp[:m], "ids": ids[:m], "replica": None if rep is None else rep[:m],
                "next_id": nxt, "step": step.value, "status": rc}

    def set_state(self, x, species, ids, replica=None, next_id=None, step: int = 0):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        species = np.ascontiguousarray(species, dtype=np.int32)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        n = ids.shape[0]
        rep = None if replica is None else np.ascontiguousarray(replica, dtype=np.int32)
        nxt = None if next_id is None else np.ascontiguousarray(next_id, dtype=np.uint32)
        rc = _lib().rd_set_state(self._h, n, _ptr(x, C.c_double), _ptr(species, C.c_int32),
                                 _ptr(ids, C.c_uint32), _ptr(rep, C.c_int32), _ptr(nxt, C.c_uint32),
                                 int(step))
        _check(rc, "rd_set_state")

    def last_fired(self, cap: int = 1 << 22):
        n = C.c_int64()
        _check(_lib().rd_last_fired(self._h, 0, C.byref(n), None, None, None, None, None, None),
               "rd_last_fired")
        m = min(n.value, cap)
        ida = np.zeros(max(m, 1), np.uint32)
        idb = np.zeros(max(m, 1), np.uint32)
        p = np.zeros(max(m, 1))
        acc = np.zeros(max(m, 1), np.int32)
        rep = np.zeros(max(m, 1), np.int32)
        key = np.zeros(max(m, 1))
        _check(_lib().rd_last_fired(self._h, m, C.byref(n), _ptr(ida, C.c_uint32), _ptr(idb, C.c_uint32),
                                    _ptr(p, C.c_double), _ptr(acc, C.c_int32), _ptr(rep, C.c_int32),
                                    _ptr(key, C.c_double)),
               "rd_last_fired")
        return {"id_a": ida[:m], "id_b": idb[:m], "p_enc": p[:m], "accepted": acc[:m].astype(bool),
                "replica": rep[:m], "key": key[:m]}

    # -- per-pair probability and propagator batches (device tensors) ------------------------
    def pair_probs(self, r0, r, rule: int = 0, out=None):
        import torch

        assert r0.is_cuda and r.is_cuda and r0.dtype == torch.float64 and r.dtype == torch.float64
        r0 = r0.contiguous()
        r = r.contiguous()
        n = r0.numel()
        pe = torch.empty(n, dtype=torch.float64, device=r0.device) if out is None else out[0]
        pr = torch.empty(n, dtype=torch.float64, device=r0.device) if out is None else out[1]
        self.stream.wait_stream(torch.cuda.current_stream(r0.device))
        rc = _lib().rd_pair_probs(self._h, rule, r0.data_ptr(), r.data_ptr(), n, pe.data_ptr(),
                                  pr.data_ptr() if pr is not None else None)
        _check(rc, "rd_pair_probs")
        torch.cuda.current_stream(r0.device).wait_stream(self.stream)
        return pe, pr

    def resample(self, r0, u, rule: int = 0):
        import torch

        r0 = r0.contiguous()
        u = u.contiguous()
        out = torch.empty_like(r0)
        self.stream.wait_stream(torch.cuda.current_stream(r0.device))
        _check(_lib().rd_resample(self._h, rule, r0.data_ptr(), u.data_ptr(), r0.numel(), out.data_ptr()),
               "rd_resample")
        torch.cuda.current_stream(r0.device).wait_stream(self.stream)
        return out

    def propagate(self, r0, u, rule: int = 0):
        """New separation vectors of encountered pairs (device tensors: r0 float64 (n, 3), u float64
        (n, 4)) drawn from the full propagator G_ref - G_abs (rd_propagate)."""
        import torch

        r0 = r0.contiguous()
        u = u.contiguous()
        assert r0.dtype == torch.float64 and u.dtype == torch.float64 and r0.shape[0] == u.shape[0]
        out = torch.empty_like(r0)
        self.stream.wait_stream(torch.cuda.current_stream(r0.device))
        _check(_lib().rd_propagate(self._h, rule, r0.data_ptr(), u.data_ptr(), r0.shape[0], out.data_ptr()),
               "rd_propagate")
        torch.cuda.current_stream(r0.device).wait_stream(self.stream)
        return out

    def first_passage(self, r0, r, stream, levels: int, rule: int = 0, max_attempts: int = 0):
        """First-passage refinement of encountered pairs (device tensors r0, r float64 and stream
        int64): dict of bin (int32 view of uint32), r_lo, r_hi, attempts."""
        import torch

        assert r0.is_cuda and r.is_cuda and stream.is_cuda and stream.dtype == torch.int64
        r0, r, stream = r0.contiguous(), r.contiguous(), stream.contiguous()
        n = r0.numel()
        dev = r0.device
        out = {"bin": torch.empty(n, dtype=torch.int32, device=dev),
               "r_lo": torch.empty(n, dtype=torch.float64, device=dev),
               "r_hi": torch.empty(n, dtype=torch.float64, device=dev),
               "attempts": torch.empty(n, dtype=torch.int32, device=dev)}
        self.stream.wait_stream(torch.cuda.current_stream(dev))
        _check(_lib().rd_first_passage(self._h, rule, r0.data_ptr(), r.data_ptr(), stream.data_ptr(), n, levels,
                                       max_attempts, out["bin"].data_ptr(), out["r_lo"].data_ptr(),
                                       out["r_hi"].data_ptr(), out["attempts"].data_ptr()),
               "rd_first_passage")
        torch.cuda.current_stream(dev).wait_stream(self.stream)
        return out

    # -- per-kernel timing of one step -----------------------------------------------------------
    def timed_step(self):
        _check(_lib().rd_time_kernels(self._h, 1), "rd_time_kernels")
        self.step()
        n = C.c_int32()
        names = C.create_string_buffer(64 * 32)
        ms = (C.c_float * 64)()
        _check(_lib().rd_kernel_times(self._h, 64, C.byref(n), names, ms), "rd_kernel_times")
        out = []
        for k in range(min(n.value, 64)):
            nm = names.raw[32 * k:32 * (k + 1)].split(b"\0", 1)[0].decode()
            out.append((nm, float(ms[k])))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib().rd_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_static(system, x, species, ids, next_id: int, step: int, precision: Optional[str] = None,
                stream=None):
    """One step of a small single-replica system through the allocation-free entry point
    ``rd_step_static``: its scratch lives in the library's fixed device array, so the library
    allocates nothing.  Inputs are CUDA tensors (x float64 [n,3], species int32 [n], ids int32 [n]
    holding uint32 ids); output tensors are created here by the caller side of the ABI.
    Returns (x, species, ids, next_id, status) with the new particle count."""
    import torch

    lib = _lib()
    n = int(ids.numel())
    dev = x.device
    # the entry point takes raw device pointers: check shapes, types and device here
    if not (x.is_cuda and species.is_cuda and ids.is_cuda):
        raise ValueError("x, species and ids must be CUDA tensors")
    if not (x.device == species.device == ids.device):
        raise ValueError("x, species and ids must be on one device")
    if dev.index != torch.cuda.current_device():
        raise ValueError("the tensors' device must be the current CUDA device")
    if x.dtype != torch.float64 or tuple(x.shape) != (n, 3):
        raise ValueError("x must be float64 of shape (n, 3)")
    if species.dtype != torch.int32 or species.numel() != n:
        raise ValueError("species must be int32 with n entries")
    if ids.dtype != torch.int32:
        raise ValueError("ids must be int32 (holding uint32 ids) with n entries")
    cfg, rep_arr = make_config(system, precision)
    cap = max(2 * n, 1)
    x_out = torch.empty((cap, 3), dtype=torch.float64, device=dev)
    sp_out = torch.empty(cap, dtype=torch.int32, device=dev)
    id_out = torch.empty(cap, dtype=torch.int32, device=dev)
    meta = torch.zeros(4, dtype=torch.int64, device=dev)      # n_out | next_id | status
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = lib.rd_step_static(C.byref(cfg), C.c_void_p(s.cuda_stream), n, x.contiguous().data_ptr(),
                            species.contiguous().data_ptr(), ids.contiguous().data_ptr(), int(next_id),
                            int(step), cap, x_out.data_ptr(), sp_out.data_ptr(), id_out.data_ptr(),
                            meta.data_ptr(), meta.data_ptr() + 8, meta.data_ptr() + 16)
    _check(rc, "rd_step_static")
    s.synchronize()
    m = meta.cpu()
    n_new = int(m[0])
    next_new = int(m[1]) & 0xFFFFFFFF
    status = int(m[2]) & 0xFFFFFFFF
    return x_out[:n_new], sp_out[:n_new], id_out[:n_new], next_new, status
