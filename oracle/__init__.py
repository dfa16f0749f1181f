"""Python access to the plain FP64 CPU oracle (``oracle/rd_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's CPU-baseline leg are
the only callers.  This module never imports the CUDA library package, and the CUDA library never
imports this module.  ``build()`` compiles the C oracle with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")   # the all-core CPU-baseline build
_SOURCES = [os.path.join(_HERE, "rd_oracle.c")]

MAX_SPECIES, MAX_PAIRS, MAX_DECAYS = 16, 32, 16
BC = {"none": 0, "abs": 1, "ref": 2, "rad": 3}


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no floating-point contraction) and return the .so path; also
    the OpenMP build of the same source (the all-core CPU baseline: the pair loop on all threads,
    same results) when the compiler supports it."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SOURCES + [os.path.join(_HERE, "oracle.h")])
    for path, extra in ((_LIB_PATH, []), (_LIB_OMP_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
            tmp = path + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC", "-shared"] + extra + \
                  ["-o", tmp] + _SOURCES + ["-lm"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                if extra:          # no OpenMP here: the baseline reports the single-thread build only
                    continue
                raise RuntimeError(f"oracle build failed:\n{r.stderr}")
            os.replace(tmp, path)
    return _LIB_PATH


class _Pair(C.Structure):
    _fields_ = [("s1", C.c_int32), ("s2", C.c_int32), ("bc", C.c_int32), ("product", C.c_int32),
                ("sigma", C.c_double), ("ka", C.c_double)]


class _Decay(C.Structure):
    _fields_ = [("parent", C.c_int32), ("n_products", C.c_int32), ("p0", C.c_int32),
                ("p1", C.c_int32), ("kd", C.c_double), ("sigma_place", C.c_double)]


class _System(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_species", C.c_int32), ("n_pairs", C.c_int32),
                ("n_decays", C.c_int32), ("L", C.c_double), ("dt", C.c_double),
                ("c_cut", C.c_double), ("tau_s", C.c_double), ("seed", C.c_uint64),
                ("replica", C.c_uint32), ("pad_", C.c_uint32),
                ("D", C.c_double * MAX_SPECIES), ("pairs", _Pair * MAX_PAIRS),
                ("decays", _Decay * MAX_DECAYS), ("drift_dx", (C.c_double * 3) * MAX_SPECIES),
                ("has_drift", C.c_int32), ("angle_mode", C.c_int32)]


class _State(C.Structure):
    _fields_ = [("n", C.c_int64), ("cap", C.c_int64), ("x", C.POINTER(C.c_double)),
                ("sp", C.POINTER(C.c_int32)), ("id", C.POINTER(C.c_uint32)),
                ("step", C.c_uint32), ("next_id", C.c_uint32), ("t", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("candidates", "fired", "matched", "reactions", "resampled",
                                          "decays", "recombined", "near_threshold", "overlaps",
                                          "products")]


class _Trace(C.Structure):
    _fields_ = [("cap", C.c_int64), ("n", C.c_int64), ("ida", C.POINTER(C.c_uint32)),
                ("idb", C.POINTER(C.c_uint32)), ("p_enc", C.POINTER(C.c_double)),
                ("u_enc", C.POINTER(C.c_double)), ("fired", C.POINTER(C.c_int32)),
                ("matched", C.POINTER(C.c_int32))]


_lib = None
_lib_omp = None


def lib(openmp: bool = False):
    """The oracle library; openmp=True: the OpenMP build (None if it could not be built)."""
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            build()
            if not os.path.exists(_LIB_OMP_PATH):
                return None
            _lib_omp = _bind(C.CDLL(_LIB_OMP_PATH))
        return _lib_omp
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(L):
    if True:
        d = C.c_double
        for name, args in [("or_p_enc3", [d, d, d]), ("or_p_reac3", [d, d, d, d]),
                           ("or_tail3", [d, d, d]), ("or_resample3", [d, d, d]),
                           ("or_S_abs3", [d, d]), ("or_S_rad3", [d, d, d]),
                           ("or_erfcx", [d]), ("or_gfree2", [d, d, d]),
                           ("or_p_enc2", [d, d, d, d]), ("or_p_reac2", [d, d, d, d, d]),
                           ("or_tail2", [d, d, d, d]), ("or_resample2", [d, d, d, d]),
                           ("or_gbc2_weber", [C.c_int, d, d, d, d]), ("or_S_abs2", [d, d])]:
            fn = getattr(L, name)
            fn.restype = d
            fn.argtypes = args
        L.or_ierfc_scaled.restype = d
        L.or_ierfc_scaled.argtypes = [C.c_int, d]
        L.or_gamma2.restype = d
        L.or_gamma2.argtypes = [C.c_int, C.c_int, d, d, d]
        L.or_gbc2_series.restype = d
        L.or_gbc2_series.argtypes = [C.c_int, d, d, d, d, C.c_int]
        L.or_u52.restype = d
        L.or_u52.argtypes = [C.c_uint32, C.c_uint32]
        L.or_philox4x32_10.restype = None
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                       C.POINTER(C.c_uint32)]
        L.or_fpt_refine.restype = C.c_int
        L.or_fpt_refine.argtypes = [C.c_int, d, d, d, d, C.c_int, C.c_uint64, C.c_uint64, C.c_uint32,
                                    C.POINTER(C.c_uint32), C.POINTER(d), C.POINTER(d),
                                    C.POINTER(C.c_uint32), C.POINTER(d)]
        L.or_fpt_direction.restype = C.c_int
        L.or_fpt_direction.argtypes = [C.c_int, d, C.c_uint64, C.c_uint64, C.c_uint32, C.POINTER(d),
                                       C.POINTER(d)]
        L.or_init_positions.restype = C.c_int
        L.or_init_positions.argtypes = [C.POINTER(_System), C.POINTER(C.c_int64), C.POINTER(_State)]
        L.or_ang_coeffs.restype = C.c_int
        L.or_ang_coeffs.argtypes = [C.c_int, C.c_int, d, d, d, C.POINTER(d), C.c_int]
        L.or_ang_sample.restype = d
        L.or_ang_sample.argtypes = [C.c_int, d, d, d, d]
        L.or_ang_density.restype = d
        L.or_ang_density.argtypes = [C.c_int, d, d, d, d]
        L.or_ang_cdf.restype = d
        L.or_ang_cdf.argtypes = [C.c_int, d, d, d, d]
        L.or_gf_partial.restype = d
        L.or_gf_partial.argtypes = [C.c_int, C.c_int, d, d, d, d]
        L.or_propagate.restype = None
        L.or_propagate.argtypes = [C.c_int, C.POINTER(d), d, d, d, d, d, C.POINTER(d)]
        L.or_set_fault.restype = None
        L.or_set_fault.argtypes = [C.c_int]
        L.or_step.restype = C.c_int
        L.or_step.argtypes = [C.POINTER(_System), C.POINTER(_State), C.POINTER(_State),
                              C.POINTER(_Stats), C.POINTER(_Trace)]
        L.or_threads.restype = C.c_int
        L.or_threads.argtypes = []
    return L


def threads(openmp: bool = True) -> int:
    """Threads the (OpenMP) oracle build uses for a step; 1 for the serial build."""
    L = lib(openmp)
    return 1 if L is None else int(L.or_threads())


# ------------------------------------------------------------------------------------------------
# scalar functions (scaled units: R = r/a, tau = D t / a^2)
# ------------------------------------------------------------------------------------------------

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def u52(hi, lo):
    return lib().or_u52(hi, lo)


def erfcx(x):
    return lib().or_erfcx(float(x))


def p_enc3(R, R0, tau):
    return lib().or_p_enc3(R, R0, tau)


def p_reac3(R, R0, tau, h):
    return lib().or_p_reac3(R, R0, tau, h)


def tail3(V, R0, tau):
    return lib().or_tail3(V, R0, tau)


def resample3(U, R0, tau):
    return lib().or_resample3(U, R0, tau)


def S_abs3(R0, tau):
    return lib().or_S_abs3(R0, tau)


def S_rad3(R0, tau, h):
    return lib().or_S_rad3(R0, tau, h)


def ierfc_scaled(n, z):
    return lib().or_ierfc_scaled(n, z)


def gamma2(k, bc, R, R0, h):
    return lib().or_gamma2(k, BC[bc] if isinstance(bc, str) else bc, R, R0, h)


def gbc2_series(bc, R, R0, tau, h, nterms=12):
    return lib().or_gbc2_series(BC[bc] if isinstance(bc, str) else bc, R, R0, tau, h, nterms)


def gbc2_weber(bc, R, R0, tau, h):
    return lib().or_gbc2_weber(BC[bc] if isinstance(bc, str) else bc, R, R0, tau, h)


def gfree2(R, R0, tau):
    return lib().or_gfree2(R, R0, tau)


def p_enc2(R, R0, tau, tau_s=0.01):
    return lib().or_p_enc2(R, R0, tau, tau_s)


def p_reac2(R, R0, tau, h, tau_s=0.01):
    return lib().or_p_reac2(R, R0, tau, h, tau_s)


def tail2(V, R0, tau, tau_s=0.01):
    return lib().or_tail2(V, R0, tau, tau_s)


def S_abs2(R0, tau):
    return lib().or_S_abs2(R0, tau)


def resample2(U, R0, tau, tau_s=0.01):
    return lib().or_resample2(U, R0, tau, tau_s)


def fpt_refine(dim, R0, R, tau, levels, seed, stream, tau_s=0.01, max_attempts=1 << 20):
    """First-passage refinement of one encountered pair (Appendix; scaled units): returns
    (bin, R_lo, R_hi, attempts, margin, ok); the first contact lies in [bin, bin + 1) tau / 2^levels."""
    b, a = C.c_uint32(), C.c_uint32()
    lo, hi, mg = C.c_double(), C.c_double(), C.c_double()
    st = lib().or_fpt_refine(int(dim), float(R0), float(R), float(tau), float(tau_s), int(levels),
                             int(seed) & (2**64 - 1), int(stream) & (2**64 - 1), int(max_attempts),
                             C.byref(b), C.byref(lo), C.byref(hi), C.byref(a), C.byref(mg))
    return b.value, lo.value, hi.value, a.value, mg.value, st == 0


def fpt_direction(dim, kappa, seed, stream, attempt):
    """The refinement's end-point direction draw: (1 - cos(theta), sin(theta)), or None."""
    omc, sn = C.c_double(), C.c_double()
    ok = lib().or_fpt_direction(int(dim), float(kappa), int(seed), int(stream), int(attempt),
                                C.byref(omc), C.byref(sn))
    return (omc.value, sn.value) if ok else None


def fpt_refine_batch(dim, R0, R, tau, levels, seed, streams, tau_s=0.01, max_attempts=1 << 20):
    """fpt_refine over arrays R0, R, streams (same tau): arrays bin, R_lo, R_hi, attempts, margin."""
    n = len(R0)
    out = {"bin": np.zeros(n, np.uint32), "R_lo": np.zeros(n), "R_hi": np.zeros(n),
           "attempts": np.zeros(n, np.uint32), "margin": np.zeros(n)}
    for k in range(n):
        b, lo, hi, a, mg, _ = fpt_refine(dim, R0[k], R[k], tau, levels, seed, int(streams[k]), tau_s,
                                         max_attempts)
        out["bin"][k], out["R_lo"][k], out["R_hi"][k], out["attempts"][k], out["margin"][k] = b, lo, hi, a, mg
    return out


ANG_WHICH = {"encountered": 0, "abs": 1, "ref": 2, "free": 3}


def ang_coeffs(dim, R, R0, tau, which="encountered", cap=1201):
    """Partial-wave integrals D_n (n = 0..N) of the exact propagation law (scaled units)."""
    D = np.zeros(cap)
    N = lib().or_ang_coeffs(int(dim), ANG_WHICH[which], float(R), float(R0), float(tau),
                            D.ctypes.data_as(C.POINTER(C.c_double)), cap)
    return D[:N + 1].copy()


def ang_sample(dim, U, R, R0, tau):
    """Angle of the new separation to the start separation at CDF value U (3D: its cosine)."""
    return lib().or_ang_sample(int(dim), float(U), float(R), float(R0), float(tau))


def ang_density(dim, v, R, R0, tau):
    return lib().or_ang_density(int(dim), float(v), float(R), float(R0), float(tau))


def ang_cdf(dim, v, R, R0, tau):
    """CDF of the conditional angle at v (3D: its cosine), the function ang_sample inverts."""
    return lib().or_ang_cdf(int(dim), float(v), float(R), float(R0), float(tau))


def propagate(dim, r0, tau, u_res, u_ang, u_azi, tau_s=0.01):
    """New separation vector (scaled units) of an encountered pair from start vector r0."""
    a = (C.c_double * 3)(*[float(v) for v in list(r0) + [0.0] * (3 - len(r0))])
    o = (C.c_double * 3)()
    lib().or_propagate(int(dim), a, float(tau), float(tau_s), float(u_res), float(u_ang), float(u_azi), o)
    return np.array([o[0], o[1], o[2]])


def gf_partial(dim, which, v, R, R0, tau):
    """Full Green's function at separation R and angle v (3D: v = cos) from its partial waves."""
    return lib().or_gf_partial(int(dim), ANG_WHICH[which], float(v), float(R), float(R0), float(tau))


def pair_probs(system, r0, r, rule: int = 0):
    """p_enc and p_reac (reaction probability at end separation r from start r0) for arrays of
    physical separations, for pair rule ``rule`` of ``system`` (dimension-aware)."""
    pr = system.pairs[rule]
    D = system.D[pr.s1] + system.D[pr.s2]
    tau = D * system.dt / pr.sigma ** 2
    if system.dim == 3:
        h = pr.ka / (4 * np.pi * pr.sigma * D)
        fe, fr = p_enc3, p_reac3
        pe = np.array([fe(b / pr.sigma, a / pr.sigma, tau) for a, b in zip(r0, r)])
        prc = np.array([fr(b / pr.sigma, a / pr.sigma, tau, h) for a, b in zip(r0, r)])
    else:
        h = pr.ka / (2 * np.pi * D)
        pe = np.array([p_enc2(b / pr.sigma, a / pr.sigma, tau, system.tau_s) for a, b in zip(r0, r)])
        prc = np.array([p_reac2(b / pr.sigma, a / pr.sigma, tau, h, system.tau_s)
                        for a, b in zip(r0, r)])
    return pe, prc


class planted_fault:
    """Context manager of the negative controls: plants one deliberate mistake in the oracle
    (1: conflict key -ln(U_sel) * p_enc; 2: descending greedy order; 3: U_enc reused as U_sel; 4: the
    cylindrical Bessel derivative in the 3D boundary coefficients) and removes it on exit."""

    def __init__(self, fault: int):
        self.fault = int(fault)

    def __enter__(self):
        lib().or_set_fault(self.fault)
        return self

    def __exit__(self, *exc):
        lib().or_set_fault(0)
        return False


# ------------------------------------------------------------------------------------------------
# whole-step interface
# ------------------------------------------------------------------------------------------------

@dataclass
class State:
    x: np.ndarray        # (n, 3) float64, z = 0 in 2D
    species: np.ndarray  # (n,) int32
    ids: np.ndarray      # (n,) uint32
    step: int = 0
    next_id: int = 0
    t: float = 0.0

    @property
    def n(self):
        return int(self.ids.shape[0])

    def counts(self, n_species):
        return np.bincount(self.species, minlength=n_species)


def _system_struct(system, replica: int = 0, L: float | None = None) -> _System:
    s = _System()
    s.dim = system.dim
    s.n_species = len(system.D)
    s.n_pairs = len(system.pairs)
    s.n_decays = len(system.decays)
    s.L = float(system.L if L is None else L)
    s.dt = float(system.dt)
    s.c_cut = float(system.c_cut)
    s.tau_s = float(system.tau_s)
    s.seed = int(system.seed)
    s.replica = int(replica)
    for i, d in enumerate(system.D):
        s.D[i] = float(d)
    for i, p in enumerate(system.pairs):
        s.pairs[i] = _Pair(p.s1, p.s2, BC[p.bc], p.product, p.sigma, p.ka)
    for i, dc in enumerate(system.decays):
        prods = list(dc.products) + [-1, -1]
        s.decays[i] = _Decay(dc.parent, len(dc.products), prods[0], prods[1], dc.kd, dc.sigma_place)
    s.angle_mode = 1 if getattr(system, "angle", "exact") == "free_step" else 0
    drift = getattr(system, "drift", None)
    if drift is not None:
        s.has_drift = 1
        for i, v in enumerate(drift):
            for d in range(3):
                s.drift_dx[i][d] = float(v[d]) * float(system.dt)    # displacement per step, v dt
    return s


def _state_struct(x, sp, ids, n, cap, step, next_id, t):
    st = _State()
    st.n = n
    st.cap = cap
    st.x = x.ctypes.data_as(C.POINTER(C.c_double))
    st.sp = sp.ctypes.data_as(C.POINTER(C.c_int32))
    st.id = ids.ctypes.data_as(C.POINTER(C.c_uint32))
    st.step = step
    st.next_id = next_id
    st.t = t
    return st


def init_state(system, replica: int = 0) -> State:
    rep = system.replica_list()[replica]
    n = int(sum(rep.n_init))
    x = np.zeros((max(n, 1), 3))
    sp = np.zeros(max(n, 1), np.int32)
    ids = np.zeros(max(n, 1), np.uint32)
    st = _state_struct(x, sp, ids, 0, max(n, 1), 0, 0, 0.0)
    sysc = _system_struct(system, replica, rep.L)
    ninit = (C.c_int64 * MAX_SPECIES)(*[int(v) for v in rep.n_init])
    rc = lib().or_init_positions(C.byref(sysc), ninit, C.byref(st))
    if rc != 0:
        raise RuntimeError(f"or_init_positions failed: {rc}")
    return State(x[:n].copy(), sp[:n].copy(), ids[:n].copy(), 0, int(st.next_id), 0.0)


def step(system, state: State, replica: int = 0, L: float | None = None, trace: bool = False,
         openmp: bool = False):
    """Advance ``state`` by one step.  Returns (new_state, stats dict[, trace dict]).  openmp: run
    the pair loop on all threads (the OpenMP build; same result, no trace)."""
    n = state.n
    cap = 2 * n + 16
    xin = np.ascontiguousarray(state.x, dtype=np.float64).reshape(-1, 3)
    spin = np.ascontiguousarray(state.species, dtype=np.int32)
    idin = np.ascontiguousarray(state.ids, dtype=np.uint32)
    if n == 0:
        xin = np.zeros((1, 3))
        spin = np.zeros(1, np.int32)
        idin = np.zeros(1, np.uint32)
    stin = _state_struct(xin, spin, idin, n, max(n, 1), state.step, state.next_id, state.t)
    xo = np.zeros((cap, 3))
    spo = np.zeros(cap, np.int32)
    ido = np.zeros(cap, np.uint32)
    stout = _state_struct(xo, spo, ido, 0, cap, 0, 0, 0.0)
    stats = _Stats()
    tr = None
    arrays = None
    if trace:
        tcap = n * (n - 1) // 2 + 1024 if n < 4000 else 256 * n
        arrays = dict(ida=np.zeros(tcap, np.uint32), idb=np.zeros(tcap, np.uint32),
                      p_enc=np.zeros(tcap), u_enc=np.zeros(tcap), fired=np.zeros(tcap, np.int32),
                      matched=np.zeros(tcap, np.int32))
        tr = _Trace()
        tr.cap = tcap
        tr.n = 0
        tr.ida = arrays["ida"].ctypes.data_as(C.POINTER(C.c_uint32))
        tr.idb = arrays["idb"].ctypes.data_as(C.POINTER(C.c_uint32))
        tr.p_enc = arrays["p_enc"].ctypes.data_as(C.POINTER(C.c_double))
        tr.u_enc = arrays["u_enc"].ctypes.data_as(C.POINTER(C.c_double))
        tr.fired = arrays["fired"].ctypes.data_as(C.POINTER(C.c_int32))
        tr.matched = arrays["matched"].ctypes.data_as(C.POINTER(C.c_int32))
    Lrep = system.replica_list()[replica].L if L is None else L
    sysc = _system_struct(system, replica, Lrep)
    Lb = lib(True) if (openmp and not trace) else None
    rc = (Lb or lib()).or_step(C.byref(sysc), C.byref(stin), C.byref(stout), C.byref(stats),
                              C.byref(tr) if tr is not None else None)
    if rc != 0:
        raise RuntimeError(f"or_step failed: {rc}")
    m = int(stout.n)
    new = State(xo[:m].copy(), spo[:m].copy(), ido[:m].copy(), int(stout.step), int(stout.next_id),
                float(stout.t))
    sd = {k: int(getattr(stats, k)) for k, _ in _Stats._fields_}
    if trace:
        k = int(tr.n)
        return new, sd, {key: v[:k].copy() for key, v in arrays.items()}
    return new, sd
