"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only *describes* systems (species, contact radii, boundary conditions, rates, box,
time step, seed) and draws seeded random test inputs.  It contains none of the method's
arithmetic: no Green's functions, no probabilities, no random streams of the simulation itself.
Both the CUDA library binding and the CPU oracle read these descriptions; neither imports the
other.

Units: micrometres and seconds.  Boundary-condition names follow Section 2.1 of the paper
(absorbing, reflective, radiation); "none" marks a non-interacting species pair.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

BC_CODES = {"none": 0, "abs": 1, "ref": 2, "rad": 3}
PRECISION_CODES = {"fp64": 0, "mixed": 1}

# Avogadro's number expressed as particles per (um^3 * uM): 1 uM = 602.214 um^-3.
PER_UM3_PER_UM = 602.214076


@dataclass
class PairRule:
    """Interaction of species ``s1`` and ``s2``: contact radius ``sigma``, boundary condition
    ``bc`` and intrinsic association rate ``ka`` (um^3/s in 3D, um^2/s in 2D).  ``product`` is the
    species formed by a bimolecular reaction (-1: the pair vanishes without product)."""

    s1: int
    s2: int
    sigma: float
    bc: str
    ka: float = 0.0
    product: int = -1


@dataclass
class Decay:
    """Unimolecular reaction ``parent -> products`` with rate ``kd`` (1/s).  Two products that form an
    interacting pair are placed at that pair's contact radius; otherwise at ``sigma_place``."""

    parent: int
    kd: float
    products: Tuple[int, ...] = ()
    sigma_place: float = 0.0


@dataclass
class Replica:
    """One independent system of a batched ensemble: its own box edge and initial counts."""

    L: float
    n_init: Sequence[int]


@dataclass
class System:
    dim: int
    L: float
    dt: float
    seed: int
    D: Sequence[float]
    n_init: Sequence[int]
    pairs: List[PairRule]
    decays: List[Decay] = field(default_factory=list)
    names: Optional[Sequence[str]] = None
    c_cut: float = 5.0
    tau_s: float = 0.01
    precision: str = "fp64"
    replicas: Optional[List[Replica]] = None
    # deterministic drift velocity per species (um/s, a 3-vector each), applied as a split step
    drift: Optional[Sequence[Sequence[float]]] = None
    # direction of an encountered pair's new separation: "exact" (from the full propagator) or
    # "free_step" (the free step's direction kept, only the length resampled)
    angle: str = "exact"

    @property
    def n_species(self) -> int:
        return len(self.D)

    def replica_list(self) -> List[Replica]:
        if self.replicas:
            return list(self.replicas)
        return [Replica(self.L, list(self.n_init))]

    def total_particles(self) -> int:
        return int(sum(sum(r.n_init) for r in self.replica_list()))


# ---------------------------------------------------------------------------------------------
# The five workloads (units um, s).  Parameters follow the experiment descriptions; where a value is
# not given (e.g. the diffusion constant of an inert product) the choice is stated inline.
# ---------------------------------------------------------------------------------------------

def irreversible_3d(seed: int = 1) -> System:
    """3D A+B->C, radiation BC: cube L=1, 1000 A + 1000 B, sigma 0.01, D_A=D_B=1, ka=0.05, dt=1e-5.
    C does not interact; its diffusion constant (0.5) only moves it."""
    return System(dim=3, L=1.0, dt=1e-5, seed=seed, D=[1.0, 1.0, 0.5], n_init=[1000, 1000, 0],
                  names=["A", "B", "C"],
                  pairs=[PairRule(0, 1, 0.01, "rad", 0.05, 2)])


def reversible_3d(dt: float = 1e-5, seed: int = 1, n_each: int = 100_000, L: float = 2.55,
                  equilibrium_start: bool = False) -> System:
    """3D A+B<->C, radiation BC: L=2.55 (10 uM), 1e5 A + 1e5 B, sigma 0.005, D=1 (C: 0.5),
    ka=0.02, kd=10, unbinding at contact.  ``equilibrium_start`` seeds the mass-action composition
    (bound fraction 0.7505) instead of all-unbound."""
    n_a = n_b = n_each
    n_c = 0
    if equilibrium_start:
        n_c = int(round(0.7505 * n_each))
        n_a = n_b = n_each - n_c
    return System(dim=3, L=L, dt=dt, seed=seed, D=[1.0, 1.0, 0.5], n_init=[n_a, n_b, n_c],
                  names=["A", "B", "C"],
                  pairs=[PairRule(0, 1, 0.005, "rad", 0.02, 2)],
                  decays=[Decay(2, 10.0, (0, 1))])


def membrane_2d(seed: int = 1, n_each: int = 200_000, L: float = 10.0, dt: float = 1e-4,
                equilibrium_start: bool = False) -> System:
    """2D A+B<->C on a membrane: square L=10, 2e5 A + 2e5 B, sigma 0.005, D=0.1, ka=0.01 um^2/s,
    kd=1, dt=1e-4.  A+B carries the radiation BC; C+C is reflective (excluded volume).
    ``equilibrium_start`` seeds the mass-action composition (bound fraction 0.8) instead of
    all-unbound."""
    n_c = int(round(0.8 * n_each)) if equilibrium_start else 0
    return System(dim=2, L=L, dt=dt, seed=seed, D=[0.1, 0.1, 0.1], n_init=[n_each - n_c, n_each - n_c, n_c],
                  names=["A", "B", "C"],
                  pairs=[PairRule(0, 1, 0.005, "rad", 0.01, 2),
                         PairRule(2, 2, 0.005, "ref")],
                  decays=[Decay(2, 1.0, (0, 1))])


def ensemble_3d(n_replicas: int = 4096, seed: int = 1, n_min: int = 64, n_max: int = 8192,
                c_min_uM: float = 1.0, c_max_uM: float = 20.0) -> System:
    """Batched ensemble of independent 3D A+B<->C replicas: N per species log-uniform in
    [n_min, n_max], concentration uniform in [c_min, c_max] uM setting each box edge,
    sigma 0.005, D=1 (C: 0.5), ka=0.02, kd=10, dt=1e-5."""
    rng = np.random.default_rng([seed, 0x5EED])
    reps = []
    for _ in range(n_replicas):
        n = int(math.floor(math.exp(rng.uniform(0.0, math.log(n_max / n_min))) * n_min))
        n = max(n_min, min(n, n_max))
        conc = rng.uniform(c_min_uM, c_max_uM)
        L = (n / (PER_UM3_PER_UM * conc)) ** (1.0 / 3.0)
        reps.append(Replica(L, [n, n, 0]))
    return System(dim=3, L=reps[0].L, dt=1e-5, seed=seed, D=[1.0, 1.0, 0.5], n_init=reps[0].n_init,
                  names=["A", "B", "C"],
                  pairs=[PairRule(0, 1, 0.005, "rad", 0.02, 2)],
                  decays=[Decay(2, 10.0, (0, 1))], replicas=reps)


def network_3d(dt: float = 1e-5, seed: int = 1, scale: float = 1.0, L: float = 20.0) -> System:
    """5-species 3D network in L=20: A+B<->C (radiation), C+D->E (absorbing), E->A+D (rate 5),
    C+C reflective excluded volume.  Initial A:B:C:D:E = 3:3:1:2:1 x 1e6 (x ``scale``),
    D = 2, 1, 0.5, 1, 0.2; sigma 0.004-0.008; E's products are placed 0.004 apart, non-interacting."""
    base = [3, 3, 1, 2, 1]
    n_init = [int(round(b * 1_000_000 * scale)) for b in base]
    Lx = L * (scale ** (1.0 / 3.0))
    return System(dim=3, L=Lx, dt=dt, seed=seed, D=[2.0, 1.0, 0.5, 1.0, 0.2], n_init=n_init,
                  names=["A", "B", "C", "D", "E"],
                  pairs=[PairRule(0, 1, 0.005, "rad", 0.02, 2),
                         PairRule(2, 3, 0.006, "abs", 0.0, 4),
                         PairRule(2, 2, 0.008, "ref")],
                  decays=[Decay(2, 10.0, (0, 1)), Decay(4, 5.0, (0, 3), sigma_place=0.004)])


def isolated_pairs_3d(n_pairs: int, R0: float, sigma: float = 0.01, D: float = 1.0, ka: float = 0.05,
                      dt: float = 1e-5, spacing: float = 0.5, bc: str = "rad", seed: int = 7):
    """Many A-B pairs on a cubic lattice, each pair at separation ``R0*sigma`` along a seeded random
    direction and ``spacing`` away from every other pair.  Returns (system, positions, species)."""
    m = int(math.ceil(n_pairs ** (1.0 / 3.0)))
    L = m * spacing
    rng = np.random.default_rng([seed, 11])
    idx = np.arange(n_pairs)
    centres = np.stack([(idx % m), (idx // m) % m, idx // (m * m)], axis=1) * spacing + 0.25 * spacing
    v = rng.normal(size=(n_pairs, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    half = 0.5 * R0 * sigma * v
    pos = np.concatenate([centres - half, centres + half]) % L
    species = np.concatenate([np.zeros(n_pairs, np.int32), np.ones(n_pairs, np.int32)])
    sys_ = System(dim=3, L=L, dt=dt, seed=seed, D=[D, D, 0.5], n_init=[n_pairs, n_pairs, 0],
                  names=["A", "B", "C"], pairs=[PairRule(0, 1, sigma, bc, ka, 2)])
    return sys_, pos, species


def pair_samples(n: int, sigma: float, D_rel: float, dt: float, c_cut: float = 5.0, dim: int = 3,
                 seed: int = 3, near_contact_fraction: float = 0.25):
    """Seeded (r0, r) separations shaped like a step's candidate pairs: r0 uniform in the shell
    sigma < |r0| < sigma + c_cut*sqrt(2 D dt) (volume measure), r = |r0 + sqrt(2 D dt) N|, plus a
    fraction drawn close to contact (r0 - sigma and r - sigma within 0.05 sqrt(2 D dt))."""
    rng = np.random.default_rng([seed, 29])
    ell = math.sqrt(2.0 * D_rel * dt)
    rc = sigma + c_cut * ell
    u = rng.uniform(size=n)
    r0 = (sigma ** dim + u * (rc ** dim - sigma ** dim)) ** (1.0 / dim)
    v = rng.normal(size=(n, dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x1 = r0[:, None] * v + ell * rng.normal(size=(n, dim))
    r = np.linalg.norm(x1, axis=1)
    k = int(near_contact_fraction * n)
    if k:
        r0[:k] = sigma + 0.05 * ell * rng.uniform(size=k)
        r[:k] = sigma + 0.05 * ell * rng.uniform(size=k)
    return r0, r
