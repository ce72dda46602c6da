"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds initial-condition geometry and random draws only: lattices,
random site removal, random walks, Maxwell-Boltzmann peculiar velocities and
request traces.  None of the shear-flow method's arithmetic (Lees-Edwards images,
forces, integration, thermostat, stress) lives here, so the CPU oracle and the
CUDA path can both take their inputs from it without sharing any of the method.

The workloads follow the parameter sets of the paper's simulations (Sec. 2.4):
LJ fluids at density ~0.844 with r_c = 2.5 (Eq. 9/10) and Kremer-Grest melts
with WCA + FENE (Eq. 10/11).  The paper's own configurations were "equilibrated"
states that are not published, so every input here is generated from a seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2109

_FCC_BASIS = np.array(
    [[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]]
)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def fcc_sites(k: int, box: float) -> np.ndarray:
    """The 4*k^3 sites of a face-centred cubic lattice filling a cubic box."""
    a = box / k
    g = np.arange(k, dtype=np.float64)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    corners = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (corners[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    # shift by a quarter cell so no site sits on a box face
    sites += 0.25 * a
    return np.mod(sites, box)


def lj_box(n: int, rho: float, seed: int) -> tuple[np.ndarray, float]:
    """n particles on an fcc lattice in a cubic box of density rho.

    When n is not 4*k^3, the lattice with k = ceil((n/4)^(1/3)) is filled and
    the surplus sites are removed at random (seeded), so the density is exact.
    """
    box = (n / rho) ** (1.0 / 3.0)
    k = math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9)
    sites = fcc_sites(k, box)
    if sites.shape[0] > n:
        keep = rng(seed).choice(sites.shape[0], size=n, replace=False)
        keep.sort()
        sites = sites[keep]
    return np.ascontiguousarray(sites), box


def mb_velocities(n: int, kT: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """Maxwell-Boltzmann peculiar velocities with zero centre-of-mass motion,
    rescaled so that sum(m v^2) = (3n - 3) kT exactly."""
    v = rng(seed + 7919).normal(0.0, math.sqrt(kT / mass), size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    if n > 1:
        scale = math.sqrt((3 * n - 3) * kT / (mass * float(np.sum(v * v))))
        v *= scale
    return np.ascontiguousarray(v)


def random_walk_chains(nchains: int, nbeads: int, rho: float, seed: int,
                       bond: float = 0.97) -> tuple[np.ndarray, float, np.ndarray]:
    """Freely jointed random walks of fixed step length in a periodic cubic box.

    Returns wrapped positions (nchains*nbeads, 3), the box edge and the bond
    pairs (global ids of consecutive beads).  Overlaps are not removed: a
    force-capped push-off is needed before such a melt can be integrated.
    """
    n = nchains * nbeads
    box = (n / rho) ** (1.0 / 3.0)
    g = rng(seed)
    pos = np.empty((n, 3))
    for c in range(nchains):
        p = g.uniform(0.0, box, size=3)
        steps = g.normal(size=(nbeads - 1, 3))
        steps *= bond / np.linalg.norm(steps, axis=1, keepdims=True)
        chain = np.vstack([p, p + np.cumsum(steps, axis=0)])
        pos[c * nbeads:(c + 1) * nbeads] = chain
    return np.ascontiguousarray(np.mod(pos, box)), box, chain_bonds(nchains, nbeads)


def lattice_chains(nchains: int, nbeads: int, rho: float, seed: int
                   ) -> tuple[np.ndarray, float, np.ndarray]:
    """Non-overlapping linear chains laid along a serpentine path through a
    simple-cubic lattice of density rho (bond length = lattice spacing).

    Consecutive sites of the path are nearest neighbours, so every bond has the
    lattice spacing and no two beads are closer than that spacing.  The chains
    are then placed at a seeded random translation of the whole lattice.
    """
    n = nchains * nbeads
    k = math.ceil(n ** (1.0 / 3.0) - 1e-9)
    box = (k ** 3 / rho) ** (1.0 / 3.0)
    a = box / k
    order = []
    for iz in range(k):
        ys = range(k) if iz % 2 == 0 else range(k - 1, -1, -1)
        for jy, iy in enumerate(ys):
            forward = (iz * k + jy) % 2 == 0
            xs = range(k) if forward else range(k - 1, -1, -1)
            for ix in xs:
                order.append((ix, iy, iz))
    sites = (np.array(order[:n], dtype=np.float64) + 0.5) * a
    sites += rng(seed).uniform(0.0, a, size=3)
    # the serpentine path can jump between z layers only through a neighbour,
    # so every consecutive pair is one lattice spacing apart
    return np.ascontiguousarray(np.mod(sites, box)), box, chain_bonds(nchains, nbeads)


def chain_bonds(nchains: int, nbeads: int) -> np.ndarray:
    ids = np.arange(nchains * nbeads, dtype=np.int32).reshape(nchains, nbeads)
    pairs = np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], axis=1)
    return np.ascontiguousarray(pairs.astype(np.int32))


@dataclass
class Workload:
    """Parameters of one synthetic workload (reduced LJ units, m = kB = 1)."""
    name: str
    n: int
    rho: float
    box: float
    shear_rate: float
    rc: float
    skin: float
    dt: float
    kT: float
    xi: float
    steps: int
    precision: int          # 0 = FP64, 1 = FP32 forces / FP64-class positions
    lj_shift: int = 1
    fene_k: float = 0.0
    fene_R0: float = 1.5
    seed: int = BASE_SEED
    nchains: int = 0
    nbeads: int = 0
    extra: dict = field(default_factory=dict)


def lj_fluid_4000() -> Workload:
    """Plain LJ fluid under shear, FP64: fcc 10x10x10 (4000 sites), rho 0.8442."""
    n, rho = 4000, 0.8442
    return Workload("lj_fluid_n4000_fp64", n, rho, (n / rho) ** (1 / 3), 0.1, 2.5,
                    0.3, 0.005, 1.0, 1.0, 500, 0, seed=BASE_SEED + 0)


def kg_melt_200x100() -> Workload:
    """Kremer-Grest melt, 200 chains x 100 beads, WCA + FENE, rho 0.85."""
    n, rho = 20000, 0.85
    return Workload("kg_melt_200x100_fp32", n, rho, (n / rho) ** (1 / 3), 1e-3,
                    2 ** (1 / 6), 0.3, 0.01, 1.0, 0.5, 10000, 1, fene_k=30.0,
                    fene_R0=1.5, seed=BASE_SEED + 1, nchains=200, nbeads=100)


def lj_box_4m() -> Workload:
    """Large single LJ box: N = 4,194,304 particles at rho 0.8442, FP32 forces."""
    n, rho = 4194304, 0.8442
    return Workload("lj_box_n4194304_fp32", n, rho, (n / rho) ** (1 / 3), 0.05, 2.5,
                    0.3, 0.005, 1.0, 1.0, 1000, 1, seed=BASE_SEED + 2)


def scaled_lj(base: Workload, n: int, name: str | None = None) -> Workload:
    """The same LJ workload (density, cut-off, skin, shear, thermostat) with n
    particles: used for bounded CPU samples and small parity cases."""
    return Workload(name or f"{base.name}_sample_n{n}", n, base.rho,
                    (n / base.rho) ** (1 / 3), base.shear_rate, base.rc, base.skin,
                    base.dt, base.kT, base.xi, base.steps, base.precision,
                    base.lj_shift, base.fene_k, base.fene_R0, base.seed)


def lj_initial_state(w: Workload) -> tuple[np.ndarray, np.ndarray]:
    """Positions (fcc, seeded site removal) and MB peculiar velocities."""
    pos, _ = lj_box(w.n, w.rho, w.seed)
    vel = mb_velocities(w.n, w.kT, w.seed)
    return pos, vel


def batched_systems(count: int = 256, seed: int = BASE_SEED + 3,
                    nmin: int = 500, nmax: int = 32000) -> list[dict]:
    """Independent LJ systems of uneven size: N log-uniform in [nmin, nmax],
    density uniform in [0.7, 0.9], shear rate log-uniform in [1e-3, 1]."""
    g = rng(seed)
    out = []
    for s in range(count):
        n = int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax)))))
        out.append(dict(n=n, rho=float(g.uniform(0.7, 0.9)),
                        shear_rate=float(math.exp(g.uniform(math.log(1e-3), 0.0))),
                        seed=seed * 1000 + s))
    return out


def request_trace(count: int = 1000, rate: float = 50.0, seed: int = BASE_SEED + 4
                  ) -> list[dict]:
    """Poisson arrivals of shear-sweep requests: LJ (N log-uniform in [1e3, 2e5]
    at rho 0.8442) or KG (chains log-uniform in [50, 1000], length log-uniform in
    [20, 200], rho 0.85), each at one of 8 shear rates log-spaced in [1e-4, 1]."""
    g = rng(seed)
    rates = np.logspace(-4, 0, 8)
    t = 0.0
    out = []
    for r in range(count):
        t += float(g.exponential(1.0 / rate))
        kind = "lj" if g.uniform() < 0.5 else "kg"
        req = dict(id=r, arrival=t, kind=kind, shear_rate=float(rates[g.integers(8)]),
                   seed=seed * 100000 + r)
        if kind == "lj":
            req["n"] = int(round(math.exp(g.uniform(math.log(1e3), math.log(2e5)))))
            req["rho"] = 0.8442
        else:
            req["nchains"] = int(round(math.exp(g.uniform(math.log(50), math.log(1000)))))
            req["nbeads"] = int(round(math.exp(g.uniform(math.log(20), math.log(200)))))
            req["n"] = req["nchains"] * req["nbeads"]
            req["rho"] = 0.85
        out.append(req)
    return out
