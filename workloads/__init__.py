"""Seeded synthetic DPD workloads shared by the tests, the smoke check and the
benchmark.

This module only draws inputs (positions, velocities, species, bond lists)
from numpy's seeded PCG64 generator and holds the parameter sets of the
workloads; it contains none of the method's arithmetic (no forces, hashes or
integration), so the CUDA path and the FP64 oracle can both be fed from it
without sharing any computation.

Workloads (Sec. 4 of Tang & Karniadakis describes the paper's own runs; these
are the synthetic stand-ins, with the shapes and densities of those runs):

* ``fluid_small``   -- periodic cube L = 10, rho = 3 (3,000 particles),
  a = 25, gamma = 4.5, kT = 1 (sigma = 3), s = 1, dt = 0.01, lambda = 1/2.
* ``poiseuille``    -- periodic 40 x 20 x 10 box, rho = 4 (32,000 particles),
  a = 18.75, gamma = 4.5, kT = 1, s = 1/2, body force +-0.055 along x on
  the two halves in y, dt = 0.01.
* ``fluid_large``   -- periodic cube L = 100, rho = 3 (3,000,000 particles),
  otherwise as ``fluid_small``.
* ``amphiphile``    -- periodic cube L = 64, rho = 3 (786,432 beads), species
  W/H/T, 10 % of the beads in H1T3 chains with harmonic bonds k = 100,
  r0 = 0.7, a_WW = a_HH = a_TT = a_WH = 25, a_WT = a_HT = 75, dt = 0.005.
* ``serving_stream`` -- the batched-serving workload: a seeded Poisson
  stream of independent periodic cubes, L uniform in 6..30 (integer),
  rho = 3 (648 to 81,000 particles), a uniform in [15, 40], gamma uniform in
  [3, 6], kT = 1, rc = 1, s = 1, dt = 0.01, 500-5000 steps each.
"""
from __future__ import annotations

import numpy as np

SPECIES_W, SPECIES_H, SPECIES_T = 0, 1, 2

# name -> parameters (box, density, pair parameters, step)
CONFIGS = {
    "fluid_small": dict(box=(10.0, 10.0, 10.0), rho=3.0, a=[[25.0]], gamma=4.5, kT=1.0, rc=1.0, s=1.0,
                        dt=0.01, lam=0.5, seed_offset=0),
    "poiseuille": dict(box=(40.0, 20.0, 10.0), rho=4.0, a=[[18.75]], gamma=4.5, kT=1.0, rc=1.0, s=0.5,
                       dt=0.01, lam=0.5, body_mode=2, body=(0.055, 0.0, 0.0), seed_offset=1),
    "fluid_large": dict(box=(100.0, 100.0, 100.0), rho=3.0, a=[[25.0]], gamma=4.5, kT=1.0, rc=1.0, s=1.0,
                        dt=0.01, lam=0.5, seed_offset=2),
    "amphiphile": dict(box=(64.0, 64.0, 64.0), rho=3.0,
                       a=[[25.0, 25.0, 75.0], [25.0, 25.0, 75.0], [75.0, 75.0, 25.0]],
                       gamma=4.5, kT=1.0, rc=1.0, s=1.0, dt=0.005, lam=0.5, k_bond=100.0, r0_bond=0.7,
                       chain_fraction=0.10, seed_offset=3),
}

BASE_SEED = 1234
TEA_SEED = 42
# neighbour-list skin of the throughput benchmark (and of the full-size tests
# that check its configuration); the fastest of 0.3 / 0.4 / 0.5 measured on
# the 3M fluid
BENCH_SKIN = 0.4


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def maxwell(n: int, kT: float, g: np.random.Generator) -> np.ndarray:
    """Gaussian velocities of variance kT per component, zero total momentum."""
    v = g.standard_normal((n, 3)) * np.sqrt(kT)
    v -= v.mean(axis=0, keepdims=True)
    return v


def uniform_fluid(box, n: int, kT: float, seed: int):
    """n particles uniform in the box, Maxwell velocities; tags 0..n-1."""
    g = rng(seed)
    box = np.asarray(box, np.float64)
    x = g.random((n, 3)) * box
    v = maxwell(n, kT, g)
    return x, v


def n_particles(box, rho) -> int:
    return int(round(rho * float(np.prod(box))))


def make(name: str, seed: int | None = None, box=None):
    """Draw the initial state of a named workload.

    Returns a dict with x, v (n x 3 float64), species (int32 or None), bonds
    ((m, 2) uint32 particle indices or None) and the parameter dict."""
    cfg = dict(CONFIGS[name])
    if box is not None:
        cfg["box"] = tuple(float(b) for b in box)
    if seed is None:
        seed = BASE_SEED + cfg["seed_offset"]
    n = n_particles(cfg["box"], cfg["rho"])
    species = None
    bonds = None
    if name == "amphiphile":
        x, v, species, bonds = amphiphile_state(cfg["box"], n, cfg["kT"], cfg["chain_fraction"],
                                                cfg["r0_bond"], seed)
    else:
        x, v = uniform_fluid(cfg["box"], n, cfg["kT"], seed)
    return dict(x=x, v=v, species=species, bonds=bonds, cfg=cfg, n=n, seed=seed)


def amphiphile_state(box, n: int, kT: float, chain_fraction: float, r0: float, seed: int):
    """Random mixture of W beads and H1T3 chains (bead order H, T, T, T).

    Chains start at a uniform point and continue as random walks with step
    length r0; every other bead is a uniform W bead.  Bonds join consecutive
    beads of a chain."""
    g = rng(seed)
    box = np.asarray(box, np.float64)
    n_chain = int(round(chain_fraction * n / 4.0))
    nb = 4 * n_chain
    x = np.empty((n, 3), np.float64)
    species = np.full(n, SPECIES_W, np.int32)
    start = g.random((n_chain, 3)) * box
    steps = g.standard_normal((n_chain, 3, 3))
    steps *= r0 / np.linalg.norm(steps, axis=2, keepdims=True)
    pos = np.empty((n_chain, 4, 3))
    pos[:, 0] = start
    for k in range(3):
        pos[:, k + 1] = pos[:, k] + steps[:, k]
    x[:nb] = np.mod(pos.reshape(-1, 3), box)
    species[:nb] = np.tile(np.array([SPECIES_H, SPECIES_T, SPECIES_T, SPECIES_T], np.int32), n_chain)
    x[nb:] = g.random((n - nb, 3)) * box
    v = maxwell(n, kT, g)
    b = np.arange(n_chain, dtype=np.uint32)[:, None] * 4 + np.arange(3, dtype=np.uint32)[None, :]
    bonds = np.stack([b.reshape(-1), b.reshape(-1) + 1], axis=1).astype(np.uint32)
    return x, v, species, bonds


def serving_stream(nboxes: int, seed: int = BASE_SEED + 5, L_range=(6, 30), steps_range=(500, 5000),
                   rate: float | None = None, with_state: bool = True):
    """A list of independent boxes for the serving workload, each a dict with
    box, a, gamma, kT, rc, s, dt, steps, seed (its random-force key) and, with
    with_state, x and v; and, when rate (boxes per second) is given, Poisson
    arrival times t_arrive (exponential gaps, first arrival at 0)."""
    g = rng(seed)
    out = []
    t = 0.0
    for k in range(nboxes):
        L = float(g.integers(L_range[0], L_range[1] + 1))
        a = float(g.uniform(15.0, 40.0))
        gamma = float(g.uniform(3.0, 6.0))
        steps = int(g.integers(steps_range[0], steps_range[1] + 1))
        box = (L, L, L)
        b = dict(box=box, a=[[a]], gamma=gamma, kT=1.0, rc=1.0, s=1.0, dt=0.01, lam=0.5, steps=steps,
                 seed=int(TEA_SEED + k), n=n_particles(box, 3.0))
        if rate is not None:
            if k > 0:
                t += float(g.exponential(1.0 / rate))
            b["t_arrive"] = t
        if with_state:
            b["x"], b["v"] = uniform_fluid(box, b["n"], 1.0, int(g.integers(1 << 31)))[:2]
        out.append(b)
    return out
