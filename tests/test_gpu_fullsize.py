"""Parity at the full sizes of the workloads, in the configuration the
benchmark runs (its skin, CUDA graphs): every force of the 3M-particle
fluid, the 786k-bead amphiphile (3 species, harmonic bonds) and the 32k
reverse-Poiseuille box against the FP64 oracle (1e-4 of the RMS force, max
over all particles), sampled neighbour rows of the 3M fluid bit-exact, and
the forces again after steps (the stepping path at scale)."""
import numpy as np
import pytest

import oracle
import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import force_error, make_pair, need_gpu

pytestmark = pytest.mark.gpu
FORCE_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def large():
    st = workloads.make("fluid_large")
    g, o = make_pair(st["cfg"], skin=workloads.BENCH_SKIN)
    g.set_state(st["x"], st["v"], step=11)
    yield st, g, o
    g.close()


def test_fluid_large_forces_all_particles(large):
    st, g, o = large
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, step=step)
    err, rms = force_error(g.forces(), fo)
    assert err < FORCE_TOL, (err, rms)


def test_fluid_large_neighbor_rows_sampled(large):
    st, g, o = large
    x32, _, _ = g.state()
    pairs = g.neighbors()
    rl = st["cfg"]["rc"] + workloads.BENCH_SKIN
    rng = np.random.default_rng(3)
    sample = rng.choice(st["n"], 128, replace=False)
    # neighbours of i from the GPU pair list (both orientations)
    lo = np.searchsorted(pairs[:, 0], sample)
    for idx, i in enumerate(sample):
        ref = oracle.neighbors_of(x32, st["cfg"]["box"], rl, int(i))
        a = pairs[pairs[:, 0] == i, 1]
        b = pairs[pairs[:, 1] == i, 0]
        got = np.sort(np.concatenate([a, b]))
        assert np.array_equal(got, ref), int(i)


def test_fluid_large_after_steps(large):
    st, g, o = large
    g.step(12)
    x32, v32, step = g.state()
    assert step == 23
    fo, _ = o.forces(x32, v32, step=step)
    err, _ = force_error(g.forces(), fo)
    assert err < FORCE_TOL, err


def test_amphiphile_full_size_forces():
    st = workloads.make("amphiphile")
    cfg = st["cfg"]
    g, o = make_pair(cfg, bonds=st["bonds"])
    g.set_state(st["x"], st["v"], st["species"], step=2)
    g.set_bonds(st["bonds"], cfg["k_bond"], cfg["r0_bond"])
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, species=st["species"], step=step)
    err, rms = force_error(g.forces(), fo)
    assert err < FORCE_TOL, (err, rms)
    g.step(10)
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, species=st["species"], step=step)
    err, _ = force_error(g.forces(), fo)
    assert err < FORCE_TOL, err
    g.close()


def test_poiseuille_full_size_forces():
    st = workloads.make("poiseuille")
    g, o = make_pair(st["cfg"])
    g.set_state(st["x"], st["v"], step=4)
    g.step(25)
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, step=step)
    err, _ = force_error(g.forces(), fo)
    assert err < FORCE_TOL, err
    g.close()
