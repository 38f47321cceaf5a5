"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs: neighbour sets and RNG integers bit-exact, forces within 1e-4 of the
RMS force (max over all particles and components), observables and short
trajectories within the tolerances stated per test."""
import numpy as np
import pytest

import oracle
import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import force_error, make_pair, need_gpu, pair_set

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4  # relative to the RMS force, max over particles/components


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_pair_rng_bit_exact():
    rng = np.random.default_rng(5)
    m = 200_000
    ti = rng.integers(0, 2**32, m, dtype=np.uint64).astype(np.uint32)
    tj = rng.integers(0, 2**32, m, dtype=np.uint64).astype(np.uint32)
    for seed, step in [(42, 0), (42, 12345), ((7 << 32) | 99, 2**32 + 5)]:
        hh, xi = dpd.dpd_pair_rng(seed, step, ti, tj)
        # every pair's two hash words, bit for bit
        ref = oracle.pair_hash_batch(seed, step, ti, tj)
        assert np.array_equal(hh, ref)
        xr = oracle.xi_batch(seed, step, ti, tj)
        assert np.abs(xi - xr).max() < 2e-5 * max(1.0, np.abs(xr).max())
        hh2, _ = dpd.dpd_pair_rng(seed, step, tj, ti)
        assert np.array_equal(hh, hh2)


def test_pair_rng_extreme_words():
    # u1 near 1 and near 0, all phase quadrants: exercise both -ln branches
    ti = np.arange(0, 4096, dtype=np.uint32)
    tj = ti + 100_000
    hh, xi = dpd.dpd_pair_rng(42, 3, ti, tj)
    xr = oracle.xi_batch(42, 3, ti, tj)
    assert np.abs(xi - xr).max() < 2e-5 * max(1.0, np.abs(xr).max())


ALL = ["fluid_small", "poiseuille_small", "amphiphile_small", "dense_small", "tiny_box"]


@pytest.mark.parametrize("deterministic", [0, 1])
@pytest.mark.parametrize("name", ALL)
def test_neighbors_bit_exact(name, deterministic):
    st, cfg, box, bonds = _workload(name)
    g, o = make_pair(cfg, box=box, deterministic=deterministic)
    g.set_state(st["x"], st["v"], st["species"])
    x32, _, _ = g.state()
    rl = cfg["rc"] + 0.3
    ref = oracle.pairs_fp32(x32, box, rl)
    got = g.neighbors()
    assert pair_set(got) == pair_set(ref)
    assert len(got) == len(ref)


def _workload(name):
    if name == "dense_small":
        # rho = 8: brick halos overflow the staging buffer (global-index rows)
        box = (8.0, 8.0, 8.0)
        x, v = workloads.uniform_fluid(box, 4096, 1.0, 77)
        cfg = dict(workloads.CONFIGS["fluid_small"], box=box)
        return dict(x=x, v=v, species=None, n=4096), cfg, box, None
    if name == "tiny_box":
        # 2 cells per axis: no bricks, the per-particle builder and force path
        box = (3.2, 3.5, 2.9)
        x, v = workloads.uniform_fluid(box, 98, 1.0, 78)
        cfg = dict(workloads.CONFIGS["fluid_small"], box=box)
        return dict(x=x, v=v, species=None, n=98), cfg, box, None
    if name == "fluid_small":
        st = workloads.make("fluid_small")
        return st, st["cfg"], st["cfg"]["box"], None
    if name == "poiseuille_small":
        st = workloads.make("poiseuille", box=(12.0, 10.0, 6.0))
        return st, st["cfg"], (12.0, 10.0, 6.0), None
    if name == "amphiphile_small":
        st = workloads.make("amphiphile", box=(12.0, 12.0, 12.0))
        return st, st["cfg"], (12.0, 12.0, 12.0), st["bonds"]
    raise KeyError(name)


@pytest.mark.parametrize("deterministic", [0, 1])
@pytest.mark.parametrize("name", ALL)
def test_forces_match_oracle(name, deterministic):
    st, cfg, box, bonds = _workload(name)
    g, o = make_pair(cfg, box=box, bonds=bonds, deterministic=deterministic)
    g.set_state(st["x"], st["v"], st["species"], step=17)
    if bonds is not None:
        g.set_bonds(bonds, cfg["k_bond"], cfg["r0_bond"])
    x32, v32, step = g.state()
    assert step == 17
    fo, _ = o.forces(x32, v32, species=st["species"], step=17)
    fg = g.forces()
    err, rms = force_error(fg, fo)
    assert err < FORCE_TOL, (err, rms)
    # the integrator's stored force is the same evaluation (bit-identical
    # when sums run in a fixed order)
    if deterministic:
        assert np.abs(g.force() - fg).max() == 0.0
    else:
        assert force_error(g.force(), fg)[0] < 1e-6


@pytest.mark.parametrize("deterministic", [0, 1])
@pytest.mark.parametrize("s_exp", [0.25, 0.75, 2.0])
def test_forces_general_weight_exponent(s_exp, deterministic):
    """w_R = w^s for exponents other than 1 and 1/2 (Eq. 8): the general
    exp2(s log2 w) path of the pair kernel, and its s = 2 specialisation."""
    st = workloads.make("fluid_small")
    cfg = dict(st["cfg"])
    cfg["s"] = s_exp
    g, o = make_pair(cfg, deterministic=deterministic)
    g.set_state(st["x"], st["v"], step=5)
    x32, v32, _ = g.state()
    fo, _ = o.forces(x32, v32, step=5)
    err, rms = force_error(g.forces(), fo)
    assert err < FORCE_TOL, (err, rms)


def test_observables_match_oracle():
    st = workloads.make("fluid_small")
    cfg = st["cfg"]
    g, o = make_pair(cfg)
    g.set_state(st["x"], st["v"])
    x32, v32, _ = g.state()
    _, vir = o.forces(x32, v32)
    ob = g.observables()
    v2 = (v32 ** 2).sum()
    assert abs(ob["temperature"] - v2 / (3 * st["n"] - 3)) < 1e-9 * v2
    assert abs(ob["virial"] - vir) < 1e-5 * abs(vir)
    assert np.abs(ob["momentum"] - v32.sum(0)).max() < 1e-9 * np.abs(v32).sum()


def test_short_trajectory_matches_oracle():
    """A few steps from the same FP32 state: positions, velocities and the
    force agree before FP32 rounding has had time to grow."""
    st = workloads.make("fluid_small")
    cfg = st["cfg"]
    g, o = make_pair(cfg)
    g.set_state(st["x"], st["v"], step=3)
    x32, v32, _ = g.state()
    f0, _ = o.forces(x32, v32, step=3)
    res = o.run(x32, v32, 1, step=3, f=f0)
    g.step(1)
    xg, vg, sg = g.state()
    assert sg == 4 and res["step"] == 4
    dx = xg - res["x"]
    dx -= np.asarray(cfg["box"]) * np.round(dx / np.asarray(cfg["box"]))
    assert np.abs(dx).max() < 1e-5
    err, _ = force_error(g.force(), res["f"])
    assert err < 1e-3, err
    assert np.abs(vg - res["v"]).max() < 1e-3


def test_step_counter_and_rebuilds_progress():
    st = workloads.make("fluid_small")
    g, _ = make_pair(st["cfg"])
    g.set_state(st["x"], st["v"])
    r0 = g.info()["rebuilds"]
    g.step(37)
    _, _, step = g.state()
    assert step == 37
    assert g.info()["rebuilds"] > r0
    ob = g.observables()
    assert abs(ob["momentum"]).max() < 1e-2


def test_atomic_insertion_builder_same_pairs():
    """The atomic-insertion list builder (the paper's Table 2 comparison)
    lists the same pairs as the oracle, in another order, and gives the same
    forces."""
    st = workloads.make("fluid_small")
    cfg = st["cfg"]
    g, o = make_pair(cfg, list_builder=1)
    g.set_state(st["x"], st["v"], step=3)
    x32, v32, _ = g.state()
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, cfg["box"], cfg["rc"] + 0.3))
    fo, _ = o.forces(x32, v32, step=3)
    err, rms = force_error(g.forces(), fo)
    assert err < FORCE_TOL, (err, rms)


@pytest.mark.parametrize("deterministic", [0, 1])
def test_no_reorder_ablation_same_physics(deterministic):
    """With the particles kept in load order (the paper's reorder on/off
    comparison) the list and the forces are the same, also after steps that
    rebuild the list."""
    st = workloads.make("fluid_small")
    cfg = st["cfg"]
    g, o = make_pair(cfg, no_reorder=1, deterministic=deterministic)
    g.set_state(st["x"], st["v"], step=3)
    x32, v32, step = g.state()
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, cfg["box"], cfg["rc"] + 0.3))
    fo, _ = o.forces(x32, v32, step=step)
    assert force_error(g.forces(), fo)[0] < FORCE_TOL
    g.step(25)
    assert g.info()["rebuilds"] > 1
    # forces from the list the run last built; the set after a rebuild at the
    # current positions (the list of a run dates from its last rebuild)
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, step=step)
    assert force_error(g.forces(), fo)[0] < FORCE_TOL
    g.build_neighbors()
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, cfg["box"], cfg["rc"] + 0.3))


@pytest.mark.parametrize("name", ["fluid_small", "poiseuille_small", "amphiphile_small", "dense_small"])
def test_row_layout_matches_oracle(name):
    """The paper's list layout (Sec. 3.3): one row per particle with the core
    pairs inserted from the front and the skin pairs from the back, the two
    parts joined, each 32 x 32 tile transposed in place, and one thread per
    particle in the pair force.  The same pairs as the oracle's FP32
    predicate, the same forces within the tolerance, and after steps that
    rebuild the list (regrowing the rows in the dense box) still both."""
    st, cfg, box, bonds = _workload(name)
    g, o = make_pair(cfg, box=box, bonds=bonds, list_layout=1)
    g.set_state(st["x"], st["v"], st["species"], step=11)
    if bonds is not None:
        g.set_bonds(bonds, cfg["k_bond"], cfg["r0_bond"])
    x32, v32, step = g.state()
    rl = cfg["rc"] + 0.3
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, box, rl))
    fo, _ = o.forces(x32, v32, species=st["species"], step=step)
    err, rms = force_error(g.forces(), fo)
    assert err < FORCE_TOL, (err, rms)
    g.step(20)
    assert g.info()["rebuilds"] > 1
    # the forces use the list the run last built (a superset of the pairs
    # inside r_c at the current positions); the set is compared after a
    # rebuild at the current positions
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, species=st["species"], step=step)
    err, rms = force_error(g.forces(), fo)
    assert err < FORCE_TOL, (err, rms)
    g.build_neighbors()
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, box, rl))
    g.close()


def test_row_layout_trajectory_equals_packed_deterministic():
    """Both layouts evaluate every pair from both particles and sum each force
    in a fixed order; two row-layout runs of 30 steps are bit-identical, and
    over 5 steps the two layouts agree to rounding (their summation orders
    differ)."""
    st = workloads.make("fluid_small")
    cfg = st["cfg"]
    runs = []
    for layout, nsteps in ((1, 30), (1, 30), (1, 5), (0, 5)):
        g, _ = make_pair(cfg, deterministic=1, list_layout=layout)
        g.set_state(st["x"], st["v"])
        g.step(nsteps)
        runs.append(g.state())
        g.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    dx = runs[2][0] - runs[3][0]
    dx -= np.asarray(cfg["box"]) * np.round(dx / np.asarray(cfg["box"]))
    assert np.abs(dx).max() < 1e-5
    assert np.abs(runs[2][1] - runs[3][1]).max() < 1e-3


def test_row_layout_needs_three_cells_per_axis():
    box = (3.2, 3.5, 2.9)  # 2 cells per axis
    with pytest.raises(dpd.DPDError) as e:
        dpd.Sim(box, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, list_layout=1)
    assert e.value.status == 1
