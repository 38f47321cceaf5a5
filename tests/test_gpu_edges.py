"""Edge cases of the GPU path: degenerate particle counts, a dense clump
(neighbour capacity grows), particles on cell faces, argument and
call-order errors, determinism, and checkpoint / resume."""
import numpy as np
import pytest

import oracle
import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import force_error, make_pair, need_gpu, pair_set

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


CFG = workloads.CONFIGS["fluid_small"]


def test_single_and_pair():
    g, o = make_pair(CFG)
    g.set_state(np.array([[5.0, 5, 5]]), np.array([[0.1, 0, 0]]))
    assert np.all(g.forces() == 0.0)
    assert len(g.neighbors()) == 0
    g.step(3)
    g.set_state(np.array([[5.5, 5, 5], [5.0, 5, 5]]), np.zeros((2, 3)), step=1)
    x32, v32, _ = g.state()
    fo, _ = o.forces(x32, v32, step=1)
    assert np.abs(g.forces() - fo).max() < 1e-4 * np.abs(fo).max()


def test_dense_clump_grows_capacity():
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.random((400, 3)) * 0.8 + 4.0, rng.random((2000, 3)) * 10.0])
    v = rng.standard_normal(x.shape)
    g, o = make_pair(CFG)
    g.set_state(x, v)
    # the automatic capacity for the mean density is 64; the clump needs more
    assert g.info()["nbr_capacity"] > 128
    x32, v32, _ = g.state()
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, CFG["box"], 1.3))
    fo, _ = o.forces(x32, v32)
    err, _ = force_error(g.forces(), fo)
    assert err < 1e-4


def test_particles_on_cell_faces():
    # 7 cells of side 10/7 per axis: place particles exactly on faces and corners
    side = 10.0 / 7.0
    grid = np.arange(7) * side
    xs = np.array(np.meshgrid(grid, grid, grid[:3], indexing="ij")).reshape(3, -1).T
    x = np.concatenate([xs, xs + np.array([0.65, 0.0, 0.0])])
    v = np.zeros_like(x)
    g, o = make_pair(CFG)
    g.set_state(x, v)
    x32, v32, _ = g.state()
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, CFG["box"], 1.3))
    fo, _ = o.forces(x32, v32)
    err, _ = force_error(g.forces(), fo)
    assert err < 1e-4


def test_argument_and_state_errors():
    g = dpd.Sim(CFG["box"], CFG["a"], 4.5, 1.0, 1.0, 1.0, 0.01)
    with pytest.raises(dpd.DPDError) as e:
        g.step(1)
    assert e.value.status == 7  # DPD_ERR_STATE
    with pytest.raises(dpd.DPDError) as e:
        g.set_state(np.zeros((0, 3)), np.zeros((0, 3)))
    assert e.value.status == 1
    with pytest.raises(dpd.DPDError) as e:
        g.set_state(np.ones((3, 3)), np.zeros((3, 3)), species=np.array([0, 1, 0]))
    assert e.value.status == 1
    with pytest.raises(dpd.DPDError) as e:
        g.set_state(np.ones((3, 3)), np.zeros((3, 3)), tag=np.array([4, 4, 5]))
    assert e.value.status == 1
    x = np.ones((3, 3))
    x[1, 2] = np.nan
    with pytest.raises(dpd.DPDError):
        g.set_state(x, np.zeros((3, 3)))
    g.close()


def test_deterministic_runs():
    st = workloads.make("fluid_small")
    outs = []
    for _ in range(2):
        g, _ = make_pair(st["cfg"], deterministic=1)
        g.set_state(st["x"], st["v"])
        g.step(57)
        outs.append(g.state())
        g.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_checkpoint_resume():
    st = workloads.make("fluid_small")
    a, _ = make_pair(st["cfg"])
    a.set_state(st["x"], st["v"])
    a.step(30)
    x, v, step = a.state()
    f = a.force()
    b, _ = make_pair(st["cfg"])
    b.set_state(x, v, step=step)
    b.set_force(f)
    a.step(3)
    b.step(3)
    xa, va, sa = a.state()
    xb, vb, sb = b.state()
    assert sa == sb == step + 3
    # the lists differ in build time, so sums differ in rounding order only
    assert np.abs(xa - xb).max() < 1e-5
    assert np.abs(va - vb).max() < 1e-3


def test_newton3_and_deterministic_modes_agree():
    """One evaluation per pair with atomics for the partner, against every pair
    evaluated from both sides in fixed order: same forces within rounding, and
    the same trajectory over a few steps."""
    st = workloads.make("fluid_small")
    a, _ = make_pair(st["cfg"], deterministic=0)
    b, _ = make_pair(st["cfg"], deterministic=1)
    a.set_state(st["x"], st["v"], step=4)
    b.set_state(st["x"], st["v"], step=4)
    assert force_error(a.forces(), b.forces())[0] < 1e-6
    a.step(5)
    b.step(5)
    assert np.abs(a.state()[0] - b.state()[0]).max() < 1e-5


def test_launch_modes_give_identical_trajectories():
    """The same step sequence launched three ways -- captured graphs with the
    rebuild chain under conditional nodes, captured graphs launching the chain
    every step, and eager launches without graphs -- gives bit-identical
    states and the same rebuilds (deterministic mode: fixed summation order).
    Each dpd_step call is one velocity-Verlet unit, so the eager run steps in
    the graphs' 8-step units."""
    st = workloads.make("fluid_small")
    c = st["cfg"]
    outs = []
    for graph_steps, cond, calls in ((8, 1, [48]), (8, 0, [48]), (0, 1, [8] * 6)):
        g = dpd.Sim(c["box"], c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], graph_steps=graph_steps,
                    conditional_rebuild=cond, deterministic=1)
        g.set_state(st["x"], st["v"])
        for k in calls:
            g.step(k)
        x, v, step = g.state()
        outs.append((x, v, step, g.info()["rebuilds"]))
        g.close()
    for x, v, step, rebuilds in outs[1:]:
        assert step == outs[0][2] == 48
        assert rebuilds == outs[0][3] and rebuilds > 2
        assert np.array_equal(x, outs[0][0]) and np.array_equal(v, outs[0][1])


def test_bounded_device_wait_reports_timeout_and_recovers():
    """Failure detection without a fault: the device's bounded wait (the one
    guarding the builder's TMA-staged halos) on a transaction that nothing
    delivers gives up, the host reads DPD_ERR_TIMEOUT, and the handle keeps
    working."""
    st = workloads.make("fluid_small")
    c = st["cfg"]
    g, o = make_pair(c)
    g.set_state(st["x"], st["v"])
    assert dpd.dpd_wait_selftest(g.h, 256) == 6  # DPD_ERR_TIMEOUT
    g.step(10)
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, step=step)
    assert force_error(g.forces(), fo)[0] < 1e-4
