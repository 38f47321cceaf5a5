"""Edge cases of the GPU path: degenerate particle counts, a dense clump
(neighbour capacity grows), particles on cell faces, argument and
call-order errors, determinism, and checkpoint / resume."""
import ctypes

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
    # the particle count is checked before any array is read: one past the
    # 2^27 a list entry can index is refused (the C call, small buffers)
    buf = np.zeros((3, 3))
    ptr = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert dpd.lib().dpd_set_state(g.h, (1 << 27) + 1, ptr, ptr, None, None, 0) == 1  # DPD_ERR_ARG
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


def _edge_units(L, rl):
    """Pairs of particles whose FP32 predicate distance d^2 is exactly
    fp32(r_list)^2, one ulp below it and one ulp above it, each pair straddling
    a periodic face (x, y and z in turn).  Built by a search over FP32
    positions with the predicate's rounding (numpy float32 arithmetic, every
    operation rounded on its own); the oracle then decides membership."""
    f32 = np.float32
    Lf, h = f32(L), f32(0.5) * f32(L)
    rl2 = f32(f32(rl) * f32(rl))
    targets = {"eq": rl2, "prev": np.nextafter(rl2, f32(0)), "next": np.nextafter(rl2, f32(10))}

    def d2(a, b):
        d = []
        for k in range(3):
            t = f32(b[k] - a[k])
            t = f32(t - Lf) if t > h else (f32(t + Lf) if t < -h else t)
            d.append(t)
        return f32(f32(f32(d[0] * d[0]) + f32(d[1] * d[1])) + f32(d[2] * d[2]))

    units = []
    slots = {"eq": (4.5, 4.5), "prev": (4.5, 7.5), "next": (7.5, 4.5)}
    for axis in range(3):
        other, third = (axis + 1) % 3, (axis + 2) % 3
        for name, tgt in targets.items():
            hit = None
            for base_t in np.linspace(rl - 0.02, rl - 0.06, 41):
                for high_side in (True, False):
                    xi = np.zeros(3, f32)
                    xi[other], xi[third] = f32(slots[name][0]), f32(slots[name][1])
                    xi[axis] = f32(L - 0.35) if high_side else f32(0.3)
                    xj = xi.copy()
                    xj[axis] = f32((float(xi[axis]) + (base_t if high_side else -base_t)) % L)
                    need = float(tgt) - float(d2(xi, xj))
                    y0 = f32(float(xi[other]) + np.sqrt(need))
                    cands, a, b = [y0], y0, y0
                    for _ in range(30):
                        a, b = np.nextafter(a, f32(-1)), np.nextafter(b, f32(100))
                        cands += [a, b]
                    for y in cands:
                        x2 = xj.copy()
                        x2[other] = y
                        if d2(xi, x2) == tgt:
                            hit = (xi, x2)
                            break
                    if hit:
                        break
                if hit:
                    break
            assert hit is not None, (axis, name)
            units.append((name, hit[0], hit[1]))
    return units, targets


@pytest.mark.parametrize("deterministic", [0, 1])
def test_neighbor_predicate_edges_across_periodic_faces(deterministic):
    """Pairs placed at d^2 = r_list^2 and one ulp either side of it, across the
    periodic faces: the GPU builder keeps exactly the pairs the oracle's FP32
    predicate keeps (strict d^2 < r_list^2)."""
    L = 12.0
    cfg = dict(CFG, box=(L, L, L))
    units, targets = _edge_units(L, cfg["rc"] + 0.3)
    x = np.array([p for _, a, b in units for p in (a, b)], np.float64)
    g, _ = make_pair(cfg, box=cfg["box"], deterministic=deterministic)
    g.set_state(x, np.zeros_like(x))
    x32, _, _ = g.state()
    assert np.array_equal(x32, x)  # the FP32 positions arrive unchanged
    ref = oracle.pairs_fp32(x32, cfg["box"], cfg["rc"] + 0.3)
    # the construction hits the edge: each unit's own distance is the target
    for k, (name, a, b) in enumerate(units):
        assert np.float32(oracle.fp32_d2(a, b, cfg["box"])) == targets[name]
    want = {(2 * k, 2 * k + 1) for k, (name, _, _) in enumerate(units) if name == "prev"}
    assert pair_set(ref) == pair_set(np.array(sorted(want), np.uint32))
    assert pair_set(g.neighbors()) == pair_set(ref)
    g.close()


def test_allocation_failure_leaves_handle_unchanged(monkeypatch):
    """Host-made allocation failure (DPD_TEST_FAIL_ALLOC=1 refuses every
    device allocation without reaching the allocator): creating a handle and
    loading a state report DPD_ERR_OOM, and a handle whose load was refused
    keeps its previous state and goes on stepping."""
    st = workloads.make("fluid_small")
    c = st["cfg"]
    g, o = make_pair(c)
    g.set_state(st["x"], st["v"], step=3)
    x0, v0, s0 = g.state()
    monkeypatch.setenv("DPD_TEST_FAIL_ALLOC", "1")
    with pytest.raises(dpd.DPDError) as e:
        dpd.Sim(c["box"], c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"])
    assert e.value.status == 2  # DPD_ERR_OOM
    with pytest.raises(dpd.DPDError) as e:
        g.set_state(st["x"][::-1].copy(), st["v"][::-1].copy(), step=77)
    assert e.value.status == 2
    monkeypatch.delenv("DPD_TEST_FAIL_ALLOC")
    x1, v1, s1 = g.state()
    assert s1 == s0 and np.array_equal(x1, x0) and np.array_equal(v1, v0)
    g.step(5)
    x2, v2, s2 = g.state()
    fo, _ = o.forces(x2, v2, step=s2)
    assert s2 == s0 + 5 and force_error(g.forces(), fo)[0] < 1e-4
    g.close()


@pytest.mark.parametrize("deterministic", [0, 1])
def test_force_overflow_during_a_step_latches_nonfinite(deterministic):
    """Finite inputs whose force overflows FP32 inside a step: two particles
    1.3 apart (no force at load) close to 0.4 in the first step, where the
    conservative term a w / r with a = 3e38 exceeds the FP32 range.  The
    device latches its non-finite flag, dpd_step returns DPD_ERR_NONFINITE,
    and the handle accepts a new state afterwards."""
    c = dict(CFG, a=[[3.0e38]])
    g, _ = make_pair(c, deterministic=deterministic)
    x = np.array([[5.0, 5.0, 5.0], [6.3, 5.0, 5.0]])
    v = np.array([[45.0, 0.0, 0.0], [-45.0, 0.0, 0.0]])
    g.set_state(x, v)
    assert np.all(np.isfinite(g.forces()))
    with pytest.raises(dpd.DPDError) as e:
        g.step(1)
    assert e.value.status == 5  # DPD_ERR_NONFINITE
    g.set_state(np.array([[5.0, 5.0, 5.0], [7.0, 5.0, 5.0]]), np.zeros((2, 3)))
    g.step(2)
    assert np.all(np.isfinite(g.state()[0]))
    g.close()


def test_async_observables_match_sync_every_step():
    """dpd_observables_async queued behind single steps gives, once synced,
    the same bits dpd_observables returns for each of those states (the same
    run repeated with a host wait per step), with consecutive step numbers;
    a destination that is not page-locked is refused."""
    st = workloads.make("fluid_small")
    c = st["cfg"]
    k = 6

    def run():
        # deterministic mode: two runs of the same state are bit-identical
        return dpd.Sim(c["box"], c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], seed=3, deterministic=1)

    a = run()
    a.set_state(st["x"], st["v"])
    buf = dpd.ObsBuffer(k)
    for i in range(k):
        a.step_async(1)
        a.observables_async(buf, i)
    a.sync()
    got = [buf.get(i) for i in range(k)]
    b = run()
    b.set_state(st["x"], st["v"])
    want = []
    for i in range(k):
        b.step(1)
        want.append(b.observables())
    for g_, w_ in zip(got, want):
        for key in ("step", "n", "kinetic", "temperature", "virial", "pressure"):
            assert g_[key] == w_[key], (key, g_[key], w_[key])
        assert np.array_equal(g_["momentum"], w_["momentum"])
    assert [g_["step"] for g_ in got] == list(range(1, k + 1))
    pageable = dpd.dpd_obs()
    with pytest.raises(dpd.DPDError):
        dpd.dpd_observables_async(a.h, ctypes.addressof(pageable))
    # the refusal leaves the handle usable
    a.step(1)
    assert a.observables()["step"] == k + 1
    a.close()
    b.close()


@pytest.mark.parametrize("deterministic", [0, 1])
def test_coincident_particles(deterministic):
    """Pairs at r = 0 (60 particles moved onto others of the fluid): the list
    keeps them (d^2 = 0 < r_list^2, as the oracle's FP32 brute force does), the
    pair contributes no force on either side (e_ij is undefined there), every
    other force matches the oracle, and steps stay finite."""
    st = workloads.make("fluid_small")
    x = st["x"].copy()
    x[3000 - 60:] = x[:60]
    g, o = make_pair(CFG, deterministic=deterministic)
    g.set_state(x, st["v"], step=2)
    x32, v32, _ = g.state()
    assert np.array_equal(x32[3000 - 60:], x32[:60])
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, CFG["box"], 1.3))
    fo, _ = o.forces(x32, v32, step=2)
    err, _ = force_error(g.forces(), fo)
    assert err < 1e-4, err
    g.step(5)
    xs, vs, _ = g.state()
    assert np.isfinite(xs).all() and np.isfinite(vs).all()
    g.close()
