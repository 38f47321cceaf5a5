"""Ensemble kernel (include/dpd_ensemble.h): many small boxes, one cluster
of CTAs per box, the box resident in shared memory for a chunk of steps.

Against the FP64 oracle on the same seeded inputs: the initial force within
1e-4 of the RMS force (max over particles and components), for one and two
species, the general weight exponent and lambda != 1/2; a short trajectory
within the tolerances of the engine's own trajectory test.  Determinism: a
box's trajectory is bit-identical whatever the cluster size, block size and
the other boxes of the launch.  Physics: temperature and pressure of a long
run agree with the neighbour-list engine within statistical error."""
import numpy as np
import pytest

import oracle
import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import force_error, need_gpu

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _fluid(L, seed, rho=3.0, kT=1.0):
    box = (float(L),) * 3
    n = workloads.n_particles(box, rho)
    x, v = workloads.uniform_fluid(box, n, kT, seed)[:2]
    return box, x, v


def _add(ens, box, x, v, a=25.0, gamma=4.5, s=1.0, lam=0.5, seed=42, step=0, species=None, dt=0.01, **kw):
    a_ij = np.atleast_2d(np.asarray(a, np.float64))
    return ens.add(box, a_ij, gamma, 1.0, 1.0, s, dt, x, v, species=species, step=step, lam=lam, seed=seed, **kw)


@pytest.mark.parametrize("case", ["one_species", "two_species", "s_quarter", "lambda_065"])
def test_initial_force_matches_oracle(case):
    box, x, v = _fluid(8, 101)
    a, s, lam, sp = 25.0, 1.0, 0.5, None
    if case == "two_species":
        a = [[25.0, 60.0], [60.0, 25.0]]
        sp = (np.arange(x.shape[0]) % 2).astype(np.int32)
    elif case == "s_quarter":
        s = 0.25
    elif case == "lambda_065":
        lam = 0.65
    ens = dpd.Ensemble()
    i = _add(ens, box, x, v, a=a, s=s, lam=lam, step=9, species=sp)
    x32, v32, step = ens.state(i)
    assert step == 9
    o = oracle.System(box, a, 4.5, 1.0, 1.0, s, 0.01, lam=lam, seed=42, cut_fp32=True)
    fo, vir = o.forces(x32, v32, species=sp, step=9)
    fg = ens.forces(i)
    err, rms = force_error(fg, fo)
    assert err < FORCE_TOL, (err, rms)
    ob = ens.observables(i)
    assert abs(ob["virial"] - vir) < 1e-5 * abs(vir)
    assert np.abs(ob["momentum"] - v32.sum(0)).max() < 1e-9 * np.abs(v32).sum()
    ens.close()


@pytest.mark.parametrize("lam", [0.5, 0.65])
def test_short_trajectory_matches_oracle(lam):
    box, x, v = _fluid(9, 102)
    ens = dpd.Ensemble(cluster=4)
    i = _add(ens, box, x, v, lam=lam, step=3)
    x32, v32, _ = ens.state(i)
    o = oracle.System(box, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, lam=lam, seed=42, cut_fp32=True)
    f0, _ = o.forces(x32, v32, step=3)
    res = o.run(x32, v32, 2, step=3, f=f0)
    ens.step(2)
    ens.sync()
    xg, vg, sg = ens.state(i)
    assert sg == 5 and res["step"] == 5
    dx = xg - res["x"]
    dx -= np.asarray(box) * np.round(dx / np.asarray(box))
    assert np.abs(dx).max() < 1e-5
    err, _ = force_error(ens.forces(i), res["f"])
    assert err < 1e-3, err
    assert np.abs(vg - res["v"]).max() < 1e-3
    ens.close()


def _run(boxes, threads, cluster, steps, chunks=2):
    ens = dpd.Ensemble(threads=threads, cluster=cluster)
    ids = [_add(ens, b["box"], b["x"], b["v"], a=b["a"], gamma=b["gamma"], seed=b["seed"]) for b in boxes]
    for _ in range(chunks):
        ens.step(steps)
    ens.sync()
    out = [(ens.state(i), ens.observables(i)) for i in ids]
    ens.close()
    return out


def test_bit_identical_across_shapes_and_mixes():
    boxes = workloads.serving_stream(5, seed=21, L_range=(6, 10), steps_range=(10, 10))
    alone = _run(boxes[:1], 128, 1, 25)[0]
    for threads, cluster in ((256, 2), (512, 8), (256, 4)):
        mixed = _run(boxes, threads, cluster, 25)
        (x, v, step), ob = mixed[0]
        assert step == 50
        assert np.array_equal(x, alone[0][0]) and np.array_equal(v, alone[0][1]), (threads, cluster)
        assert ob["temperature"] == alone[1]["temperature"] and ob["virial"] == alone[1]["virial"]


def test_per_box_steps_and_ids():
    boxes = workloads.serving_stream(3, seed=22, L_range=(6, 8), steps_range=(10, 10))
    ens = dpd.Ensemble()
    ids = [_add(ens, b["box"], b["x"], b["v"], seed=b["seed"]) for b in boxes]
    ens.step([5, 0, 12], ids=ids)
    ens.step(3, ids=[ids[1]])
    ens.sync()
    assert [ens.state(i)[2] for i in ids] == [5, 3, 12]
    # box 2 run alone in one 12-step chunk: the same state (a chunk boundary
    # rounds phase 2 and the next phase 1 separately, so the split must match)
    ens2 = dpd.Ensemble()
    j = _add(ens2, boxes[2]["box"], boxes[2]["x"], boxes[2]["v"], seed=boxes[2]["seed"])
    ens2.step(12)
    ens2.sync()
    assert np.array_equal(ens2.state(j)[0], ens.state(ids[2])[0])
    ens.remove(ids[0])
    assert ens.info()[0] == 2
    with pytest.raises(dpd.DPDError):
        ens.state(ids[0])
    ens.close()
    ens2.close()


SEEDS = 8  # boxes (random-force seeds) per side of a long-run comparison


def test_thermodynamics_match_the_engine():
    """rho = 3, a = 25, kT = 1 in an L = 10 box: temperature and pressure over
    a long run, eight boxes in one ensemble against eight runs of the
    neighbour-list engine (independent random streams).  One run's average T
    varies by about 0.35 % from seed to seed, so the means over eight a side
    are compared within 1 % (about 5.7 standard deviations of their
    difference)."""
    box, x, v = _fluid(10, 103)
    ens = dpd.Ensemble()
    ids = [_add(ens, box, x, v, seed=42 + k) for k in range(SEEDS)]
    ens.step(500)
    te, pe = [], []
    for _ in range(200):
        ens.step(20)
        ens.sync()
        obs = [ens.observables(i) for i in ids]
        te.append(np.mean([o["temperature"] for o in obs]))
        pe.append(np.mean([o["pressure"] for o in obs]))
    assert max(abs(ens.observables(i)["momentum"]).max() for i in ids) < 1e-2
    ens.close()
    ts, ps = [], []
    for k in range(SEEDS):
        sim = dpd.Sim(box, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, deterministic=1, seed=142 + k)
        sim.set_state(x, v)
        sim.step(500)
        for _ in range(200):
            sim.step(20)
            b = sim.observables()
            ts.append(b["temperature"])
            ps.append(b["pressure"])
        sim.close()
    Te, Pe, Ts, Ps = np.mean(te), np.mean(pe), np.mean(ts), np.mean(ps)
    assert abs(Te - 1.0) < 0.03 and 22.5 < Pe < 25.0
    assert abs(Te - Ts) < 0.01 * Ts, (Te, Ts)
    assert abs(Pe - Ps) < 0.01 * Ps, (Pe, Ps)


def test_reverse_poiseuille_body_force():
    box, x, v = _fluid(8, 104)
    ens = dpd.Ensemble()
    i = _add(ens, box, x, v, body_mode=2, body=(0.3, 0.0, 0.0))
    ens.step(400)
    ens.sync()
    xg, vg, _ = ens.state(i)
    low = xg[:, 1] < box[1] / 2
    assert vg[low, 0].mean() > 0.1 and vg[~low, 0].mean() < -0.1
    ens.close()


def test_limits_and_errors():
    assert dpd.dpd_ensemble_fits((10.0,) * 3, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, 3000)
    assert not dpd.dpd_ensemble_fits((20.0,) * 3, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, 24000)
    assert not dpd.dpd_ensemble_fits((2.9,) * 3, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, 10)
    ens = dpd.Ensemble()
    box, x, v = _fluid(6, 105)
    bad = x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(dpd.DPDError) as e:
        _add(ens, box, bad, v)
    assert e.value.status == 1
    with pytest.raises(dpd.DPDError) as e:
        _add(ens, (20.0,) * 3, np.zeros((24000, 3)), np.zeros((24000, 3)))
    assert e.value.status == 1
    assert ens.info() == (0, 0)
    with pytest.raises(dpd.DPDError):
        ens.step(5, ids=[7])
    ens.close()


def test_tuner_picks_a_measured_shape():
    boxes = workloads.serving_stream(24, seed=23, L_range=(6, 10), steps_range=(10, 10))
    ens = dpd.Ensemble()
    ids = [_add(ens, b["box"], b["x"], b["v"], seed=b["seed"]) for b in boxes]
    before = [ens.state(i)[0] for i in ids[:3]]
    table = ens.tune(steps=10)
    finite = {k: t for k, t in table.items() if np.isfinite(t)}
    assert finite and all(t > 0 for t in finite.values())
    threads, cluster = ens.config()
    assert any(t in (128, 256, 512) for t in threads)
    # tuning runs on copies: the boxes have not moved
    for i, x0 in zip(ids[:3], before):
        x1, _, step = ens.state(i)
        assert step == 0 and np.array_equal(x0, x1)
    ens.step(10)
    ens.sync()
    assert ens.state(ids[0])[2] == 10
    ens.close()


def _largest_fitting_n(box):
    lo, hi = 1, 65535
    while lo < hi:  # largest n with fits(n)
        mid = (lo + hi + 1) // 2
        if dpd.dpd_ensemble_fits(box, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, mid):
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("case", ["non_cubic_three_cells", "largest_fitting_box", "two_species_ragged"])
def test_edge_boxes_match_oracle(case):
    """Edge cases of the ensemble kernel against the oracle: a non-cubic box
    with exactly three cells along x (the smallest stencil without repeated
    cells), the largest box one CTA's shared memory holds (its launch steps
    the block size down), and a ragged particle count with two species."""
    sp, a = None, 25.0
    if case == "non_cubic_three_cells":
        box = (3.2, 7.5, 5.1)
        n = workloads.n_particles(box, 3.0)
    elif case == "largest_fitting_box":
        box = (11.0, 11.0, 11.0)
        n = _largest_fitting_n(box)
        assert 3993 < n < 65535  # denser than rho = 3
        assert not dpd.dpd_ensemble_fits(box, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, n + 1)
    else:
        box = (7.3, 6.1, 8.9)
        n = 1187
        a = [[25.0, 40.0], [40.0, 30.0]]
        sp = (np.arange(n) % 3 == 0).astype(np.int32)
    x, v = workloads.uniform_fluid(box, n, 1.0, 106)[:2]
    ens = dpd.Ensemble()
    i = _add(ens, box, x, v, a=a, species=sp, step=4)
    x32, v32, _ = ens.state(i)
    o = oracle.System(box, a, 4.5, 1.0, 1.0, 1.0, 0.01, seed=42, cut_fp32=True)
    fo, vir = o.forces(x32, v32, species=sp, step=4)
    err, rms = force_error(ens.forces(i), fo)
    assert err < FORCE_TOL, (case, n, err, rms)
    assert abs(ens.observables(i)["virial"] - vir) < 1e-5 * abs(vir)
    ens.step(30)
    ens.sync()
    xg, vg, step = ens.state(i)
    assert step == 34 and np.isfinite(xg).all() and np.isfinite(vg).all()
    assert (xg >= 0).all() and (xg < np.asarray(box)).all()
    ens.close()


def test_single_particle_box():
    box = (4.0, 4.0, 4.0)
    ens = dpd.Ensemble()
    i = _add(ens, box, np.array([[1.0, 2.0, 3.0]]), np.array([[0.5, -0.25, 0.125]]))
    assert np.array_equal(ens.forces(i), np.zeros((1, 3)))
    ens.step(10)
    ens.sync()
    x, v, step = ens.state(i)
    # no force: free flight, wrapped
    assert step == 10
    assert np.allclose(v, [[0.5, -0.25, 0.125]], atol=0)
    assert np.allclose(x, np.mod(np.array([[1.0, 2.0, 3.0]]) + 10 * 0.01 * v, 4.0), atol=1e-5)
    ens.close()


@pytest.mark.parametrize("cluster", [1, 4])
@pytest.mark.parametrize("case", ["one_species", "s_quarter", "non_cubic_three_cells", "two_species"])
def test_newton3_forces_match_oracle(case, cluster):
    """Newton-3 mode (half stencil, the partner's share added by an atomic in
    the shared memory of the CTA that owns it, across the cluster with 4 CTAs
    per box): the same forces within 1e-4 of the RMS force."""
    box, x, v = _fluid(8, 107)
    a, s, sp = 25.0, 1.0, None
    if case == "s_quarter":
        s = 0.25
    elif case == "non_cubic_three_cells":
        box = (3.2, 7.5, 5.1)
        x, v = workloads.uniform_fluid(box, workloads.n_particles(box, 3.0), 1.0, 108)[:2]
    elif case == "two_species":
        a = [[25.0, 60.0], [60.0, 25.0]]
        sp = (np.arange(x.shape[0]) % 2).astype(np.int32)
    ens = dpd.Ensemble(newton3=1, cluster=cluster)
    i = _add(ens, box, x, v, a=a, s=s, species=sp, step=6)
    x32, v32, _ = ens.state(i)
    o = oracle.System(box, a, 4.5, 1.0, 1.0, s, 0.01, seed=42, cut_fp32=True)
    fo, vir = o.forces(x32, v32, species=sp, step=6)
    err, rms = force_error(ens.forces(i), fo)
    assert err < FORCE_TOL, (case, err, rms)
    assert abs(ens.observables(i)["virial"] - vir) < 1e-5 * abs(vir)
    ens.close()


def test_newton3_trajectory_and_thermodynamics():
    box, x, v = _fluid(9, 109)
    ens = dpd.Ensemble(newton3=1, cluster=2)
    i = _add(ens, box, x, v, step=3)
    x32, v32, _ = ens.state(i)
    o = oracle.System(box, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, seed=42, cut_fp32=True)
    f0, _ = o.forces(x32, v32, step=3)
    res = o.run(x32, v32, 2, step=3, f=f0)
    ens.step(2)
    ens.sync()
    xg, vg, _ = ens.state(i)
    dx = xg - res["x"]
    dx -= np.asarray(box) * np.round(dx / np.asarray(box))
    assert np.abs(dx).max() < 1e-5 and np.abs(vg - res["v"]).max() < 1e-3
    # long run against the deterministic mode (independent rounding, same
    # physics): eight boxes (seeds) a side, means compared within 1 %
    ens.remove(i)
    ids3 = [_add(ens, box, x, v, seed=42 + k) for k in range(SEEDS)]
    det = dpd.Ensemble()
    idsd = [_add(det, box, x, v, seed=142 + k) for k in range(SEEDS)]
    ens.step(500)
    det.step(500)
    t3, p3, td, pd = [], [], [], []
    for _ in range(200):
        ens.step(20)
        det.step(20)
        ens.sync()
        det.sync()
        a = [ens.observables(k) for k in ids3]
        b = [det.observables(k) for k in idsd]
        t3.append(np.mean([o["temperature"] for o in a])); p3.append(np.mean([o["pressure"] for o in a]))
        td.append(np.mean([o["temperature"] for o in b])); pd.append(np.mean([o["pressure"] for o in b]))
    assert abs(np.mean(t3) - np.mean(td)) < 0.01 * np.mean(td), (np.mean(t3), np.mean(td))
    assert abs(np.mean(p3) - np.mean(pd)) < 0.01 * np.mean(pd), (np.mean(p3), np.mean(pd))
    assert max(abs(ens.observables(k)["momentum"]).max() for k in ids3) < 1e-2
    ens.close()
    det.close()


def test_chunk_launches_replay_a_captured_graph():
    """Step calls with the same boxes per class replay one captured CUDA graph
    (the step counts travel in the device descriptors), and the trajectory is
    the same bit for bit as with a fresh capture for every call (another
    ensemble whose structure changes between calls)."""
    box, x, v = _fluid(7, 141)
    a = dpd.Ensemble()
    i = _add(a, box, x, v)
    for k in (5, 7, 5, 9):
        a.step(k)
    a.sync()
    cap, rep = a.graph_stats()
    # the first call also computes the initial force (its own structure)
    assert cap == 2 and rep == 2, (cap, rep)
    b = dpd.Ensemble()
    j = _add(b, box, x, v)
    box2, x2, v2 = _fluid(6, 142)
    for n, k in enumerate((5, 7, 5, 9)):
        # a second box added and removed between calls changes the structure
        extra = _add(b, box2, x2, v2) if n % 2 == 0 else None
        b.step(k, ids=[j] if extra is None else [j, extra])
        b.sync()
        if extra is not None:
            b.remove(extra)
    xa, va, sa = a.state(i)
    xb, vb, sb = b.state(j)
    assert sa == sb == 26
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    a.close()
    b.close()
