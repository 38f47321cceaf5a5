"""Serving loop (include/dpd_server.h): boxes of different sizes and
parameters admitted by device memory and run concurrently give the same
result as each box run alone, the admission respects the memory budget, and
the per-box times are consistent.  Each box is the oracle-checked engine of
the other GPU tests; these tests check the scheduling around it."""
import time

import numpy as np
import pytest

import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

CHUNK = 40


def _boxes(n, seed, L_range=(6, 14), steps_range=(60, 160)):
    return workloads.serving_stream(n, seed=seed, L_range=L_range, steps_range=steps_range)


def _alone(b, deterministic):
    """The box run by itself through the plain path, in the server's chunks."""
    sim = dpd.Sim(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], seed=b["seed"],
                  deterministic=deterministic)
    sim.set_state(b["x"], b["v"])
    left = b["steps"]
    while left > 0:
        c = min(CHUNK, left)
        sim.step(c)
        left -= c
    x, v, step = sim.state()
    ob = sim.observables()
    sim.close()
    return x, v, step, ob


def _mix(boxes, deterministic, max_active=8, budget=0.0):
    srv = dpd.Server(max_active=max_active, chunk_steps=CHUNK, deterministic=deterministic, mem_budget_bytes=budget)
    tickets = [srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                          b["steps"], seed=b["seed"]) for b in boxes]
    out = [srv.wait(t, timeout_s=300.0) for t in tickets]
    srv.close()
    return out


def test_alone_and_in_the_mix_are_bit_identical():
    need_gpu()
    boxes = _boxes(12, seed=11)
    mixed = _mix(boxes, deterministic=1)
    for b, r in zip(boxes, mixed):
        assert r["status"] == 0
        x, v, step, ob = _alone(b, 1)
        assert step == b["steps"] and r["obs"]["step"] == b["steps"]
        assert np.array_equal(r["x"], x) and np.array_equal(r["v"], v), "box L=%g" % b["box"][0]
        assert r["obs"]["temperature"] == ob["temperature"] and r["obs"]["virial"] == ob["virial"]


def test_newton3_mix_within_tolerance():
    # float reductions make the last bits of a Newton-3 run vary run to run,
    # alone or not; over a short run the states agree to FP32 rounding growth
    need_gpu()
    boxes = _boxes(6, seed=12, steps_range=(30, 40))
    mixed = _mix(boxes, deterministic=0, max_active=6)
    for b, r in zip(boxes, mixed):
        assert r["status"] == 0
        x, v, _, ob = _alone(b, 0)
        d = np.abs(r["x"] - x)
        d = np.minimum(d, np.asarray(b["box"]) - d)  # periodic
        assert d.max() < 1e-3
        assert abs(r["obs"]["temperature"] - ob["temperature"]) < 1e-3 * ob["temperature"]


def test_admission_respects_the_memory_budget():
    need_gpu()
    boxes = _boxes(8, seed=13, L_range=(10, 10), steps_range=(200, 200))
    # the server's estimate for one of these boxes, read while it runs alone
    est = None
    srv = dpd.Server(max_active=8, chunk_steps=CHUNK, mem_budget_bytes=1e12)
    t = srv.submit(boxes[0]["box"], boxes[0]["a"], 4.5, 1.0, 1.0, 1.0, 0.01, boxes[0]["x"], boxes[0]["v"], 400)
    for _ in range(400):
        c = srv.counts()
        if c["running"] == 1:
            est = c["mem_bytes"]
            break
        time.sleep(0.002)
    srv.wait(t)
    srv.close()
    assert est and est > 0
    # a budget that holds two of them
    srv = dpd.Server(max_active=8, chunk_steps=CHUNK, mem_budget_bytes=2.5 * est)
    tickets = [srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                          b["steps"], seed=b["seed"]) for b in boxes]
    peak = 0
    while True:
        c = srv.counts()
        peak = max(peak, c["running"])
        assert c["mem_bytes"] <= 2.5 * est + 1.0
        if c["finished"] == len(boxes):
            break
        time.sleep(0.002)
    res = [srv.wait(t) for t in tickets]
    srv.close()
    assert peak <= 2
    assert all(r["status"] == 0 for r in res)
    # first-fit in submission order: admissions never overtake with equal sizes
    admits = [r["t_admit"] for r in res]
    assert admits == sorted(admits)


def test_times_and_errors():
    need_gpu()
    boxes = _boxes(4, seed=14)
    srv = dpd.Server(max_active=2, chunk_steps=CHUNK)
    tickets = [srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                          b["steps"], seed=b["seed"]) for b in boxes]
    for t in tickets:
        r = srv.wait(t)
        assert r["status"] == 0
        assert 0.0 <= r["t_submit"] <= r["t_admit"] <= r["t_done"] <= srv.now()
    with pytest.raises(dpd.DPDError) as e:
        srv.wait(tickets[0])  # already collected
    assert e.value.status == 1
    with pytest.raises(dpd.DPDError) as e:
        srv.submit((6.0, 6.0, 6.0), [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, np.zeros((0, 3)), np.zeros((0, 3)), 10)
    assert e.value.status == 1
    srv.close()


def test_tune_skin_picks_a_measured_candidate():
    need_gpu()
    st = workloads.make("fluid_small")
    c = st["cfg"]
    # skin 4.0 is too large for the L = 10 box (needs L > 2 (rc + skin)): refused, reported as infinity
    best, table = dpd.dpd_tune_skin(c["box"], c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], st["x"], st["v"],
                                    candidates=(0.2, 0.4, 4.0), steps=40)
    assert best in (0.2, 0.4)
    assert np.isfinite(table[0.2]) and np.isfinite(table[0.4]) and np.isinf(table[4.0])
    assert table[best] == min(table.values())


def test_ensemble_routing_alone_and_in_the_mix():
    """With the ensemble option, boxes that fit the ensemble kernel run there:
    each gives the same bits as the box alone in an ensemble with the same
    chunks; the larger boxes still run on their own handles, as alone."""
    need_gpu()
    boxes = _boxes(10, seed=15, L_range=(6, 14))
    fits = [dpd.dpd_ensemble_fits(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["n"])
            for b in boxes]
    assert any(fits) and not all(fits)
    srv = dpd.Server(max_active=8, chunk_steps=CHUNK, deterministic=1, ensemble=1)
    tickets = [srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                          b["steps"], seed=b["seed"]) for b in boxes]
    mixed = [srv.wait(t, timeout_s=300.0) for t in tickets]
    srv.close()
    for b, f, r in zip(boxes, fits, mixed):
        assert r["status"] == 0 and r["obs"]["step"] == b["steps"]
        if f:
            ens = dpd.Ensemble()
            i = ens.add(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                        seed=b["seed"])
            left = b["steps"]
            while left > 0:
                ens.step(min(CHUNK, left))
                left -= min(CHUNK, left)
            ens.sync()
            x, v, step = ens.state(i)
            ob = ens.observables(i)
            ens.close()
        else:
            x, v, step, ob = _alone(b, 1)
        assert step == b["steps"]
        assert np.array_equal(r["x"], x) and np.array_equal(r["v"], v), "box L=%g" % b["box"][0]
        assert r["obs"]["temperature"] == ob["temperature"] and r["obs"]["virial"] == ob["virial"]


def test_adaptive_ensemble_routing():
    """ensemble = 2: a box that fits the ensemble kernel runs there only when,
    at its admission, every handle slot is busy.  With one slot and a queue of
    small boxes some go each way; each result is bit-identical to the same box
    run alone on the path it took (deterministic mode).  A box submitted to an
    idle server runs on a handle."""
    need_gpu()
    boxes = _boxes(8, seed=21, L_range=(6, 8), steps_range=(300, 400))
    srv = dpd.Server(max_active=1, chunk_steps=CHUNK, deterministic=1, ensemble=2)
    tickets = [srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                          b["steps"], seed=b["seed"]) for b in boxes]
    res = [srv.wait(t, timeout_s=300.0) for t in tickets]
    engines = [r["engine"] for r in res]
    assert 0 in engines and 1 in engines, engines
    for b, r in zip(boxes, res):
        assert r["status"] == 0 and r["obs"]["step"] == b["steps"]
        if r["engine"] == 1:
            ens = dpd.Ensemble()
            i = ens.add(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                        seed=b["seed"])
            left = b["steps"]
            while left > 0:
                ens.step(min(CHUNK, left))
                left -= min(CHUNK, left)
            ens.sync()
            x, v, step = ens.state(i)
            ens.close()
        else:
            x, v, step, _ = _alone(b, 1)
        assert np.array_equal(r["x"], x) and np.array_equal(r["v"], v)
    # light load: one box into an idle server takes a handle
    b = boxes[0]
    t = srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"], b["steps"],
                   seed=b["seed"])
    assert srv.wait(t, timeout_s=300.0)["engine"] == 0
    srv.close()
