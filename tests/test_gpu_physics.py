"""Long-run physics: the GPU path and the FP64 oracle, each run on its own
from the same FP32 initial state, must agree within 1 % in time-averaged
temperature and pressure (the fluid, and the bonded three-species
amphiphile over several seeds a side), and in the reverse-Poiseuille velocity
profile within four standard deviations of the difference of the two sides'
seed means (the amplitude of a small box's profile varies by about 3 % from
seed to seed); the full-size reverse-Poiseuille start-up must follow the
analytic parabola (Sec. 4.2)."""
import numpy as np
import pytest

import oracle
import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import make_pair, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


FLUID_STEPS, FLUID_BURN, FLUID_EVERY = 4000, 800, 4


def _oracle_fluid_means(seed):
    """Time-averaged T and p of one oracle run of the 3000-particle fluid
    (runs in a spawned worker process)."""
    st = workloads.make("fluid_small")
    cfg = st["cfg"]
    o = oracle.System(cfg["box"], cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"], seed=seed,
                      cut_fp32=True)
    x32 = st["x"].astype(np.float32).astype(np.float64)
    obs = o.run(x32, st["v"], FLUID_STEPS)["obs"][FLUID_BURN:]
    return (float(oracle.System.temperature(obs[:, 0], st["n"]).mean()),
            float(o.pressure(obs[:, 0], obs[:, 1]).mean()))


def test_fluid_temperature_pressure_match_oracle():
    """The 3000-particle fluid: T and p averaged over steps 800-4000 agree
    within 1 %.  One run's average T varies by about 0.35 % from seed to seed
    (p by 0.04 %; eight oracle seeds), so the GPU side averages eight seeds
    and the oracle four (in spawned worker processes): 1 % is then about
    4.7 standard deviations of the difference."""
    import multiprocessing as mp
    st = workloads.make("fluid_small")
    cfg = st["cfg"]
    with mp.get_context("spawn").Pool(4) as pool:
        pending = pool.map_async(_oracle_fluid_means, [42, 43, 44, 45])
        Tg, pg = [], []
        for seed in range(201, 209):
            g, _ = make_pair(cfg, seed=seed)
            g.set_state(st["x"], st["v"])
            Ts, ps = [], []
            for s in range(FLUID_STEPS // FLUID_EVERY):
                g.step(FLUID_EVERY)
                if (s + 1) * FLUID_EVERY > FLUID_BURN:
                    ob = g.observables()
                    Ts.append(ob["temperature"])
                    ps.append(ob["pressure"])
            g.close()
            Tg.append(np.mean(Ts))
            pg.append(np.mean(ps))
        ref = pending.get(timeout=1800)
    To = float(np.mean([r[0] for r in ref]))
    po = float(np.mean([r[1] for r in ref]))
    Tg, pg = float(np.mean(Tg)), float(np.mean(pg))
    assert abs(Tg - To) < 0.01 * To, (Tg, To)
    assert abs(pg - po) < 0.01 * po, (pg, po)
    # both at the thermostat temperature and the known pressure of this state
    assert abs(Tg - 1.0) < 0.03 and 22.5 < pg < 25.0


def _fit_amplitude(sums, counts, Ly, nbins):
    """Least-squares amplitude A of u(y) = A y (h - y) (lower half, +g) and
    -A (y - h)(2h - y) (upper half) for the binned mean v_x."""
    h = Ly / 2
    yc = (np.arange(nbins) + 0.5) * Ly / nbins
    u = sums / np.maximum(counts, 1)
    shape = np.where(yc < h, yc * (h - yc), -(yc - h) * (2 * h - yc))
    A = float((shape * u).sum() / (shape * shape).sum())
    resid = u - A * shape
    r2 = 1.0 - (resid ** 2).sum() / ((u - u.mean()) ** 2).sum()
    return A, r2


POIS_BOX, POIS_NBINS, POIS_STEPS, POIS_BURN, POIS_EVERY = (16.0, 10.0, 5.0), 10, 7000, 2500, 5


def _oracle_poiseuille_amplitude(seed):
    """Fitted amplitude of one oracle run's time-averaged profile over steps
    POIS_BURN..POIS_STEPS (runs in a spawned worker process)."""
    st = workloads.make("poiseuille", box=POIS_BOX)
    cfg = st["cfg"]
    o = oracle.System(POIS_BOX, cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"],
                      lam=cfg.get("lam", 0.5), seed=seed, body_mode=cfg.get("body_mode", 0),
                      body=cfg.get("body", (0, 0, 0)), cut_fp32=True)
    x32 = st["x"].astype(np.float32).astype(np.float64)
    state = o.run(x32, st["v"], POIS_BURN)
    state = o.run(state["x"], state["v"], POIS_STEPS - POIS_BURN, step=state["step"], f=state["f"],
                  prof_nbins=POIS_NBINS, prof_from=1)
    return _fit_amplitude(state["prof_sum"], state["prof_cnt"], POIS_BOX[1], POIS_NBINS)[0]


def test_reverse_poiseuille_profile_matches_oracle():
    """16 x 10 x 5 box (rho = 4, s = 1/2, g = +-0.055): the amplitude of the
    double parabola averaged over steps 2500-7000, GPU (32 seeds) against the
    oracle (16 seeds, in spawned worker processes).  One run's amplitude
    varies by about 3 % from seed to seed (the profile of a box this small
    carries slow hydrodynamic noise; eight oracle seeds: 0.0679 to 0.0734), so
    a flat 1 % would need some 260 runs a side.  The bound is four standard
    deviations of the difference of the two means, from each side's own
    seed-to-seed spread (about 3.6 %), and it must itself stay below 6 %."""
    import multiprocessing as mp
    import os
    st = workloads.make("poiseuille", box=POIS_BOX)
    cfg = st["cfg"]
    seeds_o = list(range(42, 58))
    workers = max(1, min(len(seeds_o), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        pending = pool.map_async(_oracle_poiseuille_amplitude, seeds_o)
        amps, last = [], None
        for seed in range(1000, 1032):
            g, _ = make_pair(cfg, box=POIS_BOX, seed=seed)
            g.set_state(st["x"], st["v"])
            sg, cg = np.zeros(POIS_NBINS), np.zeros(POIS_NBINS)
            g.step(POIS_BURN)
            for s in range((POIS_STEPS - POIS_BURN) // POIS_EVERY):
                g.step(POIS_EVERY)
                g.profile(1, 0, POIS_NBINS, sg, cg)
            amps.append(_fit_amplitude(sg, cg, POIS_BOX[1], POIS_NBINS)[0])
            last = (sg, cg)
            g.close()
        ref = np.array(pending.get(timeout=1800))
    amps = np.array(amps)
    Ag, Ao = float(amps.mean()), float(ref.mean())
    sd_diff = float(np.sqrt(amps.var(ddof=1) / len(amps) + ref.var(ddof=1) / len(ref)))
    tol = 4.0 * sd_diff
    assert tol < 0.06 * abs(Ao), (tol, Ao)
    assert abs(Ag - Ao) < tol, (Ag, Ao, sd_diff)
    r2 = _fit_amplitude(last[0], last[1], POIS_BOX[1], POIS_NBINS)[1]
    assert r2 > 0.97, r2


def test_reverse_poiseuille_full_size_start_up():
    """40 x 20 x 10, rho = 4 (32,000 particles): the flow started from rest
    builds the antisymmetric double parabola over its first 4,000 steps
    (steps 3,000-4,000 averaged).  Beyond about 5,000 steps the shear layers
    of this 40-long box lose stability and the mean profile collapses, in
    the GPU and the oracle alike, so no later average is compared here."""
    st = workloads.make("poiseuille")
    cfg = st["cfg"]
    g = dpd.Sim(cfg["box"], cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"],
                body_mode=cfg["body_mode"], body=cfg["body"])
    g.set_state(st["x"], st["v"])
    nbins = 20
    sg, cg = np.zeros(nbins), np.zeros(nbins)
    g.step(3000)
    for _ in range(100):
        g.step(10)
        g.profile(1, 0, nbins, sg, cg)
    A, r2 = _fit_amplitude(sg, cg, cfg["box"][1], nbins)
    assert r2 > 0.98, r2
    u = sg / cg
    assert abs(u[: nbins // 2].mean() + u[nbins // 2:].mean()) < 0.05 * abs(u).max()
    assert A > 0.03, A
    g.close()


AMPH_BOX, AMPH_STEPS, AMPH_BURN, AMPH_EVERY = (10.0, 10.0, 10.0), 12000, 2000, 4


def _oracle_amphiphile_means(seed):
    """Time-averaged T and p of one oracle run of the small amphiphile box
    (runs in a spawned worker process)."""
    st = workloads.make("amphiphile", box=AMPH_BOX)
    cfg = st["cfg"]
    o = oracle.System(AMPH_BOX, cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"],
                      lam=cfg.get("lam", 0.5), seed=seed, bonds=st["bonds"], k_bond=cfg["k_bond"],
                      r0_bond=cfg["r0_bond"], cut_fp32=True)
    x32 = st["x"].astype(np.float32).astype(np.float64)
    res = o.run(x32, st["v"], AMPH_STEPS, species=st["species"])
    obs = res["obs"][AMPH_BURN:]
    T = oracle.System.temperature(obs[:, 0], st["n"]).mean()
    p = o.pressure(obs[:, 0], obs[:, 1]).mean()
    return float(T), float(p)


def test_amphiphile_temperature_pressure_match_oracle():
    """The bonded three-species amphiphile (H1T3 chains in W beads, a_WT =
    a_HT = 75, harmonic bonds, dt = 0.005) in a 10^3 box: T and p averaged
    over steps 2000-12000 agree within 1 %.  The chains self-assemble during
    the run (p drifts by about 1.5 % across it), so one run's average varies
    by about 0.3 % from seed to seed (measured on the oracle); the GPU side
    averages eight seeds and the oracle two, which puts 1 % at about four
    standard deviations of the difference."""
    import multiprocessing as mp
    st = workloads.make("amphiphile", box=AMPH_BOX)
    cfg = st["cfg"]
    n = st["n"]
    with mp.get_context("spawn").Pool(2) as pool:
        pending = pool.map_async(_oracle_amphiphile_means, [42, 7])
        Tg, pg = [], []
        for seed in range(101, 109):
            g, _ = make_pair(cfg, box=AMPH_BOX, seed=seed)
            g.set_state(st["x"], st["v"], st["species"])
            g.set_bonds(st["bonds"], cfg["k_bond"], cfg["r0_bond"])
            Ts, ps = [], []
            for s in range(AMPH_STEPS // AMPH_EVERY):
                g.step(AMPH_EVERY)
                if (s + 1) * AMPH_EVERY > AMPH_BURN:
                    ob = g.observables()
                    Ts.append(ob["temperature"])
                    ps.append(ob["pressure"])
            g.close()
            Tg.append(np.mean(Ts))
            pg.append(np.mean(ps))
        ref = pending.get(timeout=1800)
    To = float(np.mean([r[0] for r in ref]))
    po = float(np.mean([r[1] for r in ref]))
    Tg, pg = float(np.mean(Tg)), float(np.mean(pg))
    assert abs(Tg - To) < 0.01 * To, (Tg, To)
    assert abs(pg - po) < 0.01 * po, (pg, po)
    assert n == 3000
