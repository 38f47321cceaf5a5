#!/usr/bin/env python
"""Throughput benchmark: particle-steps/s of the 3,000,000-particle DPD fluid
(periodic cube L = 100, rho = 3, a = 25, gamma = 4.5, kT = 1, s = 1,
dt = 0.01) on one GB300, through the C ABI of libdpd.so.

A step is one full pass of the hot path: velocity-Verlet phase 1 with the
per-particle signature and displacement check, the cell/reorder/neighbour
chain (runs on the steps where a particle has moved more than skin/2), the
fused pair force, and phase 2.  The timed region is K steps replayed from
CUDA graphs, timed with CUDA events on the library's stream; the working
set (positions, velocities, forces, reference positions and the neighbour
table, ~0.9 GB) is larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own independent box (no data
exchange: replicas), timing is the max over ranks after a barrier, and the
value is the aggregate particle-steps/s.  ``--impl reference`` times the FP64
CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# more hardware work queues than the default 8, so that the serving leg's
# per-box streams run concurrently (read when CUDA initialises)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "particle-steps/s (3M-particle DPD fluid, 1 GB300)"
UNIT = "particle-steps/s"
WORKLOAD = "fluid_large"
# ALU peak from unit counts and clock: 152 SMs x 128 FP32/INT32 lanes x 2.07 GHz
ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12
# algorithmic lane-ops per unique interacting pair (distance, weights,
# TEA-4 pair hash, Box-Muller, force, accumulation on both particles)
OPS_PER_PAIR = 100.0
# per particle and step: the half kick, drift, wrap, full kick and
# displacement test of the lambda form of velocity Verlet
OPS_INTEGRATE = 25.0
PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end leg (0: as many as the timed device leg)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-boxes", type=int, default=512)
    ap.add_argument("--serve-active", type=int, default=32)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--small-boxes", type=int, default=256,
                    help="boxes of the ensemble-kernel leg (0 skips it)")
    ap.add_argument("--no-tune", action="store_true", help="skip the skin tuner's measurement of the 3M system")
    ap.add_argument("--ablations", action="store_true",
                    help="also time the atomic-insertion list builder against the ballot one (Table 2), "
                         "reorder on/off and the paper's row list layout against the packed lists")
    ap.add_argument("--no-conditional", action="store_true",
                    help="launch the rebuild chain in every step's graph (for profilers that do not enter "
                         "conditional graph nodes)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.windows = []

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self):
        return time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 10:
                        continue
                    try:
                        ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                        frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                        rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[6:10], parts[5]))
                    except Exception:
                        continue
        except Exception:
            pass
        sel = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15] or rows[-5:]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in sel for k in range(4) if r[3][k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max(r[2] for r in sel),
                "reasons": reasons, "samples": len(sel)}


def slowest(pg, local, device):
    """The largest of every rank's `local` (the job's wall time is its
    slowest rank's); `local` itself without a process group."""
    if not pg:
        return float(local)
    import torch
    t = torch.tensor([float(local)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, per_rank_units, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank has the same work)."""
    return ws * per_rank_units / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kernel_traffic():
    """DRAM bytes per force-kernel launch from the committed ncu summary, if
    it was taken on the current kernel source (else None)."""
    path = os.path.join(PROFILES, "force_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        src = open(os.path.join(ROOT, "paper_1311_0402_gb300", "csrc", "kernels_force.cu"), "rb").read()
        if rec.get("kernels_force_sha256") != hashlib.sha256(src).hexdigest():
            return None
        return rec["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


def host_cores():
    """Host cores this process may run on (read at run time)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def bench_config(workload, n, ws):
    """The `config` of the JSON line (the same for both arms)."""
    return {"workload": "%s: periodic L=100 rho=3 DPD fluid (%d particles per GPU), a=25 gamma=4.5 kT=1 "
                        "s=1 dt=0.01 lambda=0.5, skin %g, displacement-triggered rebuilds" % (
                            workload, n, _bench_skin()),
            "parallelism": "replicas" if ws > 1 else "single", "l2": "working set > L2 (no flush)"}


def _bench_skin():
    import workloads
    return workloads.BENCH_SKIN


def _oracle_worker(workload, box, seed, nsteps, warmup, barrier, out):
    """One host core: the single-threaded FP64 oracle on its own copy of the
    sample (drawn from the same seeded workload), started at a common barrier."""
    import oracle
    import workloads
    cfg = workloads.CONFIGS[workload]
    st = workloads.make(workload, seed=seed, box=box)
    sysm = oracle.System(box, cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"], lam=cfg["lam"])
    f, _ = sysm.forces(st["x"], st["v"], step=0)
    res = {"x": st["x"], "v": st["v"], "f": f, "step": 0}
    if warmup:
        res = sysm.run(res["x"], res["v"], warmup, f=res["f"], step=res["step"])
    barrier.wait()
    t0 = time.time()
    sysm.run(res["x"], res["v"], nsteps, f=res["f"], step=res["step"])
    out.put((t0, time.time(), st["n"] * nsteps))


def oracle_all_cores(workload, box, nsteps, warmup=0, cores=None):
    """Particle-steps/s of the unmodified single-threaded oracle run on every
    host core at once: one spawned process per core, each stepping its own
    copy of the sample; the rate is the work of all of them over the span
    from the common start to the last finish.  Returns (rate, cores, seconds)."""
    import multiprocessing as mp
    cores = cores or host_cores()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(workload, box, 9000 + k, nsteps, warmup, barrier, q))
             for k in range(cores)]
    for p in procs:
        p.start()
    rows = [q.get() for _ in procs]
    for p in procs:
        p.join()
    span = max(r[1] for r in rows) - min(r[0] for r in rows)
    return sum(r[2] for r in rows) / span, cores, span


def oracle_rate(x, v, cfg, nsteps, box):
    """Particle-steps/s of the FP64 oracle (single-threaded C) on a state."""
    import oracle
    sysm = oracle.System(box, cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"], lam=cfg["lam"])
    f0, _ = sysm.forces(x, v, step=0)
    t0 = time.perf_counter()
    sysm.run(x, v, nsteps, f=f0)
    dt = time.perf_counter() - t0
    return x.shape[0] * nsteps / dt, dt


def run_reference(args):
    """The oracle as the reference arm: FP64 CPU on every host core (one
    single-threaded oracle process per core), each core stepping its own
    sub-box of the same fluid, sized so the whole run takes about a minute."""
    import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cfg = workloads.CONFIGS[args.workload]
    import oracle
    # size the sub-box so that warm-up + timed steps take about a minute:
    # time a short probe run on one core, then scale the particle count
    probe = workloads.make(args.workload, box=(8.0, 8.0, 8.0))
    psys = oracle.System((8.0, 8.0, 8.0), cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"],
                         lam=cfg["lam"])
    t0 = time.perf_counter()
    psys.run(probe["x"], probe["v"], 10)
    rate = probe["n"] * 10 / max(time.perf_counter() - t0, 1e-6)
    n_target = rate * 60.0 / max(args.steps + args.warmup, 1)
    Ls = float(min(30.0, max(6.0, round((n_target / cfg["rho"]) ** (1.0 / 3.0)))))
    sub = (Ls, Ls, Ls)
    n_sub = workloads.n_particles(sub, cfg["rho"])
    value, cores, el = oracle_all_cores(args.workload, sub, args.steps, warmup=args.warmup)
    n_full = workloads.n_particles(cfg["box"], cfg["rho"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.workload, n_full, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "FP64 oracle (single-threaded C) in %d processes, one per host core, each "
                                   "stepping its own %g^3 sub-box of the same fluid (%d particles, rho=3; the sub-box is "
                                   "sized for at most about a minute of work)" % (cores, Ls, n_sub)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Batched serving leg: the seeded stream of independent boxes (L in 6..30,
    rho = 3, a in [15, 40], gamma in [3, 6], 500-5000 steps) run (1) one box at
    a time through the plain path, (2) all submitted at once to the serving
    loop, (3) submitted at Poisson arrival times, 1.2x the one-box-at-a-time
    capacity, for p50 / p99 time-to-completion."""
    import paper_1311_0402_gb300 as dpd
    import workloads
    boxes = workloads.serving_stream(args.serve_boxes, with_state=True)
    total = float(sum(b["n"] * b["steps"] for b in boxes))
    # skin per size class, chosen by the tuner on a representative box of each
    classes = [(0, 12, 9.0), (13, 21, 17.0), (22, 1000, 26.0)]
    tuned = {}
    for lo, hi, L in classes:
        probe = workloads.serving_stream(1, seed=777, L_range=(int(L), int(L)), with_state=True)[0]
        best, table = dpd.dpd_tune_skin(probe["box"], [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, probe["x"], probe["v"],
                                        candidates=(0.2, 0.3, 0.4, 0.5, 0.6), steps=300)
        tuned[(lo, hi)] = (best, table)

    def skin_of(b):
        for (lo, hi), (best, _) in tuned.items():
            if lo <= b["box"][0] <= hi:
                return best
        return 0.3

    for b in boxes:
        b["skin"] = skin_of(b)
    # (1) one box at a time, plain path: create, load, step, read back, free
    t0 = time.perf_counter()
    for b in boxes:
        sim = dpd.Sim(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], seed=b["seed"], skin=b["skin"],
                      conditional_rebuild=0)
        sim.set_state(b["x"], b["v"])
        sim.step(b["steps"])
        sim.observables()
        sim.state()
        sim.close()
    t_seq = time.perf_counter() - t0

    def submit(srv, b):
        return srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                          b["steps"], seed=b["seed"], skin=b["skin"])

    # (2) saturated: everything queued at once, every box on its own handle;
    # then the same with adaptive routing (a box that fits the ensemble kernel
    # goes there while every handle slot is busy)
    def saturated(ensemble):
        srv = dpd.Server(max_active=args.serve_active, chunk_steps=100, ensemble=ensemble)
        t0 = srv.now()
        tickets = [submit(srv, b) for b in boxes]
        res = [srv.wait(t, timeout_s=3600.0, state=True) for t in tickets]
        srv.close()
        return max(r["t_done"] for r in res) - t0, sum(1 for r in res if r["status"] != 0)

    t_sat, bad = saturated(0)
    t_sat_e, bad_e = saturated(2)
    bad += bad_e
    # (3) Poisson arrivals at 1.2x the one-box-at-a-time capacity
    rate = 1.2 * len(boxes) / t_seq
    arrivals = workloads.serving_stream(args.serve_boxes, with_state=False, rate=rate)

    def poisson(ensemble):
        srv = dpd.Server(max_active=args.serve_active, chunk_steps=100, ensemble=ensemble)
        t0 = srv.now()
        tickets = []
        for b, a in zip(boxes, arrivals):
            dt = a["t_arrive"] - (srv.now() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(submit(srv, b))
        res = [srv.wait(t, timeout_s=3600.0, state=False) for t in tickets]
        srv.close()
        ttc = np.array([r["t_done"] - r["t_submit"] for r in res])
        span = max(r["t_done"] for r in res) - t0
        return {"rate_boxes_per_s": rate, "value": total / span, "unit": UNIT, "wall_s": span,
                "p50_s": float(np.percentile(ttc, 50)), "p99_s": float(np.percentile(ttc, 99)),
                "arrival": "Poisson, 1.2x the one-box-at-a-time capacity"}, sum(1 for r in res if r["status"] != 0)

    pois, b1 = poisson(2)
    pois_plain, b2 = poisson(0)
    bad += b1 + b2
    n_ens = sum(1 for b in boxes if dpd.dpd_ensemble_fits(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"],
                                                          b["dt"], b["n"]))
    return {
        "metric": "batched-ensemble time-to-completion (p50 / p99) and particle-steps/s",
        "boxes": len(boxes), "particle_steps": total, "failed": bad,
        "workload": "seeded stream of independent periodic cubes, L uniform in 6..30, rho=3 (648..81000 "
                    "particles), a in [15,40], gamma in [3,6], kT=1, dt=0.01, 500-5000 steps each",
        "skin_by_box_length": {"L %d-%d" % (lo, min(hi, 30)): {"skin": best, "ms_per_step_tried": table}
                               for (lo, hi), (best, table) in tuned.items()},
        "boxes_fitting_the_ensemble_kernel": n_ens,
        "one_box_at_a_time": {"value": total / t_seq, "unit": UNIT, "wall_s": t_seq},
        "saturated": {"value": total / t_sat, "unit": UNIT, "wall_s": t_sat,
                      "vs_one_box_at_a_time": t_seq / t_sat, "max_active": args.serve_active,
                      "routing": "every box on its own handle (the serving loop's default)"},
        "saturated_ensemble_routing": {"value": total / t_sat_e, "unit": UNIT, "wall_s": t_sat_e,
                                       "vs_one_box_at_a_time": t_seq / t_sat_e, "max_active": args.serve_active,
                                       "routing": "adaptive: a box that fits the ensemble kernel runs there "
                                                  "while every handle slot is busy, else on its own handle"},
        "poisson": dict(pois_plain, routing="every box on its own handle (the serving loop's default)"),
        "poisson_ensemble_routing": dict(pois, routing="adaptive: a box that fits the ensemble kernel runs there "
                                                       "while every handle slot is busy, else on its own handle"),
    }


def run_small_boxes(args):
    """Ensemble kernel leg: a seeded stream of small boxes (L uniform in
    6..10, rho = 3, 500-5000 steps), all resident at once, advanced in chunks
    of 100 steps by the ensemble kernel after its autotuner has chosen threads
    per CTA and CTAs per box; against the serving loop running the same boxes
    each on its own handle, and the plain path one box at a time on a sample."""
    import paper_1311_0402_gb300 as dpd
    import workloads
    boxes = workloads.serving_stream(args.small_boxes, seed=workloads.BASE_SEED + 9, L_range=(6, 10),
                                     with_state=True)
    total = float(sum(b["n"] * b["steps"] for b in boxes))

    def ensemble_run(newton3):
        ens = dpd.Ensemble(newton3=newton3)
        ids = [ens.add(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                       seed=b["seed"]) for b in boxes]
        table = ens.tune(steps=20)
        ens.sync()
        threads, cluster = ens.config()
        left = {i: b["steps"] for i, b in zip(ids, boxes)}
        done = []
        t0 = time.perf_counter()
        while left:
            ks = list(left)
            st = [min(100, left[k]) for k in ks]
            ens.step(st, ids=ks)
            ens.sync()
            now = time.perf_counter() - t0
            for k, c in zip(ks, st):
                left[k] -= c
                if left[k] == 0:
                    del left[k]
                    done.append(now)
        wall = time.perf_counter() - t0
        ens.close()
        done = np.array(done)
        return {"value": total / wall, "unit": UNIT, "wall_s": wall,
                "p50_s": float(np.percentile(done, 50)), "p99_s": float(np.percentile(done, 99)),
                "threads_per_cta_by_class": threads, "ctas_per_box_by_class": cluster,
                "tuner_ms_per_step_last_class": {"%dx%d" % k: v for k, v in table.items()}}

    ens_det = ensemble_run(0)
    ens_n3 = ensemble_run(1)
    srv = dpd.Server(max_active=args.serve_active, chunk_steps=100)
    t1 = srv.now()
    tickets = [srv.submit(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"], b["steps"],
                          seed=b["seed"]) for b in boxes]
    res = [srv.wait(t, timeout_s=3600.0, state=False) for t in tickets]
    srv.close()
    tt = np.array([r["t_done"] - t1 for r in res])
    # one box at a time on every 8th box (the plain path is slow here)
    sample = boxes[::8]
    t2 = time.perf_counter()
    for b in sample:
        sim = dpd.Sim(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], seed=b["seed"],
                      conditional_rebuild=0)
        sim.set_state(b["x"], b["v"])
        sim.step(b["steps"])
        sim.observables()
        sim.state()
        sim.close()
    t_seq = time.perf_counter() - t2
    seq_total = float(sum(b["n"] * b["steps"] for b in sample))
    return {
        "workload": "%d seeded periodic cubes, L uniform in 6..10 (648..3000 particles), rho=3, a in [15,40], "
                    "gamma in [3,6], kT=1, dt=0.01, 500-5000 steps each, all submitted at t=0" % len(boxes),
        "particle_steps": total,
        "ensemble_kernel": dict(ens_det, mode="every pair from both sides, fixed order (bit-reproducible)"),
        "ensemble_kernel_newton3": dict(ens_n3, mode="each pair once, partner share by shared-memory atomics"),
        "serving_loop_own_handles": {"value": total / float(tt.max()), "unit": UNIT, "wall_s": float(tt.max()),
                                     "p50_s": float(np.percentile(tt, 50)), "p99_s": float(np.percentile(tt, 99)),
                                     "max_active": args.serve_active},
        "one_box_at_a_time": {"value": seq_total / t_seq, "unit": UNIT, "sample": "every 8th box"},
    }


def run_list_ablation():
    """The paper's Table 2 on this engine: the rebuild chain per rebuild with
    the list entries placed by warp-ballot prefix sums (the default) and by one
    atomic add per entry, for rho = 3 and 6 at 64k and 512k particles."""
    import paper_1311_0402_gb300 as dpd
    import workloads
    out = []
    for rho, n in ((3.0, 65536), (3.0, 524288), (6.0, 65536), (6.0, 524288)):
        L = (n / rho) ** (1.0 / 3.0)
        x, v = workloads.uniform_fluid((L, L, L), n, 1.0, 4321)
        row = {"rho": rho, "n": n}
        for name, lb in (("ballot", 0), ("atomic", 1)):
            sim = dpd.Sim((L, L, L), [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, skin=0.3, list_builder=lb)
            sim.set_state(x, v)
            sim.step(50)
            t = sim.step_profiled(400)
            sim.close()
            row[name + "_ms_per_rebuild"] = t["rebuild_ms"] / max(t["rebuilds"], 1)
        row["atomic_over_ballot"] = row["atomic_ms_per_rebuild"] / row["ballot_ms_per_rebuild"]
        out.append(row)
    return out


def run_layout_ablation():
    """The paper's list layout (Sec. 3.3: rows per particle written with core
    pairs in front and skin pairs at the back, joined, 32 x 32 tiles
    transposed, one thread per particle in the pair force, full lists) against
    the packed group lists, on the 3M fluid: the packed lists with each pair
    once (the default) and with full lists in fixed order (the same work as
    the paper's layout)."""
    import paper_1311_0402_gb300 as dpd
    import workloads
    st = workloads.make("fluid_large")
    c = st["cfg"]
    out = {"workload": "fluid_large (3M), skin %g, 200 steps after 20" % workloads.BENCH_SKIN}
    for name, layout, det in (("packed_newton3", 0, 0), ("packed_full_lists", 0, 1), ("rows_paper_layout", 1, 1)):
        sim = dpd.Sim(c["box"], c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], skin=workloads.BENCH_SKIN,
                      deterministic=det, list_layout=layout)
        sim.set_state(st["x"], st["v"])
        sim.step(20)
        t = sim.step_profiled(200)
        sim.close()
        out[name] = {"ms_per_step": t["total_ms"] / 200, "pair_ms": t["pair_ms"] / 200,
                     "rebuild_ms_per_rebuild": t["rebuild_ms"] / max(t["rebuilds"], 1), "rebuilds": t["rebuilds"]}
    return out


def run_reorder_ablation():
    """The paper's reorder on/off comparison (Sec. 3.2) on the 3M fluid: the
    whole step with the particles reordered into cell order at every rebuild
    (the default) and kept in their load order (uniformly random in space)."""
    import paper_1311_0402_gb300 as dpd
    import workloads
    st = workloads.make("fluid_large")
    c = st["cfg"]
    out = {"workload": "fluid_large (3M, load order uniformly random in space), skin %g" % workloads.BENCH_SKIN}
    for name, nr in (("reordered", 0), ("load_order", 1)):
        sim = dpd.Sim(c["box"], c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], skin=workloads.BENCH_SKIN,
                      no_reorder=nr)
        sim.set_state(st["x"], st["v"])
        sim.step(20)
        t = sim.step_profiled(200)
        sim.close()
        out[name] = {"ms_per_step": t["total_ms"] / 200, "pair_ms": t["pair_ms"] / 200,
                     "rebuild_ms_per_rebuild": t["rebuild_ms"] / max(t["rebuilds"], 1)}
    out["speedup_from_reordering"] = out["load_order"]["ms_per_step"] / out["reordered"]["ms_per_step"]
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = tdist
    import paper_1311_0402_gb300 as dpd
    if rank == 0:
        dpd.build()
    if pg:
        pg.barrier()
    dpd.lib()
    import workloads

    cfg = workloads.CONFIGS[args.workload]
    st = workloads.make(args.workload, seed=workloads.BASE_SEED + cfg["seed_offset"] + 1000 * rank)
    n = st["n"]
    stream = torch.cuda.Stream()
    skin_table = None
    if not args.no_tune:
        # the tuner's measurement for this system (the run below uses the
        # skin the full-size parity tests check)
        _, skin_table = dpd.dpd_tune_skin(cfg["box"], cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"],
                                          cfg["dt"], st["x"], st["v"], candidates=(0.3, 0.4, 0.5), steps=200)
    sim = dpd.Sim(cfg["box"], cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"], lam=cfg["lam"],
                  skin=workloads.BENCH_SKIN, seed=workloads.TEA_SEED, stream=stream.cuda_stream,
                  conditional_rebuild=0 if args.no_conditional else 1)
    sim.set_state(st["x"], st["v"])
    sim.step(args.warmup)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    # ---------------------------------------------------------- timed region
    chunk = 1000
    chunks = [chunk] * (args.steps // chunk) + ([args.steps % chunk] if args.steps % chunk else [])
    for c in sorted(set(chunks)):  # capture the graphs outside the timed region
        sim.step_profiled(c)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    times = []
    for c in chunks:
        times.append(sim.step_profiled(c))
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if pg:
        pg.barrier()
    # ------------------------------------------------------------------------
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    total_ms = sum(t["total_ms"] for t in times)
    force_ms = sum(t["force_ms"] for t in times)
    pair_ms = sum(t["pair_ms"] for t in times)
    force_launches = sum(t["force_launches"] for t in times)
    launches = sum(t["kernel_launches"] for t in times)
    rebuilds = sum(t["rebuilds"] for t in times)
    integ_ms = sum(t["integrate_ms"] for t in times)
    rebuild_ms = sum(t["rebuild_ms"] for t in times)
    max_ms = slowest(pg, total_ms, "cuda")
    value = job_rate(ws, n * args.steps, max_ms / 1e3)

    # roofline of the dominant kernel (the fused pair force)
    rho = n / float(np.prod(cfg["box"]))
    pairs_per_particle = 0.5 * rho * 4.0 / 3.0 * np.pi * cfg["rc"] ** 3
    ops_per_launch = n * pairs_per_particle * OPS_PER_PAIR
    force_avg_s = pair_ms / 1e3 / max(force_launches, 1)
    achieved = ops_per_launch / force_avg_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TOPS, "unit": "TOP/s",
                "frac": achieved / ALU_PEAK_TOPS, "traffic": kernel_traffic(),
                "kernel": "k_force", "avg_launch_ms": force_avg_s * 1e3,
                "peak_source": "152 SMs x 128 lanes x 2.07 GHz (unit counts and max clock)"}
    if clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (152 * 128 * clocks["sm_mhz"] * 1e6 / 1e12)
    # measured issue rates of the same lanes (FP32 FMA chains, integer xor+add
    # chains), beside the nominal peak from unit counts and clock
    ffma = dpd.dpd_alu_peak(0, 20)["lane_ops_per_s"] / 1e12
    iop = dpd.dpd_alu_peak(1, 20)["lane_ops_per_s"] / 1e12
    roofline["measured_issue"] = {"ffma": ffma, "int_xor_add": iop, "unit": "TOP/s",
                                  "frac_of_measured_ffma": achieved / ffma,
                                  "what": "dpd_alu_peak: 8 independent chains per thread, 8 blocks of 256 "
                                          "threads per SM, 20 timed launches"}
    # the whole step against the same peak: the pair work plus the integrator's
    # lane-ops per particle, over the measured time per step (rebuilds included)
    step_ops = n * (pairs_per_particle * OPS_PER_PAIR + OPS_INTEGRATE)
    step_achieved = step_ops / (max_ms / 1e3 / args.steps) / 1e12
    roofline["whole_step"] = {"achieved": step_achieved, "frac": step_achieved / ALU_PEAK_TOPS,
                              "lane_ops_per_particle_step": step_ops / n, "unit": "TOP/s"}

    # end to end through the public API with host buffers (pinned)
    e2e_steps = max(1, args.e2e_steps if args.e2e_steps > 0 else args.steps)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        out = t.numpy()
        out[...] = a
        return t, out

    _hx, x_host = pinned(np.ascontiguousarray(st["x"]))
    _hv, v_host = pinned(np.ascontiguousarray(st["v"]))
    _ho, xo = pinned(np.zeros_like(x_host))
    _hw, vo = pinned(np.zeros_like(v_host))
    obsbuf = dpd.ObsBuffer(e2e_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_state(x_host, v_host)
    for k in range(e2e_steps):
        sim.step_async(1)
        sim.observables_async(obsbuf, k)
    sim.sync()
    sim.state(xo, vo)
    torch.cuda.synchronize()
    e2e_s = slowest(pg, time.perf_counter() - t0, "cuda")
    # every step's statistics reached the host
    got = [obsbuf.get(k) for k in range(e2e_steps)]
    if [g["step"] for g in got] != list(range(1, e2e_steps + 1)) or not all(
            np.isfinite(g["temperature"]) and np.isfinite(g["pressure"]) for g in got):
        raise RuntimeError("end-to-end leg: missing or non-finite per-step observables")
    # the same with a host wait per step (dpd_step(1), then dpd_observables)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_state(x_host, v_host)
    for _ in range(e2e_steps):
        sim.step(1)
        sim.observables()
    sim.state(xo, vo)
    torch.cuda.synchronize()
    e2e_sync_s = slowest(pg, time.perf_counter() - t0, "cuda")
    state_bytes = n * 6 * 8
    obs_bytes = ctypes.sizeof(dpd.dpd_obs)
    e2e = {"value": job_rate(ws, n * e2e_steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(state_bytes / e2e_steps),
           "d2h_bytes_per_step": int(state_bytes / e2e_steps + obs_bytes),
           "steps": e2e_steps,
           "what": "dpd_set_state from pinned host arrays, then per step dpd_step_async(1) + "
                   "dpd_observables_async into pinned host records (every step's statistics copied to the host), "
                   "dpd_sync, then dpd_get_state to pinned host arrays",
           "host_wait_per_step": {"value": job_rate(ws, n * e2e_steps, e2e_sync_s), "unit": UNIT,
                                  "what": "the same with dpd_step(1) + dpd_observables (a host wait each step)"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": bench_config(args.workload, n, ws),
        "phases_ms": {"integrate": integ_ms, "rebuild": rebuild_ms, "force": force_ms, "pair_kernel": pair_ms,
                      "rebuilds": rebuilds},
        "skin_tuning_ms_per_step": skin_table,
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample_steps = 1
        rate1, secs1 = oracle_rate(xo, vo, cfg, sample_steps, cfg["box"])
        rate, cores, secs = oracle_all_cores(args.workload, cfg["box"], sample_steps)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "FP64 oracle (single-threaded C, unmodified) in %d processes, one per host "
                                          "core, each taking %d step of its own copy of the full %d-particle box "
                                          "(%.1f s)" % (cores, sample_steps, n, secs),
                                "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                                                "sample": "%d step of the full box on one core (%.1f s)" % (
                                                    sample_steps, secs1)}}
    sim.close()
    if rank == 0 and ws == 1 and not args.no_serving:
        line["batched"] = run_serving(args)
        if args.small_boxes > 0:
            line["batched"]["small_boxes"] = run_small_boxes(args)
    if rank == 0 and ws == 1 and args.ablations:
        line["list_builder_ablation"] = run_list_ablation()
        line["reorder_ablation"] = run_reorder_ablation()
        line["list_layout_ablation"] = run_layout_ablation()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
