"""Run a named workload for profiling: load the state, take a number of
steps launched kernel by kernel (no CUDA graphs, so a profiler sees every
launch), then one standalone force evaluation.

    python -m paper_1311_0402_gb300.profile_run --workload fluid_large --steps 20

With --ensemble N: N seeded boxes of side --ensemble-L in the ensemble kernel
(dpd_ensemble.h) at the given threads per CTA and CTAs per box, the
initial-force launch and then one launch of --steps steps.

    python -m paper_1311_0402_gb300.profile_run --ensemble 152 --ensemble-L 10 --steps 20
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="fluid_large")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--skin", type=float, default=None)
    ap.add_argument("--box", type=float, nargs=3, default=None)
    ap.add_argument("--ensemble", type=int, default=0)
    ap.add_argument("--ensemble-L", type=int, default=10)
    ap.add_argument("--threads", type=int, default=512)
    ap.add_argument("--cluster", type=int, default=2)
    args = ap.parse_args()
    import paper_1311_0402_gb300 as dpd
    import workloads
    dpd.lib()
    if args.ensemble > 0:
        boxes = workloads.serving_stream(args.ensemble, seed=77, L_range=(args.ensemble_L, args.ensemble_L),
                                         steps_range=(args.steps, args.steps), with_state=True)
        ens = dpd.Ensemble(threads=args.threads, cluster=args.cluster)
        ids = [ens.add(b["box"], b["a"], b["gamma"], b["kT"], b["rc"], b["s"], b["dt"], b["x"], b["v"],
                       seed=b["seed"]) for b in boxes]
        ens.step(0)
        ens.sync()
        t0 = time.perf_counter()
        ens.step(args.steps)
        ens.sync()
        el = time.perf_counter() - t0
        n = sum(b["n"] for b in boxes)
        print("ensemble boxes=%d L=%d particles=%d steps=%d wall=%.4fs T=%.4f" % (
            args.ensemble, args.ensemble_L, n, args.steps, el, ens.observables(ids[0])["temperature"]))
        ens.close()
        return
    if args.skin is None:
        args.skin = workloads.BENCH_SKIN
    st = workloads.make(args.workload, box=args.box)
    c = st["cfg"]
    box = c["box"]
    sim = dpd.Sim(box, c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], lam=c["lam"], skin=args.skin,
                  body_mode=c.get("body_mode", 0), body=c.get("body", (0, 0, 0)), graph_steps=0)
    sim.set_state(st["x"], st["v"], st["species"])
    if st["bonds"] is not None:
        sim.set_bonds(st["bonds"], c["k_bond"], c["r0_bond"])
    t0 = time.perf_counter()
    t = sim.step_profiled(args.steps) if args.steps > 0 else None
    el = time.perf_counter() - t0
    sim.forces()
    info = sim.info()
    sim.close()
    print("workload=%s n=%d steps=%d wall=%.3fs rebuilds=%d cap=%d times=%s" % (
        args.workload, st["n"], args.steps, el, info["rebuilds"], info["nbr_capacity"], t))


if __name__ == "__main__":
    main()
