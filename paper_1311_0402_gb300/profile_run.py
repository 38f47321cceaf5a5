"""Run a named workload for profiling: load the state, take a number of
steps launched kernel by kernel (no CUDA graphs, so a profiler sees every
launch), then one standalone force evaluation.

    python -m paper_1311_0402_gb300.profile_run --workload fluid_large --steps 20
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
    args = ap.parse_args()
    import paper_1311_0402_gb300 as dpd
    import workloads
    dpd.lib()
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
