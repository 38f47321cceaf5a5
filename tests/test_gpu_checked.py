"""The checked build (libdpd_checked.so, compiled with DPD_CHECKED): its
kernels test every index they read from device memory -- list entries, the
reorder permutation, bond partners -- before using it, and report a bad one
through the device error word.  Run in a child process (the binding loads one
library per process), it must give the production build's results on the
parity workloads with no error reported: the lists, permutations and bond
tables of these runs hold only valid indices."""
import os
import subprocess
import sys

import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, sys
sys.path.insert(0, %(root)r); sys.path.insert(0, %(tests)r)
import oracle, paper_1311_0402_gb300 as dpd, workloads
from gpu_util import force_error, make_pair, pair_set
assert dpd.LIB_PATH.endswith("libdpd_checked.so"), dpd.LIB_PATH
dpd.build()
worst = 0.0
for name, box, layout in (("fluid_small", None, 0), ("amphiphile", (12.0, 12.0, 12.0), 0),
                          ("fluid_small", None, 1), ("poiseuille", (12.0, 10.0, 6.0), 0)):
    st = workloads.make(name, box=box)
    cfg = dict(st["cfg"])
    bx = cfg["box"]
    g, o = make_pair(cfg, box=bx, bonds=st["bonds"], list_layout=layout)
    g.set_state(st["x"], st["v"], st["species"], step=2)
    if st["bonds"] is not None:
        g.set_bonds(st["bonds"], cfg["k_bond"], cfg["r0_bond"])
    g.step(30)
    x32, v32, step = g.state()
    fo, _ = o.forces(x32, v32, species=st["species"], step=step)
    err, _ = force_error(g.forces(), fo)
    worst = max(worst, err)
    g.build_neighbors()
    assert pair_set(g.neighbors()) == pair_set(oracle.pairs_fp32(x32, bx, cfg["rc"] + 0.3)), name
    g.close()
assert worst < 1e-4, worst
print("checked build ok: worst force error %%.2e of RMS" %% worst)
"""


def test_checked_build_runs_clean():
    need_gpu()
    env = dict(os.environ, DPD_LIB_VARIANT="checked")
    code = SCRIPT % {"root": ROOT, "tests": os.path.join(ROOT, "tests")}
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
