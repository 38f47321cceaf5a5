"""The allocation-free force entry point (dpd_forces_static).

Some callers cannot allocate device memory (an application that owns all GPU
memory through its own pool, a plug-in inside another framework's memory
budget); they hand the library device buffers they already own, and the
library uses a fixed static scratch array instead of cudaMalloc.  This test
calls that entry point through the C ABI on buffers the test owns and checks
it against the allocating path (dpd_forces) within the force tolerance of
the parity tests, on two calls in a row (the second reuses the scratch the
first left behind).  It lives in its own file, collected last."""
import numpy as np
import pytest

import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import force_error, need_gpu

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4  # relative to the RMS force, max over particles/components


@pytest.mark.parametrize("name,box", [("fluid_small", None), ("poiseuille", (12.0, 10.0, 6.0))])
def test_static_forces_match_allocating_path_twice(name, box):
    need_gpu()
    import torch

    st = workloads.make(name, box=box)
    c = st["cfg"]
    bx = c["box"]
    sim = dpd.Sim(bx, c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], seed=42,
                  body_mode=c.get("body_mode", 0), body=c.get("body", (0, 0, 0)))
    sim.set_state(st["x"], st["v"], step=9)
    x32, v32, _ = sim.state()
    f_ref = sim.forces()
    sim.close()

    n = x32.shape[0]
    dev = torch.device("cuda", 0)
    pos = torch.zeros((n, 4), dtype=torch.float32)
    pos[:, :3] = torch.from_numpy(x32.astype(np.float32))  # species 0 = int bits of 0.0f
    vel = torch.zeros((n, 4), dtype=torch.float32)
    vel[:, :3] = torch.from_numpy(v32.astype(np.float32))
    pos, vel = pos.to(dev), vel.to(dev)
    tag = torch.arange(n, dtype=torch.int32, device=dev)  # same bits as uint32 tags 0..n-1
    out = torch.full((n, 4), float("nan"), dtype=torch.float32, device=dev)
    prm = dpd.dpd_static_params_from(bx, c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], seed=42,
                                     body_mode=c.get("body_mode", 0), body=c.get("body", (0, 0, 0)))
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out.fill_(float("nan"))
        dpd.dpd_forces_static(prm, n, pos.data_ptr(), vel.data_ptr(), tag.data_ptr(), 9, out.data_ptr(),
                              stream.cuda_stream)
        stream.synchronize()
        f = out[:, :3].double().cpu().numpy()
        assert np.isfinite(f).all(), call
        err, rms = force_error(f, f_ref)
        assert err < FORCE_TOL, (call, err, rms)


def test_static_forces_reject_oversize():
    need_gpu()
    import torch

    mx = dpd.dpd_forces_static_max_particles()
    assert mx == 131072
    prm = dpd.dpd_static_params_from((10, 10, 10), [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01)
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(dpd.DPDError) as e:
        dpd.dpd_forces_static(prm, mx + 1, buf.data_ptr(), buf.data_ptr(), None, 0, buf.data_ptr())
    assert e.value.status == 1 and "static scratch" in str(e.value)
    big = dpd.dpd_static_params_from((300, 300, 300), [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01)
    with pytest.raises(dpd.DPDError) as e:
        dpd.dpd_forces_static(big, 1000, buf.data_ptr(), buf.data_ptr(), None, 0, buf.data_ptr())
    assert e.value.status == 1 and "cells" in str(e.value)
