"""The allocation-free force entry point (dpd_forces_static).

Some callers cannot allocate device memory: an application whose own pool
already owns all GPU memory, a plug-in that runs inside another framework's
memory budget, or code in a context where cudaMalloc is not allowed.  They
hand the library device buffers they already own, and the library works in
one fixed static scratch array instead of allocating.  These tests call that
entry point through the C ABI on buffers the test owns and check it:

* against the allocating path (dpd_forces) on two calls in a row, the second
  reusing the scratch the first left behind;
* against the FP64 oracle directly, with two species in an uneven layout,
  tags left to the library (NULL) and the weight exponents s = 1/2 and 1/4;
* that repeated calls leave the device's free memory unchanged and give the
  same bits;
* that an out-of-range species gives NaN forces for that particle and its
  partners instead of a read outside the parameter table.

The file is collected last, so a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
import paper_1311_0402_gb300 as dpd
import workloads
from gpu_util import force_error, need_gpu

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4  # relative to the RMS force, max over particles/components


def _device_state(x32, v32, species=None):
    import torch
    n = x32.shape[0]
    pos = torch.zeros((n, 4), dtype=torch.float32)
    pos[:, :3] = torch.from_numpy(x32.astype(np.float32))
    if species is not None:
        # species as the int bits of the fourth float
        pos[:, 3] = torch.from_numpy(np.asarray(species, np.int32).view(np.float32))
    vel = torch.zeros((n, 4), dtype=torch.float32)
    vel[:, :3] = torch.from_numpy(v32.astype(np.float32))
    dev = torch.device("cuda", 0)
    return pos.to(dev), vel.to(dev)


def _call(prm, n, pos, vel, tag, step, out):
    import torch
    stream = torch.cuda.current_stream(out.device)
    out.fill_(float("nan"))
    dpd.dpd_forces_static(prm, n, pos.data_ptr(), vel.data_ptr(), None if tag is None else tag.data_ptr(), step,
                          out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return out[:, :3].double().cpu().numpy()


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
    pos, vel = _device_state(x32, v32)
    tag = torch.arange(n, dtype=torch.int32, device=pos.device)  # same bits as uint32 tags 0..n-1
    out = torch.empty((n, 4), dtype=torch.float32, device=pos.device)
    prm = dpd.dpd_static_params_from(bx, c["a"], c["gamma"], c["kT"], c["rc"], c["s"], c["dt"], seed=42,
                                     body_mode=c.get("body_mode", 0), body=c.get("body", (0, 0, 0)))
    for call in range(2):
        f = _call(prm, n, pos, vel, tag, 9, out)
        assert np.isfinite(f).all(), call
        err, rms = force_error(f, f_ref)
        assert err < FORCE_TOL, (call, err, rms)


@pytest.mark.parametrize("s", [0.5, 0.25])
def test_static_forces_two_species_against_oracle(s):
    """Two species with an asymmetric a_ij layout in space (the second species
    fills one slab of the box), tags left NULL (tag = index), and a general
    weight exponent; compared with the FP64 oracle on the same FP32 state."""
    need_gpu()
    import torch

    box = (11.0, 9.0, 7.0)
    n = workloads.n_particles(box, 3.0)
    x, v = workloads.uniform_fluid(box, n, 1.0, 2024)
    species = np.where(x[:, 0] < 3.5, 1, 0).astype(np.int32)
    a = [[25.0, 60.0], [60.0, 18.0]]
    gamma, kT, rc, dt, seed, step = 4.5, 1.0, 1.0, 0.01, 77, 31
    x32 = x.astype(np.float32).astype(np.float64)
    v32 = v.astype(np.float32).astype(np.float64)
    ref = oracle.System(box, a, gamma, kT, rc, s, dt, seed=seed, cut_fp32=True)
    f_ref, _ = ref.forces(x32, v32, species=species, step=step)

    pos, vel = _device_state(x32, v32, species)
    out = torch.empty((n, 4), dtype=torch.float32, device=pos.device)
    prm = dpd.dpd_static_params_from(box, a, gamma, kT, rc, s, dt, seed=seed)
    f1 = _call(prm, n, pos, vel, None, step, out)
    free0 = torch.cuda.mem_get_info()[0]
    f2 = _call(prm, n, pos, vel, None, step, out)
    free1 = torch.cuda.mem_get_info()[0]
    err, rms = force_error(f1, f_ref)
    assert err < FORCE_TOL, (err, rms)
    # fixed summation order: the second call gives the same bits
    assert np.array_equal(f1, f2)
    # and the call allocated nothing on the device
    assert free0 == free1, (free0, free1)


def test_static_forces_bad_species_give_nan_not_a_stray_read():
    need_gpu()
    import torch

    box = (8.0, 8.0, 8.0)
    n = workloads.n_particles(box, 3.0)
    x, v = workloads.uniform_fluid(box, n, 1.0, 99)
    species = np.zeros(n, np.int32)
    bad = 17
    species[bad] = 1000  # far outside the 2 x 2 table
    pos, vel = _device_state(x, v, species)
    out = torch.empty((n, 4), dtype=torch.float32, device=pos.device)
    prm = dpd.dpd_static_params_from(box, [[25.0, 30.0], [30.0, 25.0]], 4.5, 1.0, 1.0, 1.0, 0.01)
    f = _call(prm, n, pos, vel, None, 0, out)
    x32 = x.astype(np.float32)
    d = x32 - x32[bad]
    d -= np.float32(8.0) * np.round(d / np.float32(8.0))
    near = (d.astype(np.float64) ** 2).sum(1) < 1.0 - 1e-4
    far = (d.astype(np.float64) ** 2).sum(1) > 1.0 + 1e-4
    assert np.isnan(f[bad]).all()
    assert np.isnan(f[near]).all()
    assert np.isfinite(f[far]).all()


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
