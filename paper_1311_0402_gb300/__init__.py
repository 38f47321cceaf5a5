"""Python binding of libdpd.so, the GB300 DPD pair-interaction engine.

Argument marshalling only: every step of the method runs in the CUDA kernels
behind the C ABI declared in ``include/dpd.h``.  The functions here carry the
same names as the C entry points; ``Sim`` wraps a handle for convenience.
There is no CPU fallback: importing works without a GPU, but every call
that needs the library raises if ``libdpd.so`` is missing or no GPU is
present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DPD_LIB_VARIANT=checked loads the checked build (device index checks, see
# buildlib); the default is the production library
LIB_PATH = os.path.join(HERE, "libdpd_checked.so" if os.environ.get("DPD_LIB_VARIANT") == "checked" else "libdpd.so")

DPD_OK = 0
STATUS = {0: "DPD_OK", 1: "DPD_ERR_ARG", 2: "DPD_ERR_OOM", 3: "DPD_ERR_CUDA", 4: "DPD_ERR_NBR_OVERFLOW",
          5: "DPD_ERR_NONFINITE", 6: "DPD_ERR_TIMEOUT", 7: "DPD_ERR_STATE"}

# every exported symbol declared in include/dpd.h
EXPORTS = ("dpd_default_options", "dpd_create", "dpd_set_state", "dpd_set_bonds", "dpd_build_neighbors",
           "dpd_get_neighbors", "dpd_forces", "dpd_get_force", "dpd_step", "dpd_observables", "dpd_profile",
           "dpd_get_state", "dpd_info", "dpd_pair_rng", "dpd_last_error", "dpd_destroy", "dpd_step_profiled",
           "dpd_forces_static", "dpd_forces_static_max_particles", "dpd_forces_static_last_error", "dpd_set_force",
           "dpd_step_async", "dpd_sync", "dpd_query", "dpd_tune_skin", "dpd_wait_selftest",
           "dpd_observables_async", "dpd_alu_peak",
           # include/dpd_server.h
           "dpd_server_default_options", "dpd_server_create", "dpd_server_submit", "dpd_server_wait",
           "dpd_server_now", "dpd_server_counts", "dpd_server_last_error", "dpd_server_destroy",
           # include/dpd_ensemble.h
           "dpd_ensemble_default_options", "dpd_ensemble_create", "dpd_ensemble_fits", "dpd_ensemble_add",
           "dpd_ensemble_remove", "dpd_ensemble_step", "dpd_ensemble_sync", "dpd_ensemble_get_state",
           "dpd_ensemble_get_forces", "dpd_ensemble_observables", "dpd_ensemble_info", "dpd_ensemble_tune",
           "dpd_ensemble_graph_stats",
           "dpd_ensemble_config", "dpd_ensemble_destroy", "dpd_ensemble_last_error")


class DPDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class dpd_options(ctypes.Structure):
    _fields_ = [
        ("skin", ctypes.c_double),
        ("rebuild_every", ctypes.c_int32),
        ("body_force_mode", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("lam", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("nbr_capacity", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("deterministic", ctypes.c_int32),
        ("conditional_rebuild", ctypes.c_int32),
        ("list_builder", ctypes.c_int32),
        ("no_reorder", ctypes.c_int32),
        ("list_layout", ctypes.c_int32),
        ("wait_timeout_s", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


class dpd_obs(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_uint64),
        ("n", ctypes.c_int64),
        ("kinetic", ctypes.c_double),
        ("temperature", ctypes.c_double),
        ("virial", ctypes.c_double),
        ("pressure", ctypes.c_double),
        ("momentum", ctypes.c_double * 3),
    ]


class dpd_server_options(ctypes.Structure):
    _fields_ = [
        ("max_active", ctypes.c_int32),
        ("workers", ctypes.c_int32),
        ("chunk_steps", ctypes.c_int32),
        ("mem_budget_bytes", ctypes.c_double),
        ("box_options", dpd_options),
        ("ensemble", ctypes.c_int32),
        ("ensemble_slots", ctypes.c_int32),
    ]


class dpd_request(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("n_species", ctypes.c_int32),
        ("a_ij", ctypes.POINTER(ctypes.c_double)),
        ("gamma", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("s", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("n", ctypes.c_int64),
        ("x", ctypes.POINTER(ctypes.c_double)),
        ("v", ctypes.POINTER(ctypes.c_double)),
        ("species", ctypes.POINTER(ctypes.c_int32)),
        ("steps", ctypes.c_uint64),
        ("skin", ctypes.c_double),
    ]


class dpd_result(ctypes.Structure):
    _fields_ = [
        ("ticket", ctypes.c_uint64),
        ("status", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("steps", ctypes.c_uint64),
        ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
        ("obs", dpd_obs),
        ("engine", ctypes.c_int32),
    ]


class dpd_step_times(ctypes.Structure):
    _fields_ = [
        ("total_ms", ctypes.c_double),
        ("integrate_ms", ctypes.c_double),
        ("rebuild_ms", ctypes.c_double),
        ("force_ms", ctypes.c_double),
        ("pair_ms", ctypes.c_double),
        ("steps", ctypes.c_int64),
        ("force_launches", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("rebuilds", ctypes.c_int64),
    ]


class dpd_static_params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("n_species", ctypes.c_int32),
        ("body_force_mode", ctypes.c_int32),
        ("a_ij", ctypes.c_double * 64),
        ("gamma", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("s", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("body_force", ctypes.c_double * 3),
    ]


class dpd_ensemble_options(ctypes.Structure):
    _fields_ = [
        ("threads", ctypes.c_int32),
        ("cluster", ctypes.c_int32),
        ("wait_timeout_s", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("newton3", ctypes.c_int32),
    ]


class dpd_box_params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("n_species", ctypes.c_int32),
        ("a_ij", ctypes.POINTER(ctypes.c_double)),
        ("gamma", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("s", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("body_force_mode", ctypes.c_int32),
        ("body_force", ctypes.c_double * 3),
    ]


_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose, checked=os.path.basename(LIB_PATH) == "libdpd_checked.so")


def lib():
    """Load libdpd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built (run paper_1311_0402_gb300.build())" % os.path.basename(LIB_PATH))
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        i32, i64, u32, u64, f64, vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_double, ctypes.c_void_p)
        L.dpd_default_options.argtypes = [P(dpd_options)]
        L.dpd_default_options.restype = None
        L.dpd_create.argtypes = [P(vp), P(f64), i32, P(f64), f64, f64, f64, f64, f64, P(dpd_options)]
        L.dpd_set_state.argtypes = [vp, i64, P(f64), P(f64), P(i32), P(u32), u64]
        L.dpd_set_bonds.argtypes = [vp, i64, P(u32), f64, f64]
        L.dpd_build_neighbors.argtypes = [vp]
        L.dpd_get_neighbors.argtypes = [vp, i64, P(u32), P(i64)]
        L.dpd_forces.argtypes = [vp, P(f64)]
        L.dpd_get_force.argtypes = [vp, P(f64)]
        L.dpd_set_force.argtypes = [vp, P(f64)]
        L.dpd_step.argtypes = [vp, i64]
        L.dpd_observables.argtypes = [vp, P(dpd_obs)]
        L.dpd_observables_async.argtypes = [vp, vp]
        L.dpd_alu_peak.argtypes = [i32, i32, P(f64), P(f64)]
        L.dpd_step_profiled.argtypes = [vp, i64, P(dpd_step_times)]
        L.dpd_profile.argtypes = [vp, i32, i32, i32, P(f64), P(f64)]
        L.dpd_get_state.argtypes = [vp, P(f64), P(f64), P(u64)]
        L.dpd_info.argtypes = [vp, P(i64), P(i64), P(i32)]
        L.dpd_pair_rng.argtypes = [u64, u64, i64, P(u32), P(u32), P(u32), P(ctypes.c_float)]
        L.dpd_last_error.argtypes = [vp]
        L.dpd_last_error.restype = ctypes.c_char_p
        L.dpd_forces_static.argtypes = [P(dpd_static_params), i64, vp, vp, vp, u64, vp, vp]
        L.dpd_forces_static_max_particles.argtypes = []
        L.dpd_forces_static_max_particles.restype = i64
        L.dpd_forces_static_last_error.argtypes = []
        L.dpd_forces_static_last_error.restype = ctypes.c_char_p
        L.dpd_destroy.argtypes = [vp]
        L.dpd_destroy.restype = None
        L.dpd_tune_skin.argtypes = [P(f64), i32, P(f64), f64, f64, f64, f64, f64, P(dpd_options), i64, P(f64),
                                    P(f64), P(i32), P(f64), i32, i32, P(f64), P(f64)]
        L.dpd_step_async.argtypes = [vp, i64]
        L.dpd_wait_selftest.argtypes = [vp, u32]
        L.dpd_sync.argtypes = [vp]
        L.dpd_query.argtypes = [vp, P(i32)]
        L.dpd_server_default_options.argtypes = [P(dpd_server_options)]
        L.dpd_server_default_options.restype = None
        L.dpd_server_create.argtypes = [P(dpd_server_options), P(vp)]
        L.dpd_server_submit.argtypes = [vp, P(dpd_request), P(u64)]
        L.dpd_server_wait.argtypes = [vp, u64, f64, P(dpd_result), P(f64), P(f64)]
        L.dpd_server_now.argtypes = [vp]
        L.dpd_server_now.restype = f64
        L.dpd_server_counts.argtypes = [vp, P(i64), P(i64), P(i64), P(f64)]
        L.dpd_server_last_error.argtypes = [vp]
        L.dpd_server_last_error.restype = ctypes.c_char_p
        L.dpd_server_destroy.argtypes = [vp]
        L.dpd_server_destroy.restype = None
        L.dpd_ensemble_default_options.argtypes = [P(dpd_ensemble_options)]
        L.dpd_ensemble_default_options.restype = None
        L.dpd_ensemble_create.argtypes = [P(vp), P(dpd_ensemble_options)]
        L.dpd_ensemble_fits.argtypes = [P(dpd_box_params), i64]
        L.dpd_ensemble_add.argtypes = [vp, P(dpd_box_params), i64, P(f64), P(f64), P(i32), u64, P(i32)]
        L.dpd_ensemble_remove.argtypes = [vp, i32]
        L.dpd_ensemble_step.argtypes = [vp, P(i32), P(i32), i32]
        L.dpd_ensemble_sync.argtypes = [vp]
        L.dpd_ensemble_get_state.argtypes = [vp, i32, P(f64), P(f64), P(u64)]
        L.dpd_ensemble_get_forces.argtypes = [vp, i32, P(f64)]
        L.dpd_ensemble_observables.argtypes = [vp, i32, P(dpd_obs)]
        L.dpd_ensemble_info.argtypes = [vp, P(i32), P(i64)]
        L.dpd_ensemble_graph_stats.argtypes = [vp, P(i64), P(i64)]
        L.dpd_ensemble_tune.argtypes = [vp, i32, P(f64)]
        L.dpd_ensemble_config.argtypes = [vp, P(i32), P(i32)]
        L.dpd_ensemble_destroy.argtypes = [vp]
        L.dpd_ensemble_destroy.restype = None
        L.dpd_ensemble_last_error.argtypes = [vp]
        L.dpd_ensemble_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _check(st, h=None):
    if st != DPD_OK:
        msg = lib().dpd_last_error(h)
        raise DPDError(st, msg.decode() if msg else "")


# ----------------------------------------------------------- C-named wrappers
def dpd_default_options() -> dpd_options:
    o = dpd_options()
    lib().dpd_default_options(ctypes.byref(o))
    return o


def dpd_create(box, a_ij, gamma, kT, rc, s, dt, opt: dpd_options | None = None):
    a = np.ascontiguousarray(np.atleast_2d(np.asarray(a_ij, np.float64)))
    b = np.ascontiguousarray(np.asarray(box, np.float64))
    h = ctypes.c_void_p()
    st = lib().dpd_create(ctypes.byref(h), _p(b, ctypes.c_double), a.shape[0], _p(a, ctypes.c_double), gamma, kT, rc,
                          s, dt, ctypes.byref(opt) if opt is not None else None)
    _check(st)
    return h


def dpd_set_state(h, x, v, species=None, tag=None, step=0):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
    sp = None if species is None else np.ascontiguousarray(species, np.int32)
    tg = None if tag is None else np.ascontiguousarray(tag, np.uint32)
    _check(lib().dpd_set_state(h, x.shape[0], _p(x, ctypes.c_double), _p(v, ctypes.c_double),
                               _p(sp, ctypes.c_int32), _p(tg, ctypes.c_uint32), step), h)


def dpd_set_bonds(h, pairs, k, r0):
    pr = np.ascontiguousarray(np.asarray(pairs, np.uint32).reshape(-1, 2))
    _check(lib().dpd_set_bonds(h, pr.shape[0], _p(pr, ctypes.c_uint32), k, r0), h)


def dpd_build_neighbors(h):
    _check(lib().dpd_build_neighbors(h), h)


def dpd_get_neighbors(h) -> np.ndarray:
    cnt = ctypes.c_int64(0)
    _check(lib().dpd_get_neighbors(h, 0, None, ctypes.byref(cnt)), h)
    out = np.zeros((max(cnt.value, 1), 2), np.uint32)
    _check(lib().dpd_get_neighbors(h, cnt.value, _p(out, ctypes.c_uint32), ctypes.byref(cnt)), h)
    return out[:cnt.value]


def dpd_info(h):
    n, r, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().dpd_info(h, ctypes.byref(n), ctypes.byref(r), ctypes.byref(c)), h)
    return dict(n=n.value, rebuilds=r.value, nbr_capacity=c.value)


def _nvec(h):
    return dpd_info(h)["n"]


def dpd_forces(h) -> np.ndarray:
    f = np.zeros((_nvec(h), 3), np.float64)
    _check(lib().dpd_forces(h, _p(f, ctypes.c_double)), h)
    return f


def dpd_get_force(h) -> np.ndarray:
    f = np.zeros((_nvec(h), 3), np.float64)
    _check(lib().dpd_get_force(h, _p(f, ctypes.c_double)), h)
    return f


def dpd_set_force(h, f):
    f = np.ascontiguousarray(f, np.float64).reshape(-1, 3)
    _check(lib().dpd_set_force(h, _p(f, ctypes.c_double)), h)


def dpd_step(h, nsteps: int):
    _check(lib().dpd_step(h, int(nsteps)), h)


def dpd_tune_skin(box, a_ij, gamma, kT, rc, s, dt, x, v, candidates=(0.2, 0.3, 0.4, 0.5), steps=200,
                  species=None, lam=0.5, deterministic=0):
    """The fastest neighbour-list skin for this system, by measurement (see
    dpd.h); returns (best_skin, {skin: ms_per_step})."""
    a = np.ascontiguousarray(np.atleast_2d(np.asarray(a_ij, np.float64)))
    b = np.ascontiguousarray(np.asarray(box, np.float64))
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
    sp = None if species is None else np.ascontiguousarray(species, np.int32)
    c = np.ascontiguousarray(np.asarray(candidates, np.float64))
    ms = np.zeros(c.shape[0], np.float64)
    o = dpd_default_options()
    o.lam = lam
    o.deterministic = 1 if deterministic else 0
    best = ctypes.c_double()
    _check(lib().dpd_tune_skin(_p(b, ctypes.c_double), a.shape[0], _p(a, ctypes.c_double), gamma, kT, rc, s, dt,
                               ctypes.byref(o), x.shape[0], _p(x, ctypes.c_double), _p(v, ctypes.c_double),
                               _p(sp, ctypes.c_int32), _p(c, ctypes.c_double), c.shape[0], int(steps),
                               ctypes.byref(best), _p(ms, ctypes.c_double)))
    return best.value, {float(k): float(t) for k, t in zip(c, ms)}


def dpd_wait_selftest(h, polls: int = 1024) -> int:
    """Status of the device's bounded-wait self-test (DPD_ERR_TIMEOUT = 6
    when the wait gave up as it should)."""
    return int(lib().dpd_wait_selftest(h, int(polls)))


def dpd_step_async(h, nsteps: int):
    _check(lib().dpd_step_async(h, int(nsteps)), h)


def dpd_sync(h):
    _check(lib().dpd_sync(h), h)


def dpd_query(h) -> bool:
    idle = ctypes.c_int32(0)
    _check(lib().dpd_query(h, ctypes.byref(idle)), h)
    return bool(idle.value)


def dpd_step_profiled(h, nsteps: int) -> dict:
    t = dpd_step_times()
    _check(lib().dpd_step_profiled(h, int(nsteps), ctypes.byref(t)), h)
    return {k: getattr(t, k) for k, _ in dpd_step_times._fields_}


def dpd_observables(h) -> dict:
    o = dpd_obs()
    _check(lib().dpd_observables(h, ctypes.byref(o)), h)
    return dict(step=o.step, n=o.n, kinetic=o.kinetic, temperature=o.temperature, virial=o.virial,
                pressure=o.pressure, momentum=np.array(list(o.momentum)))


def _obs_dict(o) -> dict:
    return dict(step=o.step, n=o.n, kinetic=o.kinetic, temperature=o.temperature, virial=o.virial,
                pressure=o.pressure, momentum=np.array(list(o.momentum)))


def dpd_alu_peak(kind: int, reps: int = 20) -> dict:
    """Measured issue rate of FP32 FMA (kind 0) or integer xor+add (kind 1)
    chains, in lane-operations per second."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().dpd_alu_peak(int(kind), int(reps), ctypes.byref(r), ctypes.byref(ms)))
    return {"lane_ops_per_s": r.value, "ms_per_launch": ms.value}


def dpd_observables_async(h, address: int) -> None:
    """Queue the observables into the page-locked dpd_obs at `address`
    (valid after the next sync)."""
    _check(lib().dpd_observables_async(h, ctypes.c_void_p(address)), h)


class ObsBuffer:
    """k dpd_obs records in page-locked host memory (a pinned torch tensor),
    the destination of Sim.observables_async."""

    def __init__(self, k: int):
        import torch
        self.k = int(k)
        self._t = torch.zeros(self.k * ctypes.sizeof(dpd_obs), dtype=torch.uint8, pin_memory=True)

    def address(self, i: int) -> int:
        if not 0 <= i < self.k:
            raise IndexError(i)
        return self._t.data_ptr() + i * ctypes.sizeof(dpd_obs)

    def get(self, i: int) -> dict:
        return _obs_dict(dpd_obs.from_address(self.address(i)))


def dpd_profile(h, bin_axis: int, vel_axis: int, nbins: int, sums=None, counts=None):
    s = np.zeros(nbins, np.float64) if sums is None else sums
    c = np.zeros(nbins, np.float64) if counts is None else counts
    _check(lib().dpd_profile(h, bin_axis, vel_axis, nbins, _p(s, ctypes.c_double), _p(c, ctypes.c_double)), h)
    return s, c


def dpd_get_state(h, x=None, v=None):
    """Positions and velocities into x, v (n x 3 float64, C order; allocated
    when None -- pass pinned arrays to read back at full speed) and the step."""
    n = _nvec(h)
    x = np.zeros((n, 3), np.float64) if x is None else x
    v = np.zeros((n, 3), np.float64) if v is None else v
    for a in (x, v):
        if a.shape != (n, 3) or a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("state arrays must be C-contiguous float64 of shape (n, 3)")
    st = ctypes.c_uint64()
    _check(lib().dpd_get_state(h, _p(x, ctypes.c_double), _p(v, ctypes.c_double), ctypes.byref(st)), h)
    return x, v, st.value


def dpd_pair_rng(seed: int, step: int, tag_i, tag_j):
    ti = np.ascontiguousarray(tag_i, np.uint32)
    tj = np.ascontiguousarray(tag_j, np.uint32)
    m = ti.shape[0]
    hh = np.zeros((max(m, 1), 2), np.uint32)
    xi = np.zeros(max(m, 1), np.float32)
    _check(lib().dpd_pair_rng(seed, step, m, _p(ti, ctypes.c_uint32), _p(tj, ctypes.c_uint32),
                              _p(hh, ctypes.c_uint32), _p(xi, ctypes.c_float)))
    return hh[:m], xi[:m]


def dpd_static_params_from(box, a_ij, gamma, kT, rc, s, dt, seed=42, body_mode=0, body=(0.0, 0.0, 0.0)):
    a = np.atleast_2d(np.asarray(a_ij, np.float64))
    p = dpd_static_params()
    p.box[:] = [float(b) for b in box]
    p.n_species = a.shape[0]
    p.body_force_mode = body_mode
    p.a_ij[:a.size] = [float(x) for x in a.reshape(-1)]
    p.gamma, p.kT, p.rc, p.s, p.dt = gamma, kT, rc, s, dt
    p.seed = seed
    p.body_force[:] = [float(b) for b in body]
    return p


def dpd_forces_static(params: dpd_static_params, n: int, pos_ptr: int, vel_ptr: int, tag_ptr, step: int,
                      force_ptr: int, stream_ptr=None):
    """Enqueue the allocation-free force on device pointers (see dpd.h)."""
    st = lib().dpd_forces_static(ctypes.byref(params), int(n), ctypes.c_void_p(pos_ptr), ctypes.c_void_p(vel_ptr),
                                 None if tag_ptr is None else ctypes.c_void_p(tag_ptr), int(step),
                                 ctypes.c_void_p(force_ptr), None if stream_ptr is None else ctypes.c_void_p(stream_ptr))
    if st != DPD_OK:
        m = lib().dpd_forces_static_last_error()
        raise DPDError(st, m.decode() if m else "")


def dpd_forces_static_max_particles() -> int:
    return int(lib().dpd_forces_static_max_particles())


def dpd_forces_static_last_error() -> str:
    m = lib().dpd_forces_static_last_error()
    return m.decode() if m else ""


def dpd_last_error(h=None) -> str:
    m = lib().dpd_last_error(h)
    return m.decode() if m else ""


def dpd_destroy(h):
    lib().dpd_destroy(h)


# -------------------------------------------------------------- convenience
class Sim:
    """A DPD system on the GPU (one handle of libdpd.so)."""

    def __init__(self, box, a_ij, gamma, kT, rc, s, dt, lam=0.5, skin=0.3, seed=42, body_mode=0,
                 body=(0.0, 0.0, 0.0), rebuild_every=0, nbr_capacity=0, graph_steps=8, stream=None,
                 deterministic=0, conditional_rebuild=1, list_builder=0, no_reorder=0, list_layout=0):
        o = dpd_default_options()
        o.skin = skin
        o.lam = lam
        o.seed = seed
        o.body_force_mode = body_mode
        o.body_force[:] = [float(b) for b in body]
        o.rebuild_every = rebuild_every
        o.nbr_capacity = nbr_capacity
        o.graph_steps = graph_steps
        o.deterministic = 1 if deterministic else 0
        o.conditional_rebuild = 1 if conditional_rebuild else 0
        o.list_builder = int(list_builder)
        o.no_reorder = 1 if no_reorder else 0
        o.list_layout = int(list_layout)
        o.stream = stream
        self.box = np.asarray(box, np.float64)
        self.h = dpd_create(box, a_ij, gamma, kT, rc, s, dt, o)

    def close(self):
        if self.h is not None:
            dpd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x, v, species=None, tag=None, step=0):
        dpd_set_state(self.h, x, v, species, tag, step)

    def set_bonds(self, pairs, k, r0):
        dpd_set_bonds(self.h, pairs, k, r0)

    def build_neighbors(self):
        dpd_build_neighbors(self.h)

    def neighbors(self):
        return dpd_get_neighbors(self.h)

    def forces(self):
        return dpd_forces(self.h)

    def force(self):
        return dpd_get_force(self.h)

    def set_force(self, f):
        dpd_set_force(self.h, f)

    def step(self, n):
        dpd_step(self.h, n)

    def step_async(self, n):
        dpd_step_async(self.h, n)

    def sync(self):
        dpd_sync(self.h)

    def query(self) -> bool:
        return dpd_query(self.h)

    def step_profiled(self, n):
        return dpd_step_profiled(self.h, n)

    def observables(self):
        return dpd_observables(self.h)

    def observables_async(self, buf: "ObsBuffer", i: int):
        """Queue the observables of the state the queued steps reach into
        buf's record i; read it with buf.get(i) after sync()."""
        dpd_observables_async(self.h, buf.address(i))

    def profile(self, bin_axis, vel_axis, nbins, sums=None, counts=None):
        return dpd_profile(self.h, bin_axis, vel_axis, nbins, sums, counts)

    def state(self, x=None, v=None):
        return dpd_get_state(self.h, x, v)

    def info(self):
        return dpd_info(self.h)


# ------------------------------------------------------------ serving loop
def _server_check(st, srv):
    if st != DPD_OK:
        m = lib().dpd_server_last_error(srv)
        raise DPDError(st, m.decode() if m else "")


class Server:
    """Continuous batching of independent boxes (include/dpd_server.h)."""

    def __init__(self, max_active=32, chunk_steps=100, mem_budget_bytes=0.0, skin=0.3, deterministic=0,
                 graph_steps=8, lam=0.5, conditional_rebuild=0, workers=4, ensemble=0, ensemble_slots=1024):
        o = dpd_server_options()
        lib().dpd_server_default_options(ctypes.byref(o))
        o.ensemble = int(ensemble)  # 0 off, 1 every box that fits, 2 only while the handle slots are full
        o.ensemble_slots = ensemble_slots
        o.max_active = max_active
        o.workers = workers
        o.chunk_steps = chunk_steps
        o.mem_budget_bytes = float(mem_budget_bytes)
        o.box_options.skin = skin
        o.box_options.deterministic = 1 if deterministic else 0
        o.box_options.graph_steps = graph_steps
        o.box_options.lam = lam
        o.box_options.conditional_rebuild = 1 if conditional_rebuild else 0
        self.s = ctypes.c_void_p()
        _server_check(lib().dpd_server_create(ctypes.byref(o), ctypes.byref(self.s)), None)
        self._n = {}

    def submit(self, box, a_ij, gamma, kT, rc, s, dt, x, v, steps, seed=42, species=None, skin=0.0) -> int:
        a = np.ascontiguousarray(np.atleast_2d(np.asarray(a_ij, np.float64)))
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
        sp = None if species is None else np.ascontiguousarray(species, np.int32)
        r = dpd_request()
        r.box[:] = [float(b) for b in box]
        r.n_species = a.shape[0]
        r.a_ij = _p(a, ctypes.c_double)
        r.gamma, r.kT, r.rc, r.s, r.dt = gamma, kT, rc, s, dt
        r.seed = seed
        r.n = x.shape[0]
        r.x = _p(x, ctypes.c_double)
        r.v = _p(v, ctypes.c_double)
        r.species = _p(sp, ctypes.c_int32) if sp is not None else None
        r.steps = int(steps)
        r.skin = float(skin)
        t = ctypes.c_uint64()
        _server_check(lib().dpd_server_submit(self.s, ctypes.byref(r), ctypes.byref(t)), self.s)
        self._n[t.value] = x.shape[0]
        return t.value

    def wait(self, ticket, timeout_s=600.0, state=True):
        n = self._n.get(ticket, 0)
        state = state and n > 0
        res = dpd_result()
        x = np.zeros((n, 3), np.float64) if state else None
        v = np.zeros((n, 3), np.float64) if state else None
        _server_check(lib().dpd_server_wait(self.s, ticket, timeout_s, ctypes.byref(res), _p(x, ctypes.c_double),
                                            _p(v, ctypes.c_double)), self.s)
        self._n.pop(ticket, None)
        o = res.obs
        out = dict(ticket=res.ticket, status=res.status, n=res.n, steps=res.steps, t_submit=res.t_submit,
                   t_admit=res.t_admit, t_done=res.t_done, engine=res.engine,
                   obs=dict(step=o.step, n=o.n, kinetic=o.kinetic, temperature=o.temperature, virial=o.virial,
                            pressure=o.pressure, momentum=np.array(list(o.momentum))))
        if state:
            out["x"], out["v"] = x, v
        return out

    def now(self) -> float:
        return float(lib().dpd_server_now(self.s))

    def counts(self):
        q, r, f, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _server_check(lib().dpd_server_counts(self.s, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f),
                                              ctypes.byref(m)), self.s)
        return dict(queued=q.value, running=r.value, finished=f.value, mem_bytes=m.value)

    def close(self):
        if self.s is not None and self.s.value:
            lib().dpd_server_destroy(self.s)
        self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ ensemble kernel
def _ens_check(st, e):
    if st != DPD_OK:
        m = lib().dpd_ensemble_last_error(e)
        raise DPDError(st, m.decode() if m else "")


def dpd_box_params_from(box, a_ij, gamma, kT, rc, s, dt, lam=0.5, seed=42, body_mode=0, body=(0.0, 0.0, 0.0)):
    """dpd_box_params and the a_ij array it points to (keep both alive)."""
    a = np.ascontiguousarray(np.atleast_2d(np.asarray(a_ij, np.float64)))
    p = dpd_box_params()
    p.box[:] = [float(b) for b in box]
    p.n_species = a.shape[0]
    p.a_ij = _p(a, ctypes.c_double)
    p.gamma, p.kT, p.rc, p.s, p.dt, p.lam = gamma, kT, rc, s, dt, lam
    p.seed = seed
    p.body_force_mode = body_mode
    p.body_force[:] = [float(b) for b in body]
    return p, a


def dpd_ensemble_fits(box, a_ij, gamma, kT, rc, s, dt, n, lam=0.5) -> bool:
    p, _a = dpd_box_params_from(box, a_ij, gamma, kT, rc, s, dt, lam)
    return bool(lib().dpd_ensemble_fits(ctypes.byref(p), int(n)))


class Ensemble:
    """Many small boxes advanced together by the ensemble kernel
    (include/dpd_ensemble.h): one thread-block cluster per box, the box
    resident in shared memory for a whole chunk of steps."""

    def __init__(self, threads=0, cluster=0, wait_timeout_s=600.0, newton3=0):
        o = dpd_ensemble_options()
        lib().dpd_ensemble_default_options(ctypes.byref(o))
        o.threads, o.cluster, o.wait_timeout_s, o.newton3 = threads, cluster, wait_timeout_s, newton3
        self.e = ctypes.c_void_p()
        _ens_check(lib().dpd_ensemble_create(ctypes.byref(self.e), ctypes.byref(o)), None)
        self._n = {}

    def add(self, box, a_ij, gamma, kT, rc, s, dt, x, v, species=None, step=0, lam=0.5, seed=42, body_mode=0,
            body=(0.0, 0.0, 0.0)) -> int:
        p, _a = dpd_box_params_from(box, a_ij, gamma, kT, rc, s, dt, lam, seed, body_mode, body)
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
        if v.shape != x.shape:
            raise ValueError("x and v must have the same shape")
        sp = None if species is None else np.ascontiguousarray(species, np.int32)
        i = ctypes.c_int32()
        _ens_check(lib().dpd_ensemble_add(self.e, ctypes.byref(p), x.shape[0], _p(x, ctypes.c_double),
                                          _p(v, ctypes.c_double), _p(sp, ctypes.c_int32), int(step), ctypes.byref(i)),
                   self.e)
        self._n[i.value] = x.shape[0]
        return i.value

    def remove(self, box_id):
        _ens_check(lib().dpd_ensemble_remove(self.e, int(box_id)), self.e)
        self._n.pop(box_id, None)

    def step(self, steps, ids=None):
        """Advance boxes ids (all when None) by steps (an int, or one per id);
        asynchronous, see sync()."""
        if ids is None:
            st = np.array([int(steps)], np.int32)
            _ens_check(lib().dpd_ensemble_step(self.e, None, _p(st, ctypes.c_int32), 0), self.e)
            return
        ids = np.ascontiguousarray(ids, np.int32).reshape(-1)
        st = np.ascontiguousarray(np.broadcast_to(np.asarray(steps, np.int32), ids.shape), np.int32)
        _ens_check(lib().dpd_ensemble_step(self.e, _p(ids, ctypes.c_int32), _p(st, ctypes.c_int32), ids.size),
                   self.e)

    def sync(self):
        _ens_check(lib().dpd_ensemble_sync(self.e), self.e)

    def _count(self, box_id):
        n = self._n.get(box_id)
        if n is None:
            raise DPDError(1, "unknown box id %r" % (box_id,))
        return n

    def state(self, box_id):
        n = self._count(box_id)
        x = np.zeros((n, 3), np.float64)
        v = np.zeros((n, 3), np.float64)
        step = ctypes.c_uint64()
        _ens_check(lib().dpd_ensemble_get_state(self.e, int(box_id), _p(x, ctypes.c_double), _p(v, ctypes.c_double),
                                                ctypes.byref(step)), self.e)
        return x, v, step.value

    def forces(self, box_id):
        f = np.zeros((self._count(box_id), 3), np.float64)
        _ens_check(lib().dpd_ensemble_get_forces(self.e, int(box_id), _p(f, ctypes.c_double)), self.e)
        return f

    def observables(self, box_id):
        o = dpd_obs()
        _ens_check(lib().dpd_ensemble_observables(self.e, int(box_id), ctypes.byref(o)), self.e)
        return dict(step=o.step, n=o.n, kinetic=o.kinetic, temperature=o.temperature, virial=o.virial,
                    pressure=o.pressure, momentum=np.array(list(o.momentum)))

    def info(self):
        nb, npart = ctypes.c_int32(), ctypes.c_int64()
        _ens_check(lib().dpd_ensemble_info(self.e, ctypes.byref(nb), ctypes.byref(npart)), self.e)
        return nb.value, npart.value

    def graph_stats(self):
        """(step calls that captured a new launch graph, calls that replayed one)."""
        c, r = ctypes.c_int64(), ctypes.c_int64()
        _ens_check(lib().dpd_ensemble_graph_stats(self.e, ctypes.byref(c), ctypes.byref(r)), self.e)
        return c.value, r.value

    def tune(self, steps=50):
        """Autotune threads per CTA and CTAs per box for each size class
        present; returns the last class's table {(threads, cluster): ms per step}."""
        t = np.zeros(12, np.float64)
        _ens_check(lib().dpd_ensemble_tune(self.e, int(steps), _p(t, ctypes.c_double)), self.e)
        return {(T, C): float(t[ti * 4 + ci]) for ti, T in enumerate((128, 256, 512))
                for ci, C in enumerate((1, 2, 4, 8))}

    def config(self):
        th = np.zeros(4, np.int32)
        cl = np.zeros(4, np.int32)
        _ens_check(lib().dpd_ensemble_config(self.e, _p(th, ctypes.c_int32), _p(cl, ctypes.c_int32)), self.e)
        return th.tolist(), cl.tolist()

    def close(self):
        if self.e is not None and self.e.value:
            lib().dpd_ensemble_destroy(self.e)
        self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
