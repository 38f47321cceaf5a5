"""FP64 CPU oracle for the DPD pair-interaction path (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The CUDA
library never imports, links or executes anything here, and this package
imports nothing from it.

The arithmetic lives in ``dpd_oracle.c`` (plain C, FP64, each routine citing
the passage of Tang & Karniadakis, arXiv:1311.0402, that it follows); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Everything here is argument marshalling, except the closed-form
start-up profile of the double Poiseuille flow (Eq. 10), written out in numpy.

Parity status: every routine is pinned by the ``-m "not gpu"`` tests
(published TEA vector, Gaussian moments, hand-computed pair forces, brute
force neighbour sets, momentum conservation, ideal-gas temperature, energy
conservation, harmonic-oscillator period, equation of state).  The exact
random-number values are "parity unpinned" against the paper, which prints
none; they follow the readings listed in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# gcc flags: no contraction, no fast-math (the FP32 predicate rounds each op).
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, a second or two)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of ``oc_params`` in dpd_oracle.c."""

    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("n_species", ctypes.c_int32),
        ("cut_fp32", ctypes.c_int32),
        ("a", ctypes.POINTER(ctypes.c_double)),
        ("gamma", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("rc", ctypes.c_double),
        ("s", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("body_mode", ctypes.c_int32),
        ("brute", ctypes.c_int32),
        ("body", ctypes.c_double * 3),
        ("nbonds", ctypes.c_int64),
        ("bonds", ctypes.POINTER(ctypes.c_uint32)),
        ("k_bond", ctypes.c_double),
        ("r0_bond", ctypes.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32, u64, i64, f64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
            P = ctypes.POINTER
            L.oc_tea.argtypes = [ctypes.c_int, P(u32), P(u32)]
            L.oc_tea.restype = None
            L.oc_key.argtypes = [u64, P(u32)]
            L.oc_key.restype = None
            L.oc_bitrev32.argtypes = [u32]
            L.oc_bitrev32.restype = u32
            L.oc_signature.argtypes = [u64, u32, u64]
            L.oc_signature.restype = u32
            L.oc_pair_hash.argtypes = [u64, u64, u32, u32, P(u32)]
            L.oc_pair_hash.restype = None
            L.oc_gauss.argtypes = [u32, u32]
            L.oc_gauss.restype = f64
            L.oc_xi.argtypes = [u64, u64, u32, u32]
            L.oc_xi.restype = f64
            L.oc_pair_hash_batch.argtypes = [u64, u64, i64, P(u32), P(u32), P(u32)]
            L.oc_pair_hash_batch.restype = None
            L.oc_xi_batch.argtypes = [u64, u64, i64, P(u32), P(u32), P(f64)]
            L.oc_xi_batch.restype = None
            L.oc_fp32_d2.argtypes = [P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float)]
            L.oc_fp32_d2.restype = ctypes.c_float
            L.oc_pairs_fp32_brute.argtypes = [i64, P(ctypes.c_float), P(ctypes.c_float), ctypes.c_float, P(u32), i64]
            L.oc_pairs_fp32_brute.restype = i64
            L.oc_neighbors_of.argtypes = [i64, P(ctypes.c_float), P(ctypes.c_float), ctypes.c_float, i64, P(u32), i64]
            L.oc_neighbors_of.restype = i64
            L.oc_forces.argtypes = [P(Params), i64, P(f64), P(f64), P(ctypes.c_int32), P(u32), u64, P(f64), P(f64)]
            L.oc_forces.restype = ctypes.c_int
            L.oc_run.argtypes = [P(Params), i64, P(f64), P(f64), P(f64), P(ctypes.c_int32), P(u32), P(u64), i64,
                                 P(f64), ctypes.c_int32, i64, P(f64), P(f64)]
            L.oc_run.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---------------------------------------------------------------- RNG pieces
def tea(rounds: int, key, v0: int, v1: int):
    """TEA rounds of Algorithm 4 under an explicit 4-word key."""
    k = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in key])
    v = (ctypes.c_uint32 * 2)(v0 & 0xFFFFFFFF, v1 & 0xFFFFFFFF)
    lib().oc_tea(rounds, k, v)
    return int(v[0]), int(v[1])


def key(seed: int):
    k = (ctypes.c_uint32 * 4)()
    lib().oc_key(seed, k)
    return [int(x) for x in k]


def bitrev32(x: int) -> int:
    return int(lib().oc_bitrev32(x & 0xFFFFFFFF))


def signature(seed: int, tag: int, step: int) -> int:
    return int(lib().oc_signature(seed, tag, step))


def pair_hash(seed: int, step: int, tag_i: int, tag_j: int):
    out = (ctypes.c_uint32 * 2)()
    lib().oc_pair_hash(seed, step, tag_i, tag_j, out)
    return int(out[0]), int(out[1])


def gauss(a: int, b: int) -> float:
    return float(lib().oc_gauss(a, b))


def xi(seed: int, step: int, tag_i: int, tag_j: int) -> float:
    return float(lib().oc_xi(seed, step, tag_i, tag_j))


def pair_hash_batch(seed: int, step: int, ti, tj) -> np.ndarray:
    """(m, 2) uint32 pair-hash words of Sec. 3.5 for the tag pairs (ti[k], tj[k])."""
    ti = np.ascontiguousarray(ti, np.uint32)
    tj = np.ascontiguousarray(tj, np.uint32)
    out = np.zeros((ti.shape[0], 2), np.uint32)
    lib().oc_pair_hash_batch(seed, step, ti.shape[0], _ptr(ti, ctypes.c_uint32), _ptr(tj, ctypes.c_uint32),
                             _ptr(out, ctypes.c_uint32))
    return out


def xi_batch(seed: int, step: int, ti, tj) -> np.ndarray:
    ti = np.ascontiguousarray(ti, np.uint32)
    tj = np.ascontiguousarray(tj, np.uint32)
    out = np.zeros(ti.shape[0], np.float64)
    lib().oc_xi_batch(seed, step, ti.shape[0], _ptr(ti, ctypes.c_uint32), _ptr(tj, ctypes.c_uint32),
                      _ptr(out, ctypes.c_double))
    return out


# ------------------------------------------------------------ neighbour sets
def fp32_d2(xi_, xj_, box) -> float:
    a = np.asarray(xi_, np.float32)
    b = np.asarray(xj_, np.float32)
    bx = np.asarray(box, np.float32)
    return float(lib().oc_fp32_d2(_ptr(a, ctypes.c_float), _ptr(b, ctypes.c_float), _ptr(bx, ctypes.c_float)))


def pairs_fp32(x, box, r) -> np.ndarray:
    """All index pairs (i < j) within r under the FP32 predicate, brute force.

    Returns an (m, 2) uint32 array in lexicographic order."""
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
    bx = np.asarray(box, np.float32)
    n = x.shape[0]
    L = lib()
    cnt = L.oc_pairs_fp32_brute(n, _ptr(x, ctypes.c_float), _ptr(bx, ctypes.c_float), np.float32(r), None, 0)
    out = np.zeros((max(cnt, 1), 2), np.uint32)
    L.oc_pairs_fp32_brute(n, _ptr(x, ctypes.c_float), _ptr(bx, ctypes.c_float), np.float32(r),
                          _ptr(out, ctypes.c_uint32), cnt)
    return out[:cnt]


def neighbors_of(x, box, r, i: int) -> np.ndarray:
    """Indices j != i within r of particle i (FP32 predicate), ascending."""
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
    bx = np.asarray(box, np.float32)
    n = x.shape[0]
    L = lib()
    cap = 4096
    out = np.zeros(cap, np.uint32)
    cnt = L.oc_neighbors_of(n, _ptr(x, ctypes.c_float), _ptr(bx, ctypes.c_float), np.float32(r), i,
                            _ptr(out, ctypes.c_uint32), cap)
    if cnt > cap:
        out = np.zeros(cnt, np.uint32)
        L.oc_neighbors_of(n, _ptr(x, ctypes.c_float), _ptr(bx, ctypes.c_float), np.float32(r), i,
                          _ptr(out, ctypes.c_uint32), cnt)
    return out[:cnt].copy()


# ------------------------------------------------------------------- system
class System:
    """An FP64 DPD system advanced by the oracle.

    Arrays are in the caller's particle order; ``tag`` (default 0..n-1) keys
    the random numbers, ``species`` indexes the symmetric a_ij matrix, and
    ``bonds`` holds (index, index) pairs into these arrays."""

    def __init__(self, box, a, gamma, kT, rc, s, dt, lam=0.5, seed=42, body_mode=0, body=(0.0, 0.0, 0.0),
                 bonds=None, k_bond=0.0, r0_bond=0.0, cut_fp32=True, brute=False):
        self.a = np.ascontiguousarray(np.atleast_2d(np.asarray(a, np.float64)))
        ns = self.a.shape[0]
        if self.a.shape != (ns, ns):
            raise ValueError("a_ij must be square")
        self.bonds = None if bonds is None else np.ascontiguousarray(np.asarray(bonds, np.uint32).reshape(-1, 2))
        p = Params()
        p.box[:] = [float(b) for b in box]
        p.n_species = ns
        p.cut_fp32 = 1 if cut_fp32 else 0
        p.a = _ptr(self.a, ctypes.c_double)
        p.gamma, p.kT, p.rc, p.s, p.dt, p.lam = gamma, kT, rc, s, dt, lam
        p.seed = seed
        p.body_mode = body_mode
        p.brute = 1 if brute else 0
        p.body[:] = [float(b) for b in body]
        p.nbonds = 0 if self.bonds is None else self.bonds.shape[0]
        p.bonds = _ptr(self.bonds, ctypes.c_uint32)
        p.k_bond, p.r0_bond = k_bond, r0_bond
        self.p = p
        self.box = np.asarray(box, np.float64)

    def forces(self, x, v, species=None, tag=None, step=0):
        """(f (n,3) float64, virial) at the given state and RNG step."""
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
        n = x.shape[0]
        sp = None if species is None else np.ascontiguousarray(species, np.int32)
        tg = None if tag is None else np.ascontiguousarray(tag, np.uint32)
        f = np.zeros((n, 3), np.float64)
        vir = ctypes.c_double(0.0)
        rc = lib().oc_forces(ctypes.byref(self.p), n, _ptr(x, ctypes.c_double), _ptr(v, ctypes.c_double),
                             _ptr(sp, ctypes.c_int32), _ptr(tg, ctypes.c_uint32), step, _ptr(f, ctypes.c_double),
                             ctypes.byref(vir))
        if rc:
            raise RuntimeError("oc_forces failed: %d" % rc)
        return f, vir.value

    def run(self, x, v, nsteps, species=None, tag=None, step=0, f=None, prof_nbins=0, prof_from=1):
        """Advance nsteps steps.  Returns a dict with the new x, v, f, step,
        per-step observables (sum v^2, virial, momentum) and the optional
        binned v_x profile sums / counts along y."""
        x = np.array(x, np.float64).reshape(-1, 3)
        v = np.array(v, np.float64).reshape(-1, 3)
        n = x.shape[0]
        sp = None if species is None else np.ascontiguousarray(species, np.int32)
        tg = None if tag is None else np.ascontiguousarray(tag, np.uint32)
        if f is None:
            f, _ = self.forces(x, v, species, tag, step)
        f = np.array(f, np.float64).reshape(-1, 3)
        st = ctypes.c_uint64(step)
        obs = np.zeros((max(nsteps, 1), 5), np.float64)
        ps = np.zeros(max(prof_nbins, 1), np.float64)
        pc = np.zeros(max(prof_nbins, 1), np.float64)
        rc = lib().oc_run(ctypes.byref(self.p), n, _ptr(x, ctypes.c_double), _ptr(v, ctypes.c_double),
                          _ptr(f, ctypes.c_double), _ptr(sp, ctypes.c_int32), _ptr(tg, ctypes.c_uint32),
                          ctypes.byref(st), nsteps, _ptr(obs, ctypes.c_double), prof_nbins, prof_from,
                          _ptr(ps, ctypes.c_double) if prof_nbins else None,
                          _ptr(pc, ctypes.c_double) if prof_nbins else None)
        if rc:
            raise RuntimeError("oc_run failed: %d" % rc)
        return dict(x=x, v=v, f=f, step=st.value, obs=obs[:nsteps], prof_sum=ps[:prof_nbins],
                    prof_cnt=pc[:prof_nbins])

    @staticmethod
    def temperature(sum_v2, n):
        """T = sum m v^2 / (3N - 3) (momentum-conserving DOF count)."""
        return sum_v2 / (3.0 * n - 3.0)

    def pressure(self, sum_v2, virial):
        """p = (sum m v^2 + sum_{i<j} r_ij . F_ij^{C+bond}) / (3 V)."""
        V = float(np.prod(self.box))
        return (sum_v2 + virial) / (3.0 * V)


def double_poiseuille_startup(y, t, F, d, nu, terms=400):
    """Eq. 10: the velocity of a fluid at rest at t = 0 driven by a body force
    F per unit mass between planes a distance d apart (z from the midplane,
    u = 0 at z = +-d/2):
        u(z, t) = F d^2 / (8 nu) (1 - (2z/d)^2)
                  - sum_n 4 (-1)^n F d^2 / (nu pi^3 (2n+1)^3) cos((2n+1) pi z / d)
                    exp(-(2n+1)^2 pi^2 nu t / d^2),
    with nu the kinematic viscosity, the series cut after `terms` terms.  In
    the periodic double flow the force is +F on y in [0, d) and -F on
    [d, 2d): each half is this profile, the second with the opposite sign;
    y is measured along the box's 2d length."""
    y = np.asarray(y, np.float64)
    out = np.zeros_like(y)
    for half, sgn in ((0, 1.0), (1, -1.0)):
        sel = (y >= half * d) & (y < (half + 1) * d)
        z = y[sel] - (half + 0.5) * d
        u = F * d * d / (8.0 * nu) * (1.0 - (2.0 * z / d) ** 2)
        for k in range(terms):
            m = 2 * k + 1
            u -= (4.0 * (-1) ** k * F * d * d / (nu * np.pi ** 3 * m ** 3) * np.cos(m * np.pi * z / d)
                  * np.exp(-m * m * np.pi ** 2 * nu * t / (d * d)))
        out[sel] = sgn * u
    return out
