"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/dpd.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1311_0402_gb300 as dpd
from paper_1311_0402_gb300 import buildlib as dbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dpd_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = dbuild.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    declared = _declared()
    assert {"dpd_create", "dpd_set_state", "dpd_build_neighbors", "dpd_forces", "dpd_step",
            "dpd_observables"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(dpd.EXPORTS) == declared


def test_checked_library_exports_the_same_symbols():
    path = dbuild.build(checked=True)
    assert os.path.basename(path) == "libdpd_checked.so"
    L = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_argument_errors_need_no_gpu():
    dbuild.build()
    # validation happens before any CUDA call
    with pytest.raises(dpd.DPDError) as e:
        dpd.dpd_create((2.0, 10, 10), [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01)
    assert e.value.status == 1
    with pytest.raises(dpd.DPDError) as e:
        dpd.dpd_create((10, 10, 10), [[25.0, 1.0], [2.0, 25.0]], 4.5, 1.0, 1.0, 1.0, 0.01)
    assert e.value.status == 1
    with pytest.raises(dpd.DPDError) as e:
        dpd.dpd_create((10, 10, 10), [[25.0]], -1.0, 1.0, 1.0, 1.0, 0.01)
    assert e.value.status == 1
    o = dpd.dpd_default_options()
    assert o.skin == 0.3 and o.seed == 42 and o.lam == 0.5 and o.graph_steps == 8


def test_ensemble_fails_loudly_without_a_gpu():
    dbuild.build()
    # option validation comes before any CUDA call
    with pytest.raises(dpd.DPDError) as e:
        dpd.Ensemble(threads=100)
    assert e.value.status == 1
    with pytest.raises(dpd.DPDError) as e:
        dpd.Ensemble(cluster=3)
    assert e.value.status == 1
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        # no CPU fallback: creating an ensemble needs the device
        with pytest.raises(dpd.DPDError) as e:
            dpd.Ensemble()
        assert e.value.status == 3
        assert not dpd.dpd_ensemble_fits((10.0,) * 3, [[25.0]], 4.5, 1.0, 1.0, 1.0, 0.01, 3000)
