"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

import oracle
import paper_1311_0402_gb300 as dpd
import workloads


def need_gpu():
    import pytest
    try:
        import torch
        ok = torch.cuda.is_available()
    except Exception:
        ok = False
    if not ok:
        pytest.skip("no CUDA GPU")
    dpd.build()


def make_pair(cfg, skin=0.3, seed=42, box=None, **kw):
    """A GPU Sim and an oracle System with the same parameters."""
    box = cfg["box"] if box is None else box
    bonds = kw.pop("bonds", None)
    g = dpd.Sim(box, cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"], lam=cfg.get("lam", 0.5),
                skin=skin, seed=seed, body_mode=cfg.get("body_mode", 0), body=cfg.get("body", (0, 0, 0)), **kw)
    o = oracle.System(box, cfg["a"], cfg["gamma"], cfg["kT"], cfg["rc"], cfg["s"], cfg["dt"], lam=cfg.get("lam", 0.5),
                      seed=seed, body_mode=cfg.get("body_mode", 0), body=cfg.get("body", (0, 0, 0)),
                      bonds=bonds, k_bond=cfg.get("k_bond", 0.0), r0_bond=cfg.get("r0_bond", 0.0),
                      cut_fp32=True)
    return g, o


def force_error(f_gpu, f_ref):
    """max |f_gpu - f_ref| / RMS(|f_ref|)."""
    rms = np.sqrt((f_ref ** 2).sum(1).mean())
    return np.abs(f_gpu - f_ref).max() / rms, rms


def pair_set(p):
    p = np.asarray(p, np.uint64).reshape(-1, 2)
    return set((p[:, 0] << np.uint64(32) | p[:, 1]).tolist())
