"""Helpers for the GPU parity tests: move a workloads config to the device and
build a library context for it."""

from __future__ import annotations

import numpy as np


def to_device_system(cfg, io_dtype, k_max=None, pass_rho=None):
    import torch
    d = dict(n=cfg["n"], h=cfg["h"], n_electrons=cfg["n_electrons"], kT=cfg["kT"], g=cfg["g"],
             rho_floor=cfg["rho_floor"], k_max=k_max or cfg["V"].shape[0])
    d["psi"] = [torch.as_tensor(np.ascontiguousarray(p), dtype=io_dtype, device="cuda")
                for p in cfg["psi"]]
    d["eps"] = [torch.as_tensor(np.ascontiguousarray(e), dtype=torch.float64, device="cuda")
                for e in cfg["eps"]]
    if cfg.get("occ") is not None:
        d["occ"] = [torch.as_tensor(o, dtype=torch.float64, device="cuda") for o in cfg["occ"]]
    if pass_rho is not None:
        d["rho"] = [torch.as_tensor(r, dtype=io_dtype, device="cuda") for r in pass_rho]
    return d


def directions(cfg, io_dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(cfg["V"]), dtype=io_dtype, device="cuda")


def make_context(cfgs, prec, io_dtype, **kw):
    from paper_2211_07894_gb300 import Context
    systems = [to_device_system(c, io_dtype) for c in cfgs]
    return Context(systems, prec=prec, io_dtype=io_dtype, **kw), systems
