"""Test helpers: turn a ``workloads`` config into an oracle system, and
relative-error measures.  Used by CPU pin tests and GPU parity tests."""

from __future__ import annotations

import numpy as np

import oracle


def oracle_system(cfg, occ_mode=False, poisson="spectral"):
    """oracle.System for a workloads config dict; rho = g sum f psi^2 + floor
    computed by the oracle itself (the config carries only the floor)."""
    g = cfg["g"]
    mu = oracle.solve_mu(cfg["eps"], cfg["n_electrons"], cfg["kT"], g)
    occ = [oracle.fermi(e, mu, cfg["kT"]) for e in cfg["eps"]]
    rho = [oracle.density(p, o, g, cfg["rho_floor"]) for p, o in zip(cfg["psi"], occ)]
    return oracle.System(n=cfg["n"], h=cfg["h"], psi=[np.asarray(p, dtype=np.float64) for p in cfg["psi"]],
                         eps=[np.asarray(e, dtype=np.float64) for e in cfg["eps"]], rho=rho,
                         n_electrons=cfg["n_electrons"], kT=cfg["kT"], g=g,
                         occ=occ if occ_mode else None, poisson=poisson)


def rel_err(a, b, w=1.0):
    """||a - b||_w / ||b||_w."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.sqrt(w * np.sum(b * b))
    return float(np.sqrt(w * np.sum((a - b) ** 2)) / (nb if nb > 0 else 1.0))


def per_direction_rel_err(a, b):
    """max over directions k of ||a_k - b_k|| / ||b_k|| (arrays (K, ...))."""
    return max(rel_err(a[k], b[k]) for k in range(a.shape[0]))
