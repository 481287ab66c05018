"""Pins of the oracle's Brillouin-zone-sampled response (oracle.gateaux_kpoints,
§II.C closing paragraphs, Eq. tracelessCondition), CPU only.

* One k-point with a real subspace and weight 1 reduces to the pinned real
  response (oracle.gateaux).
* Brute force: central differences (Richardson) of the BZ-averaged projected
  density rho_P(lam) = g sum_kappa w_kappa diag(Psi_kappa f(D_kappa +
  lam X_kappa, mu(lam)) Psi_kappa^H), with complex Hermitian eigen-
  decompositions and mu(lam) re-solved over all k-points together.  A dropped
  conjugate, a transposed Gamma or a per-point (instead of BZ-summed) mu'
  each fail it.
* Invariants: int drho = 0 (electron count over the BZ), <dV_a, drho_b> =
  <dV_b, drho_a> (self-adjoint chi_0), and invariance under a phase per state
  (Psi_kappa -> Psi_kappa diag(e^{i phi})) and under complex conjugation of
  every Psi (the time-reversed points -kappa).
* Adjoint (oracle.backward_kpoints): dot-product test <f_bar, J v> =
  <J^T f_bar, v> with J from gateaux_kpoints, and one real point with weight
  1 against the pinned real adjoint (oracle.backward).
* The adaptive-rank LRDM step on a BZ-sampled system (oracle.lrdm_krylov_step
  with the k-point derivative) against the Krylov space of the k-point
  Gateaux map and an lstsq solve over it.
"""

import numpy as np
import pytest
from scipy.linalg import eigh

import oracle
import workloads
from helpers import rel_err


def _system(cfg, psi=None):
    psi = cfg["psi"] if psi is None else psi
    mu = oracle.solve_mu_kpoints(cfg["eps"], cfg["k_weights"], cfg["n_electrons"], cfg["kT"], cfg["g"])
    ks = oracle.KpointSystem(n=cfg["n"], h=cfg["h"], psi=psi, eps=cfg["eps"], k_weights=cfg["k_weights"],
                             rho=np.zeros(int(np.prod(cfg["n"]))), n_electrons=cfg["n_electrons"],
                             kT=cfg["kT"], g=cfg["g"])
    ks.rho = oracle.density_kpoints(ks, mu, cfg["rho_floor"])
    return ks


@pytest.fixture(scope="module")
def kp():
    return workloads.kpoint_system(60, (8, 7, 6), 24, 4, 26.0, 0.02, 3)


def test_subspace_is_orthonormal(kp):
    w = float(np.prod(kp["h"]))
    for psi in kp["psi"]:
        assert np.abs(w * psi.conj().T @ psi - np.eye(psi.shape[1])).max() < 1e-12
    assert abs(sum(kp["k_weights"]) - 1.0) < 1e-15


def test_single_real_kpoint_equals_real_response():
    cfg = workloads.random_system(61, (8, 7, 6), 24, 26.0, 0.02, 3)
    ks = oracle.KpointSystem(n=cfg["n"], h=cfg["h"], psi=[cfg["psi"][0].astype(np.complex128)],
                             eps=cfg["eps"], k_weights=[1.0], rho=np.zeros(336),
                             n_electrons=cfg["n_electrons"], kT=cfg["kT"], g=2.0)
    mu = oracle.solve_mu(cfg["eps"], cfg["n_electrons"], cfg["kT"], 2.0)
    ks.rho = oracle.density_kpoints(ks, mu, cfg["rho_floor"])
    real = oracle.System(n=cfg["n"], h=cfg["h"], psi=cfg["psi"], eps=cfg["eps"], rho=[ks.rho],
                         n_electrons=cfg["n_electrons"], kT=cfg["kT"], g=2.0)
    a = oracle.gateaux_kpoints(ks, cfg["V"][:, 0])
    b = oracle.gateaux(real, cfg["V"])
    assert abs(a["mu"] - b["mu"]) < 1e-14
    assert rel_err(a["F"], b["F"][:, 0]) < 1e-13
    assert np.abs(a["dmu"] - b["dmu"]).max() < 1e-13


def _projected_density(ks, X, lam):
    """g sum_kappa w_kappa diag(Psi f(D + lam X, mu(lam)) Psi^H) by Hermitian
    eigendecompositions, mu(lam) from the BZ-averaged electron count."""
    evals, evecs = [], []
    for e, Xk in zip(ks.eps, X):
        d, U = eigh(np.diag(e) + lam * Xk)
        evals.append(d)
        evecs.append(U)
    mu = oracle.solve_mu_kpoints(evals, ks.k_weights, ks.n_electrons, ks.kT, ks.g)
    rho = np.zeros(ks.psi[0].shape[0])
    for psi, d, U, wk in zip(ks.psi, evals, evecs, ks.k_weights):
        P = (U * oracle.fermi(d, mu, ks.kT)) @ U.conj().T
        rho += ks.g * wk * np.einsum("ri,ij,rj->r", psi, P, psi.conj()).real
    return rho


def test_brute_force_projected_density(kp):
    ks = _system(kp)
    ref = oracle.gateaux_kpoints(ks, kp["V"])
    fx = oracle.lda_fx(ks.rho)
    for k in range(kp["V"].shape[0]):
        dV = oracle.perturbation_potential([kp["V"][k]], [fx], ks.n, ks.h)[0]
        X = []
        for psi in ks.psi:
            Xk = psi.conj().T @ ((ks.w * dV)[:, None] * psi)
            X.append(0.5 * (Xk + Xk.conj().T))
        eta = 1e-4 / max(np.abs(x).max() for x in X)

        def D(e):
            return (_projected_density(ks, X, e) - _projected_density(ks, X, -e)) / (2 * e)

        fd = (4 * D(eta / 2) - D(eta)) / 3
        assert rel_err(fd, ref["drho"][k]) < 1e-7


def test_invariants(kp):
    ks = _system(kp)
    ref = oracle.gateaux_kpoints(ks, kp["V"])
    fx = oracle.lda_fx(ks.rho)
    dV = [oracle.perturbation_potential([v], [fx], ks.n, ks.h)[0] for v in kp["V"]]
    for k in range(len(dV)):
        assert abs(ks.w * ref["drho"][k].sum()) < 1e-12 * ks.w * np.abs(ref["drho"][k]).sum()
    K = len(dV)
    for a in range(K):
        for b in range(a + 1, K):
            ab = float(np.dot(dV[a], ref["drho"][b]))
            ba = float(np.dot(dV[b], ref["drho"][a]))
            assert abs(ab - ba) < 1e-10 * max(abs(ab), abs(ba))
    for k in range(K):
        assert float(np.dot(dV[k], ref["drho"][k])) <= 0.0


def test_phase_and_conjugation_invariance(kp):
    ks = _system(kp)
    ref = oracle.gateaux_kpoints(ks, kp["V"])
    rng = workloads.rng_for(60, 5)
    phased = [p * np.exp(1j * rng.uniform(0, 2 * np.pi, p.shape[1]))[None, :] for p in kp["psi"]]
    a = oracle.gateaux_kpoints(_system(kp, phased), kp["V"])
    assert rel_err(a["F"], ref["F"]) < 1e-12
    b = oracle.gateaux_kpoints(_system(kp, [p.conj() for p in kp["psi"]]), kp["V"])
    assert rel_err(b["F"], ref["F"]) < 1e-12
    assert np.abs(b["dmu"] - ref["dmu"]).max() < 1e-12


def test_krylov_step_on_kpoints_matches_krylov_least_squares(kp):
    """The adaptive-rank LRDM step on a BZ-sampled system against an
    independent construction: span{R, JR, ..., J^(r-1) R} with J the pinned
    k-point Gateaux map, and min ||J Delta - R||_w over it by lstsq."""
    ks = _system(kp)
    w = ks.w
    R = workloads.smooth_field(ks.n, ks.h, 0.1, workloads.rng_for(60, 7))
    out = oracle.lrdm_krylov_step(ks, R, s_tol=1e-6, r_max=4)
    r = out["rank"]
    assert r == 4
    U = out["U"].reshape(r, -1)
    assert np.max(np.abs(w * U @ U.T - np.eye(r))) < 1e-12

    def J(v):
        return oracle.gateaux_kpoints(ks, v[None])["F"][0]

    Kr = [np.asarray(R, dtype=np.float64)]
    for _ in range(r):
        Kr.append(J(Kr[-1]))
    B = np.stack(Kr[:r], axis=1)
    JB = np.stack(Kr[1:], axis=1)
    b, *_ = np.linalg.lstsq(np.sqrt(w) * JB, np.sqrt(w) * R, rcond=None)
    assert rel_err(out["delta"], B @ b) < 1e-8


def test_adjoint_dot_product(kp):
    ks = _system(kp)
    rng = workloads.rng_for(60, 9)
    V = kp["V"]
    Fbar = rng.standard_normal(V.shape)
    F = oracle.gateaux_kpoints(ks, V)["F"]
    vbar = oracle.backward_kpoints(ks, Fbar)
    lhs = float(np.sum(Fbar * F))
    rhs = float(np.sum(vbar * V))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-30)


def test_adjoint_single_real_point_equals_real_adjoint():
    cfg = workloads.random_system(62, (8, 7, 6), 24, 26.0, 0.02, 3)
    mu = oracle.solve_mu(cfg["eps"], cfg["n_electrons"], cfg["kT"], 2.0)
    ks = oracle.KpointSystem(n=cfg["n"], h=cfg["h"], psi=[cfg["psi"][0].astype(np.complex128)],
                             eps=cfg["eps"], k_weights=[1.0], rho=np.zeros(336),
                             n_electrons=cfg["n_electrons"], kT=cfg["kT"], g=2.0)
    ks.rho = oracle.density_kpoints(ks, mu, cfg["rho_floor"])
    real = oracle.System(n=cfg["n"], h=cfg["h"], psi=cfg["psi"], eps=cfg["eps"], rho=[ks.rho],
                         n_electrons=cfg["n_electrons"], kT=cfg["kT"], g=2.0)
    Fbar = workloads.rng_for(62, 1).standard_normal(cfg["V"].shape)
    a = oracle.backward_kpoints(ks, Fbar[:, 0])
    b = oracle.backward(real, Fbar, V=cfg["V"])["vbar"]
    assert rel_err(a, b[:, 0]) < 1e-12
