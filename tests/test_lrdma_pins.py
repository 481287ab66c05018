"""Pins of the accumulated LRDM step's decisions (oracle.lrdma_step, §II.B.1,
Eqs. linearapprox, linearityIndicator, accum), CPU only, on a restricted
system, a spin pair (§II.D) and a Brillouin-zone-sampled system (§II.C
closing paragraphs).

The paper prints no worked example of the decisions, so they are pinned on a
residual map that is exactly linear: one fixed system (so the Jacobian J, and
with it every kept derivative t = J u, is the same at every step) and a next
residual that the test builds itself from the previous one.  For a step with
coefficients a (the w-least-squares fit T a = P R, P the w-orthogonal
projector onto span T, s = ||(I - P) R|| / ||R||) and damping alpha the
linear prediction is R_lin = R - alpha P R, and then, in closed form:

* a next residual c R_lin has beta = |1/c - 1| (Eq. linearityIndicator);
* the kept history's fit of R_lin has
  s_hist = s / sqrt(s^2 + (1 - alpha)^2 (1 - s^2)), and its coefficients are
  (1 - alpha) a, so a reused step is Delta' = (1 - alpha) Delta;
* alpha = 1 leaves R_lin = (I - P) R, which the history cannot fit at all
  (s_hist = 1).

Each clearing (CL on beta, CR on ||R||, CT after a non-converged
accumulation) is followed by a fresh build equal to the pinned LRDM step
(oracle.lrdm_krylov_step); an accumulation keeps the history, starts from the
normalised orthogonal complement of R to it, takes each next direction from
the previous derivative orthogonalised against all directions, stops at
r_max_iter or s_rel < s_tol, and flags CT when it stopped short.
"""

import numpy as np
import pytest

import oracle
import workloads
from helpers import oracle_system, rel_err


def _kpoint_system(cfg):
    mu = oracle.solve_mu_kpoints(cfg["eps"], cfg["k_weights"], cfg["n_electrons"], cfg["kT"], cfg["g"])
    ks = oracle.KpointSystem(n=cfg["n"], h=cfg["h"], psi=cfg["psi"], eps=cfg["eps"], k_weights=cfg["k_weights"],
                             rho=np.zeros(int(np.prod(cfg["n"]))), n_electrons=cfg["n_electrons"],
                             kT=cfg["kT"], g=cfg["g"])
    ks.rho = oracle.density_kpoints(ks, mu, cfg["rho_floor"])
    return ks


@pytest.fixture(scope="module", params=["real", "spin", "kpoint"])
def lin(request):
    """A fixed system (restricted, a spin pair with a shared mu, or sampled at
    4 k-points with complex subspaces), a residual R0 and the Gateaux map J
    of that system."""
    if request.param == "real":
        cfg = workloads.random_system(71, (8, 7, 6), 24, 26.0, 0.02, 3)
        sysm = oracle_system(cfg)
        R0 = workloads.smooth_field(cfg["n"], cfg["h"], 0.1, workloads.rng_for(71, 1))[None]
        return sysm, R0, lambda u: oracle.gateaux(sysm, u[None])["F"][0]
    if request.param == "spin":
        cfg = workloads.spin_pair_system(73, (8, 7, 6), 24, 20, 22.0, 0.02, 3)
        sysm = oracle_system(cfg)
        return sysm, cfg["R"], lambda u: oracle.gateaux(sysm, u[None])["F"][0]
    cfg = workloads.kpoint_system(72, (8, 7, 6), 24, 4, 26.0, 0.02, 3)
    sysm = _kpoint_system(cfg)
    R0 = workloads.smooth_field(cfg["n"], cfg["h"], 0.1, workloads.rng_for(72, 1))
    return sysm, R0, lambda u: oracle.gateaux_kpoints(sysm, u[None])["F"][0]


def _first(sysm, R0, alpha, s_tol=0.3, r_max=20):
    state = oracle.LrdmaState()
    out = oracle.lrdma_step(sysm, state, R0, s_tol=s_tol, r_max=r_max, alpha=alpha)
    assert out["event"] == "fresh"
    return state, out


def _span_residual(x, B, w):
    """||x - (w-orthogonal projection of x onto span B)||_w / ||x||_w."""
    Bm = np.stack([b.ravel() for b in B], axis=1)
    c, *_ = np.linalg.lstsq(np.sqrt(w) * Bm, np.sqrt(w) * x.ravel(), rcond=None)
    return rel_err(Bm @ c, x.ravel(), w)


def _krylov_equal(out, ref, R):
    assert out["rank"] == ref["rank"] and out["rank_new"] == ref["rank"]
    assert rel_err(out["delta"], ref["delta"]) < 1e-12
    assert abs(out["s_rel"] - ref["s_rel"][-1]) < 1e-12


@pytest.mark.parametrize("c", [2.0, 0.7, 1.05])
def test_beta_closed_form_and_CL(lin, c):
    sysm, R0, _ = lin
    state, _ = _first(sysm, R0, alpha=0.5)
    R1 = c * state.R_lin
    out = oracle.lrdma_step(sysm, state, R1, alpha=0.5, r_norm_clear=1e9)
    assert abs(out["beta"] - abs(1.0 / c - 1.0)) < 1e-13
    if abs(1.0 / c - 1.0) > 0.1:
        assert out["event"] == "CL"
        _krylov_equal(out, oracle.lrdm_krylov_step(sysm, R1, s_tol=0.3, r_max=20, alpha=0.5), R1)
    else:
        assert out["event"] in ("reuse", "accumulate")


@pytest.mark.parametrize("alpha", [0.5, 0.3])
def test_reuse_closed_form(lin, alpha):
    sysm, R0, _ = lin
    state, first = _first(sysm, R0, alpha=alpha, s_tol=0.02)
    s = first["s_rel"]
    r0 = first["rank"]
    s_hist = s / np.sqrt(s * s + (1 - alpha) ** 2 * (1 - s * s))
    assert s_hist < 0.3
    R1 = state.R_lin.copy()
    out = oracle.lrdma_step(sysm, state, R1, s_tol=0.3, alpha=alpha)
    assert out["event"] == "reuse" and out["rank"] == r0 and out["rank_new"] == 0
    assert out["beta"] < 1e-12
    assert abs(out["s_rel"] - s_hist) < 1e-10
    assert rel_err(out["delta"], (1 - alpha) * first["delta"]) < 1e-10
    assert rel_err(out["a"], (1 - alpha) * first["a"]) < 1e-10
    # a history whose fit of R_lin misses s_tol is not reused
    state2, _ = _first(sysm, R0, alpha=alpha, s_tol=0.02)
    out2 = oracle.lrdma_step(sysm, state2, state2.R_lin.copy(), s_tol=0.5 * s_hist, alpha=alpha,
                             r_norm_clear=0.0)
    assert out2["event"] == "CR"


def test_CR_rebuilds_like_lrdm(lin):
    sysm, R0, _ = lin
    state, _ = _first(sysm, R0, alpha=1.0)
    R1 = state.R_lin.copy()
    rn = float(np.sqrt(sysm.w * np.sum(R1 * R1)))
    out = oracle.lrdma_step(sysm, state, R1, alpha=0.5, r_norm_clear=0.5 * rn)
    assert out["beta"] < 1e-12 and out["event"] == "CR"
    _krylov_equal(out, oracle.lrdm_krylov_step(sysm, R1, s_tol=0.3, r_max=20, alpha=0.5), R1)


@pytest.mark.parametrize("r_max_iter", [1, 3, 5])
def test_accumulate_directions_and_CT(lin, r_max_iter):
    sysm, R0, J = lin
    w = sysm.w
    state, first = _first(sysm, R0, alpha=1.0, r_max=2, s_tol=1e-9)
    r0 = first["rank"]
    assert r0 == 2
    U_old = [u.copy() for u in state.U]
    # R_lin itself lies in span(U_old, t_last) after a Krylov build; a small
    # part outside it (beta stays below beta_tol) tells R's complement from t's
    R_lin = state.R_lin.copy()
    rz = workloads.rng_for(71, 2)
    ng = int(np.prod(sysm.n))
    z = np.stack([workloads.smooth_field(sysm.n, sysm.h, 1.0, rz) for _ in range(R_lin.size // ng)])
    z = z.reshape(R_lin.shape) / np.sqrt(w * np.sum(z * z))
    R1 = R_lin + 0.05 * np.sqrt(w * np.sum(R_lin * R_lin)) * z
    beta = abs(np.sqrt(np.sum(R_lin * R_lin) / np.sum(R1 * R1)) - 1.0)
    s_tol = 1e-9
    out = oracle.lrdma_step(sysm, state, R1, alpha=0.5, s_tol=s_tol, r_max_iter=r_max_iter, r_norm_clear=1e9)
    assert out["event"] == "accumulate" and abs(out["beta"] - beta) < 1e-13 and beta < 0.1
    assert _span_residual(R1, U_old + [state.T[r0 - 1]], w) > 1e-3
    m = out["rank_new"]
    assert m == r_max_iter and out["rank"] == r0 + m
    U = state.U
    assert all(np.array_equal(a, b) for a, b in zip(U[:r0], U_old))
    Um = np.stack(U).reshape(len(U), -1)
    assert np.max(np.abs(w * Um @ Um.T - np.eye(len(U)))) < 1e-12
    # u_1 is the normalised orthogonal complement of R to the history
    assert _span_residual(R1, U[:r0 + 1], w) < 1e-12
    comp = R1 - sum(w * float(np.sum(R1 * u)) * u for u in U_old)
    assert rel_err(U[r0], comp / np.sqrt(w * np.sum(comp * comp))) < 1e-12
    # each next one comes from the previous derivative, orthogonalised against all directions
    for j in range(1, m):
        t_prev = J(U[r0 + j - 1])
        assert rel_err(state.T[r0 + j - 1], t_prev) < 1e-14
        assert _span_residual(U[r0 + j], U[:r0 + j] + [t_prev], w) < 1e-10
    # the fit uses every kept derivative
    Tm = np.stack(state.T).reshape(len(U), -1)
    c, *_ = np.linalg.lstsq(np.sqrt(w) * Tm.T, np.sqrt(w) * R1.ravel(), rcond=None)
    assert rel_err(out["delta"], (Um.T @ c).reshape(R1.shape)) < 1e-8
    # s_rel still above s_tol: the next step clears (CT) and rebuilds like LRDM, whatever beta says
    assert state.clear_next
    R2 = state.R_lin.copy()
    nxt = oracle.lrdma_step(sysm, state, R2, alpha=0.5, s_tol=0.3, r_norm_clear=1e9)
    assert nxt["event"] == "CT"
    _krylov_equal(nxt, oracle.lrdm_krylov_step(sysm, R2, s_tol=0.3, r_max=20, alpha=0.5), R2)


def test_accumulate_stops_at_s_tol_without_CT(lin):
    sysm, R0, _ = lin
    state, _ = _first(sysm, R0, alpha=1.0, r_max=2, s_tol=1e-9)
    R1 = state.R_lin.copy()
    out = oracle.lrdma_step(sysm, state, R1, alpha=0.5, s_tol=0.3, r_max_iter=5, r_norm_clear=1e9)
    assert out["event"] == "accumulate"
    assert out["s_rel"] < 0.3 and 1 <= out["rank_new"] <= 5
    assert not state.clear_next
