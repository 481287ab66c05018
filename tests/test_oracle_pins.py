"""Pins of the FP64 oracle against things other than itself: brute-force
finite differences of the Kohn-Sham map, closed forms, a hand-worked
two-level system, high-precision arithmetic and invariants.

The paper prints no worked numerical example, so every pin comes from the
mathematics of §II (Eqs. kseqcont, jacobian, densityResponse,
densityMatResponseApprox, subspaceDensityMatResponse, plowrank,
relativeError).
"""

import os

import numpy as np
import pytest
from scipy.linalg import eigh

import oracle
import workloads
from helpers import oracle_system, rel_err
from ks_model import scf_map

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------
# P1: full-space brute force.  F[rho] by dense diagonalisation of
# H = -1/2 Lap + V_ext + V_H[rho] + V_x[rho] (Eq. kseqcont); central finite
# differences of F along v, Richardson-extrapolated, against the oracle's
# Gateaux derivative with Psi = all eigenvectors (so the subspace is exact).
# ---------------------------------------------------------------------------

_scf_map = scf_map


def _fd_gateaux(n, h, vext, lap, rho, n_e, kT, g, v, eta=2e-3):
    # eta = 2e-3: below it eigensolver rounding (~1e-15 |H| / eta) dominates,
    # above it the O(eta^4) Richardson remainder does; both stay below 3e-10.
    def D(et):
        plus, _, _ = _scf_map(n, h, vext, lap, [r + et * vv for r, vv in zip(rho, v)], n_e, kT, g)
        minus, _, _ = _scf_map(n, h, vext, lap, [r - et * vv for r, vv in zip(rho, v)], n_e, kT, g)
        return [(p - m) / (2 * et) for p, m in zip(plus, minus)]
    d1, d2 = D(eta), D(eta / 2)
    return [(4 * b - a) / 3 - vv for a, b, vv in zip(d1, d2, v)]


@pytest.fixture(scope="module")
def tiny_model():
    n, h = (6, 6, 6), (0.5, 0.5, 0.5)
    rng = workloads.rng_for(90, 0)
    vext = workloads.gaussian_wells(n, h, 3, rng)
    lap = workloads.fd_laplacian_dense(n, h)
    w = float(np.prod(h))
    e0, p0 = workloads.lowest_eigenpairs(workloads.toy_hamiltonian(n, h, vext), 8, w)
    rho0 = 2.0 * (p0[:, :4] ** 2).sum(axis=1) + 0.02
    return n, h, vext, lap, rho0


@pytest.mark.parametrize("kT", [0.05, 0.2])
def test_full_space_fd_restricted(tiny_model, kT):
    n, h, vext, lap, rho0 = tiny_model
    n_e, g = 6.0, 2.0
    _, eps, psi = _scf_map(n, h, vext, lap, [rho0], n_e, kT, g)
    V = workloads.smooth_directions(n, h, 3, 1, workloads.rng_for(90, 1))
    sysm = oracle.System(n=n, h=h, psi=psi, eps=eps, rho=[rho0], n_electrons=n_e, kT=kT, g=g)
    res = oracle.gateaux(sysm, V)
    for k in range(V.shape[0]):
        fd = _fd_gateaux(n, h, vext, lap, [rho0], n_e, kT, g, list(V[k]))
        assert rel_err(res["F"][k, 0], fd[0]) < 1e-9
        assert rel_err(res["drho"][k, 0], fd[0] + V[k, 0]) < 1e-9


def test_full_space_fd_spin(tiny_model):
    n, h, vext, lap, rho0 = tiny_model
    n_e, g, kT = 5.0, 1.0, 0.05
    rho = [0.6 * rho0, 0.4 * rho0 + 0.005]
    _, eps, psi = _scf_map(n, h, vext, lap, rho, n_e, kT, g)
    V = workloads.smooth_directions(n, h, 2, 2, workloads.rng_for(90, 2))
    sysm = oracle.System(n=n, h=h, psi=psi, eps=eps, rho=rho, n_electrons=n_e, kT=kT, g=g)
    res = oracle.gateaux(sysm, V)
    for k in range(V.shape[0]):
        fd = _fd_gateaux(n, h, vext, lap, rho, n_e, kT, g, list(V[k]))
        num = np.concatenate([res["F"][k, 0], res["F"][k, 1]])
        ref = np.concatenate(fd)
        assert rel_err(num, ref) < 1e-9


# ---------------------------------------------------------------------------
# P2: projected brute force (N_s < N_g): d/dlambda of g diag(Psi f(D + lambda X,
# mu(lambda)) Psi^T) by dense eigendecomposition of the N_s x N_s matrix,
# mu re-solved (Eq. densityMatResponseApprox), including near-degenerate pairs.
# ---------------------------------------------------------------------------

def _projected_density(psi, eps, X, lam, n_e, kT, g):
    th, Q = eigh(np.diag(eps) + lam * X)
    mu = oracle.solve_mu([th], n_e, kT, g)
    Gam = (Q * oracle.fermi(th, mu, kT)) @ Q.T
    return g * np.einsum("ri,ij,rj->r", psi, Gam, psi)


@pytest.mark.parametrize("gap", [None, 1e-9])
def test_projected_fd(gap):
    n, h = (8, 8, 8), (0.5, 0.5, 0.5)
    rng = workloads.rng_for(91, 0)
    ns, n_e, kT, g = 40, 30.0, 0.02, 2.0
    psi = workloads.random_subspace(n, h, ns, rng)
    eps = workloads.random_eigenvalues(ns, rng, -0.3, 0.3)
    if gap is not None:
        eps, _ = workloads.place_degenerate_pairs(eps, 4, 2, 15, gap, rng, window=4)
    w = float(np.prod(h))
    dV = workloads.smooth_directions(n, h, 1, 1, rng)[0, 0] * 3.0
    X = oracle.project(psi, w * dV)
    mu = oracle.solve_mu([eps], n_e, kT, g)
    L = oracle.loewner(eps, mu, kT)
    dmu = oracle.dmu_shift([L], [X])
    drho = oracle.density_response(psi, oracle.subspace_response(L, X, dmu), g)
    eta = 1e-4
    D = lambda et: (_projected_density(psi, eps, X, et, n_e, kT, g)
                    - _projected_density(psi, eps, X, -et, n_e, kT, g)) / (2 * et)
    fd = (4 * D(eta / 2) - D(eta)) / 3
    assert rel_err(drho, fd) < 1e-8


# ---------------------------------------------------------------------------
# P3: textbook special case -- the dense Adler-Wiser chi_0 matrix with the
# rank-one fixed-electron-number correction, applied to dV.
# ---------------------------------------------------------------------------

def test_adler_wiser_dense(cfg1):
    sysm = oracle_system(cfg1)
    psi, eps, g, w = sysm.psi[0], sysm.eps[0], sysm.occ_factor, sysm.w
    mu = oracle.solve_mu(sysm.eps, sysm.n_electrons, sysm.kT, g)
    L = oracle.loewner(eps, mu, sysm.kT)
    # chi0(r, r') = g sum_ij L_ij psi_i psi_j(r) psi_i psi_j(r') w - rank-one term
    P = np.einsum("ri,rj->rij", psi, psi).reshape(psi.shape[0], -1)
    chi = g * w * (P @ (L.ravel()[:, None] * P.T))
    d = (psi ** 2) @ np.diag(L)
    chi -= g * w * np.outer(d, d) / np.sum(np.diag(L))
    dV = workloads.smooth_directions(sysm.n, sysm.h, 1, 1, workloads.rng_for(92, 0))[0, 0]
    X = oracle.project(psi, w * dV)
    drho = oracle.density_response(psi, oracle.subspace_response(L, X, oracle.dmu_shift([L], [X])), g)
    assert rel_err(drho, chi @ dV) < 1e-13


# ---------------------------------------------------------------------------
# P4: invariants
# ---------------------------------------------------------------------------

def _response(sysm, dV):
    g, w = sysm.occ_factor, sysm.w
    mu = oracle.solve_mu(sysm.eps, sysm.n_electrons, sysm.kT, g)
    L = [oracle.loewner(e, mu, sysm.kT) for e in sysm.eps]
    X = [oracle.project(p, w * d) for p, d in zip(sysm.psi, dV)]
    dmu = oracle.dmu_shift(L, X)
    return [oracle.density_response(p, oracle.subspace_response(Ls, Xs, dmu), g)
            for p, Ls, Xs in zip(sysm.psi, L, X)]


def test_invariants_cfg1(cfg1):
    sysm = oracle_system(cfg1)
    w = sysm.w
    res = oracle.gateaux(sysm, cfg1["V"])
    for k in range(cfg1["V"].shape[0]):
        drho = res["drho"][k, 0]
        assert abs(w * drho.sum()) <= 1e-13 * np.sqrt(w * np.sum(drho ** 2)) * np.sqrt(drho.size)
    rng = workloads.rng_for(93, 0)
    a, b = workloads.smooth_directions(sysm.n, sysm.h, 2, 1, rng)[:, 0]
    ra, rb = _response(sysm, [a])[0], _response(sysm, [b])[0]
    lhs, rhs = w * np.dot(a, rb), w * np.dot(b, ra)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1e-300) + 1e-16
    assert w * np.dot(a, ra) < 0 and w * np.dot(b, rb) < 0   # <v, chi0 v> <= 0
    # uniform shift is absorbed by mu'
    r0 = _response(sysm, [np.full(sysm.n_grid, 0.37)])[0]
    assert np.max(np.abs(r0)) < 1e-12
    # linearity
    rab = _response(sysm, [2.0 * a - 0.5 * b])[0]
    assert rel_err(rab, 2.0 * ra - 0.5 * rb) < 1e-13


def test_chi0_negative_semidefinite():
    n, h = (6, 6, 6), (0.5, 0.5, 0.5)
    rng = workloads.rng_for(94, 0)
    psi = workloads.random_subspace(n, h, 30, rng)
    eps = workloads.random_eigenvalues(30, rng, -0.2, 0.2)
    sysm = oracle.System(n=n, h=h, psi=[psi], eps=[eps], rho=[np.ones(216)], n_electrons=20.0,
                         kT=0.03, g=2.0)
    N = sysm.n_grid
    chi = np.stack([_response(sysm, [np.eye(N)[r]])[0] for r in range(N)], axis=1)
    # chi is symmetric in the w-weighted sense: w chi must be a symmetric matrix
    A = sysm.w * chi
    assert np.max(np.abs(A - A.T)) < 1e-14 * np.max(np.abs(A))
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() <= 1e-13 * np.abs(ev).max()


def test_spin_identical_channels_equal_restricted():
    n, h = (8, 8, 8), (0.5, 0.5, 0.5)
    rng = workloads.rng_for(95, 0)
    psi = workloads.random_subspace(n, h, 24, rng)
    eps = workloads.random_eigenvalues(24, rng, -0.3, 0.3)
    rho = 0.05 + 0.5 * psi[:, 0] ** 2
    restricted = oracle.System(n=n, h=h, psi=[psi], eps=[eps], rho=[rho], n_electrons=18.0,
                               kT=0.01, g=2.0)
    spin = oracle.System(n=n, h=h, psi=[psi, psi], eps=[eps, eps], rho=[rho / 2, rho / 2],
                         n_electrons=18.0, kT=0.01, g=1.0)
    V = workloads.smooth_directions(n, h, 2, 1, rng)
    Vs = np.concatenate([V / 2, V / 2], axis=1)
    r1 = oracle.gateaux(restricted, V)
    r2 = oracle.gateaux(spin, Vs)
    assert rel_err(r2["F"].sum(axis=1), r1["F"][:, 0]) < 1e-13
    assert np.allclose(r2["dmu"], r1["dmu"], rtol=1e-13, atol=0)


def test_batch_equals_separate(cfg1):
    sysm = oracle_system(cfg1)
    V = cfg1["V"]
    full = oracle.gateaux(sysm, V)
    for k in range(V.shape[0]):
        one = oracle.gateaux(sysm, V[k:k + 1])
        assert np.array_equal(one["F"][0], full["F"][k])


# ---------------------------------------------------------------------------
# P5: closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["spectral", "fd"])
def test_hartree_plane_wave(kind):
    n, h = (12, 10, 8), (0.4, 0.5, 0.6)
    m = np.array([1, 2, 3])
    x = workloads.grid_coords(n, h)
    G = 2 * np.pi * m / (np.array(n) * np.array(h))
    v = np.cos(x @ G)
    if kind == "spectral":
        g2 = float(G @ G)
    else:
        g2 = float(np.sum(4.0 / np.array(h) ** 2 * np.sin(G * np.array(h) / 2) ** 2))
    assert rel_err(oracle.hartree(v, n, h, kind), 4 * np.pi / g2 * v) < 1e-13
    assert np.max(np.abs(oracle.hartree(np.ones(np.prod(n)), n, h, kind))) < 1e-14


@pytest.mark.parametrize("spin", [False, True])
def test_lda_kernel_is_derivative_of_potential(spin):
    rho = np.geomspace(1e-4, 10.0, 50)
    d = 1e-6 * rho
    fd = (oracle.lda_vx(rho + d, spin) - oracle.lda_vx(rho - d, spin)) / (2 * d)
    assert np.max(np.abs(oracle.lda_fx(rho, spin) - fd) / np.abs(fd)) < 1e-8
    # the closed form itself: Slater exchange V_x = -(3 rho / pi)^(1/3)
    assert np.allclose(oracle.lda_vx(rho, False), -(3 * rho / np.pi) ** (1 / 3), rtol=1e-15)
    assert np.allclose(oracle.lda_vx(rho, True), -(6 * rho / np.pi) ** (1 / 3), rtol=1e-15)


def test_two_level_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "two_level.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, *nums = line.split()
            vals[name] = np.array([float(x) for x in nums])
    eps, kT = vals["eps"], vals["kT"][0]
    mu = oracle.solve_mu([eps], 2.0, kT, 2.0)
    assert abs(mu - vals["mu"][0]) < 1e-15
    assert np.allclose(oracle.fermi(eps, mu, kT), vals["occ"], rtol=1e-15, atol=0)
    L = oracle.loewner(eps, mu, kT)
    assert np.allclose(L.ravel(), vals["L"], rtol=4e-16, atol=0)
    X = vals["X"].reshape(2, 2)
    dmu = oracle.dmu_shift([L], [X])
    assert abs(dmu - vals["dmu"][0]) < 1e-16
    assert np.allclose(oracle.subspace_response(L, X, dmu).ravel(), vals["Xp"], rtol=1e-15, atol=1e-17)


def test_loewner_matches_mpmath():
    mp = pytest.importorskip("mpmath")
    # 1100 digits: deep states have 1 - f ~ e^-1500, and the divided difference
    # of two such occupations must not cancel to zero in the reference
    mp.mp.dps = 1100
    kT = 0.002
    base = np.array([-0.3, -0.01, -1e-4, 0.0, 2e-4, 0.02, 0.5, 3.0, -2.0])
    gaps = [0.0, 1e-12, 1e-9, 1e-6, 1e-3, 0.1]
    eps = np.unique(np.concatenate([base + g for g in gaps]))
    mu = 1e-5
    L = oracle.loewner(eps, mu, kT)

    def f(e):
        return 1 / (1 + mp.e ** ((mp.mpf(e) - mp.mpf(mu)) / mp.mpf(kT)))

    worst = 0.0
    for i in range(len(eps)):
        for j in range(len(eps)):
            ei, ej = mp.mpf(float(eps[i])), mp.mpf(float(eps[j]))
            if i == j:
                fi = f(float(eps[i]))
                ref = -fi * (1 - fi) / mp.mpf(kT)
            else:
                ref = (f(float(eps[i])) - f(float(eps[j]))) / (ei - ej)
            if abs(ref) < mp.mpf("1e-300"):
                assert abs(L[i, j]) < 1e-290
                continue
            err = float(abs((mp.mpf(float(L[i, j])) - ref) / ref))
            # conditioning: rounding x = (eps - mu)/kT moves L by ~|x| ulp
            xi, xj = (eps[i] - mu) / kT, (eps[j] - mu) / kT
            bound = 4e-15 + 1.2e-16 * (abs(xi) + abs(xj) + abs(xi - xj))
            worst = max(worst, err / bound)
    assert worst < 1.0


def test_loewner_from_occ_matches_closed_form_away_from_degeneracy():
    eps = np.sort(workloads.rng_for(96, 0).uniform(-0.2, 0.2, 60))
    mu, kT = 0.01, 0.01
    occ = oracle.fermi(eps, mu, kT)
    La = oracle.loewner(eps, mu, kT)
    Lb = oracle.loewner_from_occ(eps, occ, kT)
    # subtraction of occupations loses digits only where f is close to 0 or 1
    assert np.max(np.abs(La - Lb)) < 1e-9 * np.max(np.abs(La))


def test_recursive_fermi_closed_form():
    eps = np.linspace(-0.5, 0.5, 101)
    mu, kT = 0.03, 0.01
    for T in (3, 8, 10):
        y = (eps - mu) / kT
        inside = np.abs(y) < 2.0 ** (T + 1)     # the closed form's domain
        closed = 1.0 / (1.0 + np.exp(2.0 ** (T + 1) * np.arctanh(y[inside] / 2.0 ** (T + 1))))
        rec = oracle.fermi_recursive(eps, mu, kT, T)[inside]
        assert np.max(np.abs(rec - closed)) < 1e-14
    # T = 10 is within 1e-6 of Fermi-Dirac on this window (the paper's T = 8-10)
    assert np.max(np.abs(oracle.fermi_recursive(eps, mu, kT, 10) - oracle.fermi(eps, mu, kT))) < 1e-6


def _matrix_recursion(H, mu, kT, T):
    """The paper's recursion applied to a dense symmetric matrix (brute force)."""
    n = H.shape[0]
    I = np.eye(n)
    X = 0.5 * I - 2.0 ** (-(T + 2)) * (H - mu * I) / kT
    for _ in range(T):
        X2 = X @ X
        X = np.linalg.solve(X2 + (I - X) @ (I - X), X2)   # X2 (X2 + (I-X)^2)^-1, commuting
        X = 0.5 * (X + X.T)
    return X


@pytest.mark.parametrize("T", [4, 8, 10])
def test_recursive_response_is_derivative_of_matrix_recursion(T):
    """L_T o E equals the central difference of the literal matrix recursion
    X_T(D + lam E) (one Richardson step), with a 1e-9 Ha pair in D."""
    rng = workloads.rng_for(97, T)
    eps = np.sort(rng.uniform(-0.3, 0.3, 9))
    eps[4] = eps[3] + 1e-9
    mu, kT = 0.02, 0.01
    E = rng.standard_normal((9, 9))
    E = 0.5 * (E + E.T)
    D = np.diag(eps)

    def d(eta):
        return (_matrix_recursion(D + eta * E, mu, kT, T) -
                _matrix_recursion(D - eta * E, mu, kT, T)) / (2 * eta)

    eta = 1e-4 * kT
    fd = (4 * d(eta / 2) - d(eta)) / 3
    LT = oracle.loewner_recursive(eps, mu, kT, T)
    assert np.max(np.abs(LT * E - fd)) < 1e-7 * np.max(np.abs(LT * E))


def test_recursive_response_matches_mpmath_closed_form():
    """Entries of L_T against divided differences of the closed form
    f_T(e) = 1 / (1 + exp(2^(T+1) artanh(2^-(T+1) (e - mu) / kT))) at 160 digits
    (deep states have 1 - f_T ~ e^-180, whose differences must not cancel in the
    reference), gaps down to 1e-12 Ha; the diagonal is f_T'."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 160
    T, mu, kT = 8, 0.01, 0.005
    base = np.array([-0.8, -0.05, -0.003, 0.0, 0.004, 0.02, 0.3, 0.9])
    eps = np.unique(np.concatenate([base + g for g in (0.0, 1e-12, 1e-9, 1e-6, 1e-3)]))
    LT = oracle.loewner_recursive(eps, mu, kT, T)
    c = mp.mpf(2) ** (T + 1)

    def fT(e):
        y = (mp.mpf(e) - mp.mpf(mu)) / mp.mpf(kT)
        return 1 / (1 + mp.e ** (c * mp.atanh(y / c)))

    worst = 0.0
    for i in range(len(eps)):
        for j in range(len(eps)):
            if i == j:
                ref = mp.diff(fT, mp.mpf(float(eps[i])))
            else:
                ref = (fT(float(eps[i])) - fT(float(eps[j]))) / (mp.mpf(float(eps[i])) - mp.mpf(float(eps[j])))
            err = float(abs((mp.mpf(float(LT[i, j])) - ref) / ref))
            # conditioning of x_0 = 1/2 - 2^-(T+2) y: rounding x_0 loses ~2^(T+2)|y| ulp...
            xi, xj = abs(eps[i] - mu) / kT, abs(eps[j] - mu) / kT
            bound = 2e-14 + 2.0 ** (T + 2) * 2.2e-16 * (1 + xi + xj) / 8
            worst = max(worst, err / bound)
    assert worst < 1.0


def test_recursive_response_converges_to_fermi_dirac():
    """L_T -> the Fermi-Dirac Loewner matrix with error ~ 4^-T."""
    eps = np.linspace(-1.0, 1.0, 41)
    mu, kT = 0.1, 0.05
    L = oracle.loewner(eps, mu, kT)
    errs = [np.abs(oracle.loewner_recursive(eps, mu, kT, T) - L).max() / np.abs(L).max()
            for T in (6, 7, 8, 9, 10)]
    ratios = [errs[t] / errs[t + 1] for t in range(4)]
    assert all(3.5 < r < 4.5 for r in ratios)
    assert errs[-1] < 1e-6


@pytest.mark.parametrize("spin", [False, True])
def test_krylov_step_matches_brute_force_krylov_least_squares(cfg1, spin):
    """The LRDM step (Eqs. jlowrank, krylovOrtho, plowrank, relativeError)
    against an independent construction: the Krylov space span{R, JR, ...,
    J^(r-1) R} built by applying J (the Gateaux map) repeatedly, and the
    least-squares solution min ||J Delta - R||_w over it by lstsq.  Also: the
    directions are w-orthonormal and s_rel does not increase with the rank."""
    if spin:
        sysm_cfg = workloads.spin_pair_system(98, (10, 9, 8), 40, 36, 60.0, 0.01, 1)
        sysm = oracle_system(sysm_cfg)
        R = sysm_cfg["R"]
    else:
        sysm = oracle_system(cfg1)
        R = cfg1["R"]
    w = sysm.w
    out = oracle.lrdm_krylov_step(sysm, R, s_tol=1e-6, r_max=4)
    r = out["rank"]
    assert r == 4
    U = out["U"].reshape(r, -1)
    assert np.max(np.abs(w * U @ U.T - np.eye(r))) < 1e-12
    assert all(b <= a + 1e-12 for a, b in zip(out["s_rel"], out["s_rel"][1:]))

    def J(v):
        return oracle.gateaux(sysm, v.reshape((1,) + R.shape))["F"][0]

    Kr = [np.asarray(R, dtype=np.float64)]
    for _ in range(r):
        Kr.append(J(Kr[-1]))
    B = np.stack([k.ravel() for k in Kr[:r]], axis=1)          # R, JR, ..., J^(r-1) R
    JB = np.stack([k.ravel() for k in Kr[1:]], axis=1)         # J of each
    b, *_ = np.linalg.lstsq(np.sqrt(w) * JB, np.sqrt(w) * np.ravel(R), rcond=None)
    ref = (B @ b).reshape(R.shape)
    assert rel_err(out["delta"], ref) < 1e-8
    # and the residual of the low-rank model equals the last s_rel
    res = (JB @ b) - np.ravel(R)
    s_ref = np.sqrt(np.sum(res * res) / np.sum(np.ravel(R) ** 2))
    assert abs(out["s_rel"][-1] - s_ref) < 1e-8 * max(s_ref, 1e-3)


def test_krylov_step_rank_control_and_alpha_schedule(cfg1):
    sysm = oracle_system(cfg1)
    R = cfg1["R"]
    full = oracle.lrdm_krylov_step(sysm, R, s_tol=1e-9, r_max=5)
    # the rank is the first one whose s_rel is below the tolerance
    tol = 0.5 * (full["s_rel"][1] + full["s_rel"][2])
    out = oracle.lrdm_krylov_step(sysm, R, s_tol=tol, r_max=5)
    assert out["rank"] == 3
    assert np.allclose(out["U"], full["U"][:3], atol=1e-13)
    assert oracle.alpha_schedule(2.5) == 0.1 and oracle.alpha_schedule(1.0) == 0.5
    assert out["alpha"] == (0.5 if out["r_norm"] < 2.0 else 0.1)
    rho = sysm.rho[0][None, :]
    out = oracle.lrdm_krylov_step(sysm, R, s_tol=tol, r_max=5, alpha=0.3, rho=rho)
    assert np.allclose(out["rho_new"], rho - 0.3 * out["delta"], atol=1e-15)


def test_mu_bisection():
    eps = np.array([-1.0, -0.5, 0.0, 0.5])
    # half filling of a spectrum symmetric about -0.25: mu = -0.25 exactly
    # (kT = 0.1 keeps dN/dmu large enough for mu to be well conditioned)
    mu = oracle.solve_mu([eps], 4.0, 0.1, 2.0)
    assert abs(mu - (-0.25)) < 1e-12
    with pytest.raises(ValueError):
        oracle.solve_mu([eps], 8.0, 0.01, 2.0)


# ---------------------------------------------------------------------------
# P6: least-squares step
# ---------------------------------------------------------------------------

def _ls_data(K=5, N=300, seed=0):
    rng = workloads.rng_for(97, seed)
    F = rng.standard_normal((K, 1, N))
    V = rng.standard_normal((K, 1, N))
    R = rng.standard_normal((1, N))
    return F, V, R


def test_ls_single_direction_closed_form():
    F, V, R = _ls_data(K=1)
    w = 0.125
    out = oracle.lrdm_apply(R, V, F, w, 0.5, rho=np.zeros((1, 300)))
    a = np.dot(F[0, 0], R[0]) / np.dot(F[0, 0], F[0, 0])
    assert abs(out["a"][0] - a) < 1e-14 * abs(a)
    assert np.allclose(out["rho_new"], -0.5 * a * V[0], rtol=1e-14, atol=0)


def test_ls_matches_lstsq_and_exact_span():
    F, V, R = _ls_data(K=6)
    w = 0.3
    out = oracle.lrdm_apply(R, V, F, w, 1.0)
    a_ref = np.linalg.lstsq(np.sqrt(w) * F[:, 0].T, np.sqrt(w) * R[0], rcond=None)[0]
    assert np.allclose(out["a"], a_ref, rtol=1e-12)
    res = F[:, 0].T @ a_ref - R[0]
    assert abs(out["s_rel"] - np.linalg.norm(res) / np.linalg.norm(R[0])) < 1e-13
    R2 = (F[:, 0].T @ np.arange(1.0, 7.0))[None, :]
    out2 = oracle.lrdm_apply(R2, V, F, w, 1.0)
    assert out2["s_rel"] < 1e-13
    assert np.allclose(out2["a"], np.arange(1.0, 7.0), rtol=1e-12)


def test_ls_singular_is_min_norm():
    F, V, R = _ls_data(K=4)
    F[3] = F[1]
    out = oracle.lrdm_apply(R, V, F, 1.0, 1.0)
    assert out["singular"]
    a_ref = np.linalg.lstsq(F[:, 0].T, R[0], rcond=1e-10)[0]
    assert np.allclose(out["a"], a_ref, rtol=1e-10)
    assert abs(out["a"][1] - out["a"][3]) < 1e-12 * abs(out["a"][1])


# ---------------------------------------------------------------------------
# P7: adjoint
# ---------------------------------------------------------------------------

def _small_system(occ_mode, nspin=1, seed=0, pair_gap=None):
    n, h = (8, 8, 8), (0.5, 0.5, 0.5)
    rng = workloads.rng_for(98, seed)
    ns = 20
    psi = [workloads.random_subspace(n, h, ns, rng) for _ in range(nspin)]
    eps = [workloads.random_eigenvalues(ns, rng, -0.1, 0.1) for _ in range(nspin)]
    if pair_gap is not None:
        eps[0], _ = workloads.place_degenerate_pairs(eps[0], 2, 1, 7, pair_gap, rng, window=3)
    g = 2.0 if nspin == 1 else 1.0
    ne = 14.0 if nspin == 1 else 13.0
    rho = [0.05 + 0.2 * p[:, 0] ** 2 for p in psi]
    sysm = oracle.System(n=n, h=h, psi=psi, eps=eps, rho=rho, n_electrons=ne, kT=0.02, g=g)
    if occ_mode:
        mu = oracle.solve_mu(eps, ne, 0.02, g)
        sysm.occ = [oracle.fermi(e, mu, 0.02) for e in eps]
    return sysm


@pytest.mark.parametrize("nspin", [1, 2])
def test_adjoint_dot_product(nspin):
    sysm = _small_system(False, nspin)
    rng = workloads.rng_for(99, nspin)
    V = rng.standard_normal((3, nspin, sysm.n_grid))
    fbar = rng.standard_normal((3, nspin, sysm.n_grid))
    fwd = oracle.gateaux(sysm, V)
    bwd = oracle.backward(sysm, fbar, fwd)
    lhs = float(np.sum(fbar * fwd["F"]))
    rhs = float(np.sum(bwd["vbar"] * V))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _loss(sysm, V, fbar):
    return float(np.sum(fbar * oracle.gateaux(sysm, V)["F"]))


@pytest.mark.parametrize("pair_gap", [None, 1e-9])
def test_adjoint_fd_occupations_and_eigenvalues(pair_gap):
    sysm = _small_system(True, 1, seed=3, pair_gap=pair_gap)
    rng = workloads.rng_for(99, 5)
    V = rng.standard_normal((2, 1, sysm.n_grid))
    fbar = rng.standard_normal((2, 1, sysm.n_grid))
    bwd = oracle.backward(sysm, fbar, V=V)
    eta = 1e-4
    for p in range(4):
        d_occ = rng.standard_normal(len(sysm.eps[0])) * 0.1
        d_eps = rng.standard_normal(len(sysm.eps[0])) * 1e-3
        if pair_gap is not None:
            d_eps[:] = 0.0   # eps-gradient is taken at fixed pairs only away from degeneracy
        base_occ, base_eps = sysm.occ[0].copy(), sysm.eps[0].copy()

        def at(t):
            sysm.occ[0] = base_occ + t * d_occ
            sysm.eps[0] = base_eps + t * d_eps
            return _loss(sysm, V, fbar)
        fd = (at(eta) - at(-eta)) / (2 * eta)
        sysm.occ[0], sysm.eps[0] = base_occ, base_eps
        an = float(np.dot(bwd["occ_bar"][0], d_occ) + np.dot(bwd["eps_bar"][0], d_eps))
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_adjoint_fd_total_eps_default_mode():
    sysm = _small_system(False, 1, seed=4)
    rng = workloads.rng_for(99, 6)
    V = rng.standard_normal((2, 1, sysm.n_grid))
    fbar = rng.standard_normal((2, 1, sysm.n_grid))
    fwd = oracle.gateaux(sysm, V)
    bwd = oracle.backward(sysm, fbar, fwd)
    tot = oracle.total_eps_grad(sysm, bwd["eps_bar"], bwd["occ_bar"], fwd["mu"])
    eta = 1e-5
    for p in range(4):
        d = rng.standard_normal(len(sysm.eps[0])) * 1e-2
        base = sysm.eps[0].copy()
        sysm.eps[0] = base + eta * d
        lp = _loss(sysm, V, fbar)
        sysm.eps[0] = base - eta * d
        lm = _loss(sysm, V, fbar)
        sysm.eps[0] = base
        fd = (lp - lm) / (2 * eta)
        an = float(np.dot(tot[0], d))
        assert abs(fd - an) <= 1e-6 * abs(an)
