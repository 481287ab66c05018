"""FP64 numpy oracle of the LRDM hot path (arXiv 2211.07894).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Nothing in the CUDA
library imports this file.

Discretisation used throughout (the paper's finite-element overlap M becomes a
uniform quadrature weight, which the paper allows in §II.D's closing remark on
finite-difference and plane-wave bases):

* periodic grid n0 x n1 x n2, spacing h, flat C-order index r, N_g = n0 n1 n2;
* quadrature weight w = h0 h1 h2, inner product <a, b> = w sum_r a(r) b(r);
* subspace basis Psi (N_g x N_s, row-major) with Psi^T diag(w) Psi = I, i.e.
  grid values of functions with int psi_i psi_j = delta_ij;
* occupancy factor g (2 spin-restricted, 1 per spin channel).

Functions are direct evaluations in the order of the paper's equations.  No
blocking or fusion beyond what each docstring states.

Pins: every function is checked against brute force, closed forms, mpmath or
invariants (tests/test_oracle_pins.py, tests/test_kpoint_pins.py,
tests/test_scf_lrdm.py); the decisions of lrdma_step, of which the paper
prints no worked example, against closed forms on an exactly linear residual
map (tests/test_lrdma_pins.py).
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
from scipy.special import expit

__all__ = [
    "System", "fermi", "electron_count", "solve_mu", "loewner", "loewner_from_occ",
    "lda_vx", "lda_fx", "poisson_symbol", "hartree", "density",
    "perturbation_potential", "project", "dmu_shift", "subspace_response",
    "density_response", "gateaux", "lrdm_apply", "backward", "total_eps_grad",
    "fermi_recursive", "loewner_recursive", "alpha_schedule", "lrdm_krylov_step",
    "LrdmaState", "lrdma_step", "KpointSystem", "solve_mu_kpoints", "density_kpoints",
    "gateaux_kpoints", "backward_kpoints",
]


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class System:
    """One Kohn-Sham system restricted to its Chebyshev-filtered subspace.

    psi[s]  : (N_g, N_s[s]) float64, Psi^T diag(w) Psi = I     (Psi~_R, §II.C)
    eps[s]  : (N_s[s],) float64 projected eigenvalues D        (§II.C)
    rho[s]  : (N_g,) density entering the xc kernel; for nspin = 1 the total
              density, for nspin = 2 the channel densities      (Eq. kseqcont)
    occ[s]  : optional occupations; None -> Fermi-Dirac(eps, mu, kT)
    fermi_T : 0 -> the response uses the Loewner matrix of Fermi-Dirac; T > 0
              -> the first-order response of the paper's depth-T recursive
              Fermi-operator expansion (mu and the occupations stay
              Fermi-Dirac: they describe the SCF state the response is taken
              about)
    """

    n: Sequence[int]
    h: Sequence[float]
    psi: List[np.ndarray]
    eps: List[np.ndarray]
    rho: List[np.ndarray]
    n_electrons: float
    kT: float
    g: Optional[float] = None
    occ: Optional[List[np.ndarray]] = None
    poisson: str = "spectral"
    degen_tol: float = 1e-5
    fermi_T: int = 0

    @property
    def nspin(self) -> int:
        return len(self.psi)

    @property
    def n_grid(self) -> int:
        return int(np.prod(self.n))

    @property
    def w(self) -> float:
        return float(np.prod(self.h))

    @property
    def occ_factor(self) -> float:
        if self.g is not None and self.g != 0:
            return float(self.g)
        return 2.0 if self.nspin == 1 else 1.0


# ---------------------------------------------------------------------------
# Fermi-Dirac occupations and the chemical potential (Eq. kseqcont, §II.A)
# ---------------------------------------------------------------------------

def fermi(eps, mu, kT):
    """f(eps, mu) = 1 / (1 + exp((eps - mu) / kT))  (Eq. kseqcont)."""
    return expit(-(np.asarray(eps, dtype=np.float64) - mu) / kT)


def electron_count(eps_channels, mu, kT, g):
    """g * sum over channels and states of f(eps, mu)  (Eq. kseqcont; the spin
    channels share one mu, §II.D)."""
    return g * sum(float(fermi(e, mu, kT).sum()) for e in eps_channels)


def solve_mu(eps_channels, n_electrons, kT, g, max_iter=400):
    """mu such that g sum_i f(eps_i, mu) = N_e (Eq. kseqcont), by bisection.

    Raises ValueError when N_e is not strictly between 0 and g * (number of
    states), where no finite mu exists.
    """
    n_states = sum(len(e) for e in eps_channels)
    if not (0.0 < n_electrons < g * n_states):
        raise ValueError("n_electrons must lie strictly between 0 and g * N_s")
    lo = min(float(np.min(e)) for e in eps_channels) - 800.0 * kT
    hi = max(float(np.max(e)) for e in eps_channels) + 800.0 * kT
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if electron_count(eps_channels, mid, kT, g) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# ---------------------------------------------------------------------------
# The divided-difference (Loewner) matrix of the Fermi function
# ---------------------------------------------------------------------------

def _log_cosh(y):
    a = np.abs(y)
    return a + np.log1p(np.exp(-2.0 * a)) - np.log(2.0)


def _log_sinhc(u):
    """log(sinh(u)/u), even in u, = 0 at u = 0."""
    a = np.abs(u)
    out = np.empty_like(a)
    small = a < 0.5
    with np.errstate(divide="ignore", invalid="ignore"):
        s = a[small]
        out[small] = np.log1p(np.where(s > 0, np.sinh(s) / np.where(s > 0, s, 1.0) - 1.0, 0.0))
        b = a[~small]
        out[~small] = b + np.log1p(-np.exp(-2.0 * b)) - np.log(2.0) - np.log(b)
    return out


def loewner(eps, mu, kT):
    """Loewner matrix of f at the projected eigenvalues.

    For the diagonal projected Hamiltonian D, the first-order change of
    f(D + lambda X', mu) is L o X' with L_ij = (f_i - f_j) / (eps_i - eps_j) and
    L_ii = df/deps = -f_i (1 - f_i) / kT (the derivative that the paper's
    Eq. subspaceDensityMatResponse asks for; Daleckii-Krein).

    Evaluated without cancellation through the identity
        L_ij = -sinhc((x_i - x_j)/2) / (4 kT cosh(x_i/2) cosh(x_j/2)),
    x = (eps - mu)/kT, sinhc(u) = sinh(u)/u.  Entries whose factors could
    overflow are evaluated in the log domain (they are below 1e-150).
    """
    eps = np.asarray(eps, dtype=np.float64)
    x = (eps - mu) / kT
    xi = x[:, None]
    xj = x[None, :]
    u = 0.5 * (xi - xj)
    direct = (np.abs(xi) < 700.0) & (np.abs(xj) < 700.0) & (np.abs(u) < 700.0)
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        safe_u = np.where(u == 0.0, 1.0, u)
        sinhc = np.where(u == 0.0, 1.0, np.sinh(safe_u) / safe_u)
        val_direct = -sinhc / (4.0 * kT * np.cosh(0.5 * xi) * np.cosh(0.5 * xj))
    if np.all(direct):
        return val_direct
    logmag = _log_sinhc(u) - np.log(4.0 * kT) - _log_cosh(0.5 * xi) - _log_cosh(0.5 * xj)
    return np.where(direct, val_direct, -np.exp(logmag))


def loewner_from_occ(eps, occ, kT, degen_tol=1e-5):
    """Loewner matrix built from given occupations (the adjoint's independent
    inputs): L_ij = (f_i - f_j)/(eps_i - eps_j) when |eps_i - eps_j| > tau,
    else -fbar (1 - fbar)/kT with fbar = (f_i + f_j)/2, tau = degen_tol * kT.
    The diagonal is -f_i (1 - f_i)/kT.  (Divided difference of f, §II.C.)
    """
    eps = np.asarray(eps, dtype=np.float64)
    f = np.asarray(occ, dtype=np.float64)
    de = eps[:, None] - eps[None, :]
    df = f[:, None] - f[None, :]
    fb = 0.5 * (f[:, None] + f[None, :])
    tau = degen_tol * kT
    near = np.abs(de) <= tau
    with np.errstate(divide="ignore", invalid="ignore"):
        L = np.where(near, -fb * (1.0 - fb) / kT, df / np.where(near, 1.0, de))
    return L


def fermi_recursive(eps, mu, kT, T):
    """The paper's recursive Fermi-operator expansion applied to a diagonal
    matrix (Eq. recursiveFermiOperator): X_0 = 1/2 - 2^-(T+2) (eps - mu)/kT,
    X_n = X_{n-1}^2 / (X_{n-1}^2 + (1 - X_{n-1})^2), n = 1..T."""
    X = 0.5 - 2.0 ** (-(T + 2)) * (np.asarray(eps, dtype=np.float64) - mu) / kT
    for _ in range(T):
        X2 = X * X
        X = X2 / (X2 + (1.0 - X) ** 2)
    return X


def loewner_recursive(eps, mu, kT, T):
    """First-order response of the paper's recursive Fermi-operator expansion
    at the diagonal projected Hamiltonian D = diag(eps) (Eq.
    recursiveFermiOperator, canonical density-matrix perturbation theory):
    d/dlam X_T(D + lam E) = L_T o E (mu fixed; the mu' shift enters as E - mu' I).

    The recursion's steps, perturbed in the paper's order:
      X_0 = 1/2 - 2^-(T+2) (D - mu)/kT            X_0^(1) = -2^-(T+2) E / kT
      X_n = P(X_{n-1}),  P(x) = x^2 / (x^2 + (1-x)^2)
    With X_{n-1} = diag(x) diagonal, the first-order change of P(X_{n-1}) along
    a symmetric X_{n-1}^(1) is [P](x_i, x_j) X_{n-1,ij}^(1), where [P] is the
    divided difference of P: P(a) - P(b) = (a - b)(a + b - 2ab) / (q(a) q(b)),
    q(x) = x^2 + (1-x)^2, so [P](a, b) = (a (1-b) + b (1-a)) / (q(a) q(b))
    exactly (at a = b it is P'(a)).  Hence L_T is -2^-(T+2)/kT times the
    elementwise product of the T matrices [P](x_{n-1,i}, x_{n-1,j}).  The
    recursion is carried on both X and I - X (the two matrices P is built
    from: x_n = x^2 / q, 1 - x_n = (1-x)^2 / q), so that states far below or
    above mu, where x_n rounds to 1 or 0, keep their relative accuracy."""
    z = 2.0 ** (-(T + 2)) * (np.asarray(eps, dtype=np.float64) - mu) / kT
    x, xb = 0.5 - z, 0.5 + z                  # X_0 and I - X_0
    n = x.shape[0]
    L = np.full((n, n), -(2.0 ** (-(T + 2))) / kT)
    for _ in range(T):
        q = x * x + xb * xb
        num = x[:, None] * xb[None, :] + xb[:, None] * x[None, :]
        L = L * (num / (q[:, None] * q[None, :]))
        x, xb = x * x / q, xb * xb / q
    return L


# ---------------------------------------------------------------------------
# Kernel K = K_xc + K_c (Eq. jacobian)
# ---------------------------------------------------------------------------

def lda_vx(rho, spin_polarized=False):
    """LDA exchange potential: -(3/pi)^(1/3) rho^(1/3), or for a spin channel
    -(6/pi)^(1/3) rho_s^(1/3)."""
    c = (6.0 / np.pi) ** (1.0 / 3.0) if spin_polarized else (3.0 / np.pi) ** (1.0 / 3.0)
    return -c * np.cbrt(np.asarray(rho, dtype=np.float64))


def lda_fx(rho, spin_polarized=False):
    """LDA exchange kernel dV_x/drho = -(1/3)(3/pi)^(1/3) rho^(-2/3) (spin
    channel: (6/pi)^(1/3), no cross-channel term).  The density is floored at
    1e-12.  This is K_xc of Eq. jacobian for exchange-only LDA."""
    c = (6.0 / np.pi) ** (1.0 / 3.0) if spin_polarized else (3.0 / np.pi) ** (1.0 / 3.0)
    r = np.maximum(np.asarray(rho, dtype=np.float64), 1e-12)
    return -(c / 3.0) * r ** (-2.0 / 3.0)


def poisson_symbol(n, h, kind="spectral"):
    """4 pi / |G|^2 on the FFT grid (G = 2 pi m / (n h)), G = 0 set to 0.
    kind = "fd" uses the second-order finite-difference symbol
    sum_d (4/h_d^2) sin^2(G_d h_d / 2) in place of |G|^2."""
    axes = []
    for nd, hd in zip(n, h):
        m = np.fft.fftfreq(nd) * nd
        G = 2.0 * np.pi * m / (nd * hd)
        if kind == "fd":
            axes.append((4.0 / hd ** 2) * np.sin(0.5 * G * hd) ** 2)
        else:
            axes.append(G ** 2)
    g2 = axes[0][:, None, None] + axes[1][None, :, None] + axes[2][None, None, :]
    with np.errstate(divide="ignore"):
        sym = np.where(g2 > 0.0, 4.0 * np.pi / np.where(g2 > 0.0, g2, 1.0), 0.0)
    sym[0, 0, 0] = 0.0
    return sym


def hartree(v, n, h, kind="spectral"):
    """Periodic Hartree potential of a density perturbation: solves
    -Lap V = 4 pi v with the mean dropped, V = F^-1[4 pi F[v] / |G|^2]
    (the Coulomb kernel K_c of Eq. jacobian, atomic units)."""
    vg = np.fft.fftn(np.asarray(v, dtype=np.float64).reshape(tuple(n)))
    return np.real(np.fft.ifftn(vg * poisson_symbol(n, h, kind))).ravel()


def density(psi, occ, g, floor=0.0):
    """rho(r) = g sum_i f_i psi_i(r)^2 (+ floor)  (Eq. densityChFSI with the
    overlap M replaced by the quadrature weight)."""
    return g * (np.asarray(psi) ** 2 @ np.asarray(occ)) + floor


def perturbation_potential(v_channels, fx_channels, n, h, kind="spectral"):
    """First-order potential change along direction v (H' of §II.C):
    dV_s = V_H[sum_s' v_s'] + f_xs * v_s  (Eq. jacobian K = K_xc + K_c; the
    Hartree term sees the total density, §II.D)."""
    vh = hartree(sum(np.asarray(v, dtype=np.float64) for v in v_channels), n, h, kind)
    return [vh + fx * np.asarray(v, dtype=np.float64) for v, fx in zip(v_channels, fx_channels)]


# ---------------------------------------------------------------------------
# Subspace density response (§II.C)
# ---------------------------------------------------------------------------

def project(psi, a):
    """X = Psi^T diag(a) Psi with a = w dV: the projected perturbation
    H-breve' = Psi~^T H~' Psi~ (Eq. densityMatResponseApprox).  Symmetrised."""
    X = psi.T @ (np.asarray(a)[:, None] * psi)
    return 0.5 * (X + X.T)


def dmu_shift(L_channels, X_channels):
    """mu' from Tr Gamma-breve^(1) = 0 with Gamma-breve^(1) = L o (X - mu' I):
    mu' = sum L_ii X_ii / sum L_ii, both sums over all channels (shared mu,
    §II.D; traceless condition, §II.C)."""
    num = sum(float(np.dot(np.diag(L), np.diag(X))) for L, X in zip(L_channels, X_channels))
    den = sum(float(np.sum(np.diag(L))) for L in L_channels)
    return num / den


def subspace_response(L, X, dmu):
    """Gamma-breve^(1) = L o (X - mu' I)  (Eq. subspaceDensityMatResponse)."""
    return L * (X - dmu * np.eye(X.shape[0]))


def density_response(psi, Xp, g):
    """drho(r) = g sum_ij Psi_ri Gamma-breve^(1)_ij Psi_rj: the diagonal of
    Psi Gamma-breve^(1) Psi^T (Eq. densityResponse)."""
    return g * np.einsum("ri,ri->r", psi @ Xp, psi)


def _occupations(system: System, mu: float):
    if system.occ is not None:
        return [np.asarray(o, dtype=np.float64) for o in system.occ]
    return [fermi(e, mu, system.kT) for e in system.eps]


def _loewner_channels(system: System, mu: float):
    if system.fermi_T:
        if system.occ is not None:
            raise ValueError("fermi_T with given occupations is not defined")
        return [loewner_recursive(e, mu, system.kT, system.fermi_T) for e in system.eps]
    if system.occ is not None:
        return [loewner_from_occ(e, o, system.kT, system.degen_tol)
                for e, o in zip(system.eps, system.occ)]
    return [loewner(e, mu, system.kT) for e in system.eps]


def gateaux(system: System, V):
    """Gateaux derivatives f_k of the residual R = F[rho] - rho along the
    directions V (Eq. jlowrank), computed in the subspace (§II.C, §II.D).

    V has shape (K, nspin, N_g).  Returns a dict with
      F    (K, nspin, N_g)  f_k = drho_k - v_k  (t_i of Eq. jlowrank)
      drho (K, nspin, N_g)
      dmu  (K,)             chemical-potential shifts mu'
      X    list over spin of (K, N_s, N_s) projected perturbations
      Xp   list over spin of (K, N_s, N_s) subspace density-matrix responses
      dV   (K, nspin, N_g)
      mu, L (list over spin), fx (list over spin)
    """
    V = np.asarray(V, dtype=np.float64)
    K = V.shape[0]
    ns = system.nspin
    g = system.occ_factor
    w = system.w
    mu = solve_mu(system.eps, system.n_electrons, system.kT, g)
    L = _loewner_channels(system, mu)
    fx = [lda_fx(r, spin_polarized=(ns == 2)) for r in system.rho]
    F = np.zeros_like(V)
    drho = np.zeros_like(V)
    dV = np.zeros_like(V)
    dmu = np.zeros(K)
    Xs = [np.zeros((K,) + L[s].shape) for s in range(ns)]
    Xps = [np.zeros((K,) + L[s].shape) for s in range(ns)]
    for k in range(K):
        dVk = perturbation_potential(list(V[k]), fx, system.n, system.h, system.poisson)
        X = [project(system.psi[s], w * dVk[s]) for s in range(ns)]
        dmu[k] = dmu_shift(L, X)
        for s in range(ns):
            Xp = subspace_response(L[s], X[s], dmu[k])
            drho[k, s] = density_response(system.psi[s], Xp, g)
            F[k, s] = drho[k, s] - V[k, s]
            dV[k, s] = dVk[s]
            Xs[s][k] = X[s]
            Xps[s][k] = Xp
    return {"F": F, "drho": drho, "dmu": dmu, "X": Xs, "Xp": Xps, "dV": dV,
            "mu": mu, "L": L, "fx": fx}


# ---------------------------------------------------------------------------
# Brillouin-zone sampling (§II.C closing paragraphs, Eq. tracelessCondition)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class KpointSystem:
    """A spin-restricted periodic system sampled at nk points kappa of the
    first Brillouin zone: per point a complex subspace Psi_kappa (N_g x N_s,
    Psi^H diag(w) Psi = I; the lattice-periodic parts of the Bloch functions,
    whose phase factors cancel in every product below) and its projected
    eigenvalues; BZ weights k_weights (positive, sum 1) stand for the BZ
    average.  One mu is shared by all points:
    g sum_kappa w_kappa sum_i f(eps_i,kappa, mu) = N_e."""

    n: Sequence[int]
    h: Sequence[float]
    psi: List[np.ndarray]
    eps: List[np.ndarray]
    k_weights: Sequence[float]
    rho: np.ndarray
    n_electrons: float
    kT: float
    g: float = 2.0
    poisson: str = "spectral"

    @property
    def w(self) -> float:
        return float(np.prod(self.h))


def solve_mu_kpoints(eps, k_weights, n_electrons, kT, g, max_iter=400):
    """mu with g sum_kappa w_kappa sum_i f(eps_i,kappa, mu) = N_e (the
    electron count of Eq. kseqcont averaged over the BZ), by bisection."""
    def count(mu):
        return g * sum(wk * float(fermi(e, mu, kT).sum()) for e, wk in zip(eps, k_weights))
    lo = min(float(np.min(e)) for e in eps) - 800.0 * kT
    hi = max(float(np.max(e)) for e in eps) + 800.0 * kT
    if not (count(lo) < n_electrons < count(hi)):
        raise ValueError("n_electrons outside the range the states can hold")
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if count(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def density_kpoints(system: KpointSystem, mu, floor=0.0):
    """rho(r) = g sum_kappa w_kappa sum_i f_i,kappa |psi_i,kappa(r)|^2 (+ floor)."""
    rho = np.full(system.psi[0].shape[0], float(floor))
    for psi, e, wk in zip(system.psi, system.eps, system.k_weights):
        rho = rho + system.g * wk * ((np.abs(psi) ** 2) @ fermi(e, mu, system.kT))
    return rho


def gateaux_kpoints(system: KpointSystem, V):
    """Gateaux derivatives of the residual for a BZ-sampled system.

      dV_k = V_H[v_k] + f_x v_k                        (as for one point)
      X_kappa = Psi_kappa^H diag(w dV_k) Psi_kappa     (Hermitian; H-breve')
      mu' from the BZ-averaged traceless condition (Eq. tracelessCondition):
        sum_kappa w_kappa sum_i L_kappa,ii (X_kappa,ii - mu') = 0
      Gamma_kappa = L_kappa o (X_kappa - mu' I)         (L_kappa real)
      drho_k = g sum_kappa w_kappa diag(Psi_kappa Gamma_kappa Psi_kappa^H)
      f_k = drho_k - v_k.
    V: (K, N_g) real.  Returns dict(F, drho, dmu, X (per kappa (K, N_s, N_s)
    complex), mu, L, fx).
    """
    V = np.asarray(V, dtype=np.float64)
    K = V.shape[0]
    g, w = system.g, system.w
    mu = solve_mu_kpoints(system.eps, system.k_weights, system.n_electrons, system.kT, g)
    L = [loewner(e, mu, system.kT) for e in system.eps]
    fx = lda_fx(system.rho)
    F = np.zeros_like(V)
    drho = np.zeros_like(V)
    dmu = np.zeros(K)
    Xs = [np.zeros((K,) + Lk.shape, dtype=np.complex128) for Lk in L]
    for k in range(K):
        dVk = perturbation_potential([V[k]], [fx], system.n, system.h, system.poisson)[0]
        X = []
        for psi in system.psi:
            Xk = psi.conj().T @ ((w * dVk)[:, None] * psi)
            X.append(0.5 * (Xk + Xk.conj().T))
        num = sum(wk * float(np.dot(np.diag(Lk), np.diag(Xk).real))
                  for wk, Lk, Xk in zip(system.k_weights, L, X))
        den = sum(wk * float(np.sum(np.diag(Lk))) for wk, Lk in zip(system.k_weights, L))
        dmu[k] = num / den
        for q, (psi, wk, Lk, Xk) in enumerate(zip(system.psi, system.k_weights, L, X)):
            G = Lk * (Xk - dmu[k] * np.eye(Xk.shape[0]))
            drho[k] += g * wk * np.einsum("ri,ri->r", psi @ G, psi.conj()).real
            Xs[q][k] = Xk
        F[k] = drho[k] - V[k]
    return {"F": F, "drho": drho, "dmu": dmu, "X": Xs, "mu": mu, "L": L, "fx": fx}


def backward_kpoints(system: KpointSystem, Fbar):
    """Adjoint of gateaux_kpoints with respect to the directions (Euclidean
    inner product over array entries): v_bar = J^T f_bar for f = J v.

    <f_bar, drho> = g sum_kappa w_kappa tr(Gamma_kappa B_kappa) with
    B_kappa = Psi^H diag(f_bar) Psi; moving L and the mu' constraint across
    gives Y_kappa = L_kappa o B_kappa - (T / D) diag(L_kappa), T = sum_kappa
    w_kappa sum_i L_ii B_ii, D = sum_kappa w_kappa sum_i L_ii (the same
    traceless projection as the forward: the map is self-adjoint), then
      dV_bar = w g sum_kappa w_kappa diag(Psi_kappa Y_kappa Psi_kappa^H),
      v_bar = V_H[dV_bar] + f_x dV_bar - f_bar.
    Fbar: (K, N_g).  Returns v_bar (K, N_g)."""
    Fbar = np.asarray(Fbar, dtype=np.float64)
    g, w = system.g, system.w
    mu = solve_mu_kpoints(system.eps, system.k_weights, system.n_electrons, system.kT, g)
    L = [loewner(e, mu, system.kT) for e in system.eps]
    fx = lda_fx(system.rho)
    den = sum(wk * float(np.sum(np.diag(Lk))) for wk, Lk in zip(system.k_weights, L))
    vbar = np.zeros_like(Fbar)
    for k in range(Fbar.shape[0]):
        B = []
        for psi in system.psi:
            Bk = psi.conj().T @ (Fbar[k][:, None] * psi)
            B.append(0.5 * (Bk + Bk.conj().T))
        T = sum(wk * float(np.dot(np.diag(Lk), np.diag(Bk).real))
                for wk, Lk, Bk in zip(system.k_weights, L, B))
        dvbar = np.zeros(Fbar.shape[1])
        for psi, wk, Lk, Bk in zip(system.psi, system.k_weights, L, B):
            Y = Lk * Bk - (T / den) * np.diag(np.diag(Lk))
            dvbar += w * g * wk * np.einsum("ri,ri->r", psi @ Y, psi.conj()).real
        vbar[k] = hartree(dvbar, system.n, system.h, system.poisson) + fx * dvbar - Fbar[k]
    return vbar


# ---------------------------------------------------------------------------
# Low-rank least-squares step (Eqs. plowrank, relativeError, quasinewton)
# ---------------------------------------------------------------------------

def lrdm_apply(R, V, F, w, alpha, rho=None, rcond=1e-12):
    """Preconditioned update from K Gateaux derivatives.

    S_kl = <f_k, f_l>, c_k = <f_k, R> (the spin inner product sums the two
    channels, Eq. innerproductDirectsumHilbertspace); a = S^+ c (pseudo-inverse
    by eigendecomposition, eigenvalues below rcond * max dropped); the update
    Delta = sum_k a_k v_k solves J^lr Delta = R in least squares (Eq. plowrank:
    for orthonormal v it is exactly sum_ij u_i S^-1_ij <t_j, R>);
    s_rel = ||F a - R|| / ||R|| (Eq. relativeError); rho_new = rho - alpha Delta
    (Eq. quasinewton).
    """
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    K = V.shape[0]
    Fm = F.reshape(K, -1)
    Vm = V.reshape(K, -1)
    Rm = np.asarray(R, dtype=np.float64).ravel()
    S = w * (Fm @ Fm.T)
    c = w * (Fm @ Rm)
    lam, Q = np.linalg.eigh(S)
    lmax = float(lam.max()) if lam.size else 0.0
    keep = lam > rcond * lmax if lmax > 0 else np.zeros_like(lam, dtype=bool)
    a = Q[:, keep] @ ((Q[:, keep].T @ c) / lam[keep])
    singular = bool(np.count_nonzero(keep) < K)
    res = Fm.T @ a - Rm
    r2 = w * float(Rm @ Rm)
    s_rel = np.sqrt(w * float(res @ res) / r2) if r2 > 0 else 0.0
    delta = (Vm.T @ a).reshape(V.shape[1:])
    out = {"a": a, "S": S, "c": c, "s_rel": s_rel, "delta": delta, "singular": singular,
           "r_norm": np.sqrt(r2)}
    if rho is not None:
        out["rho_new"] = np.asarray(rho, dtype=np.float64) - alpha * delta
    return out


def alpha_schedule(r_norm, threshold=2.0):
    """The paper's damping: alpha = 0.1 while ||R|| is above a threshold of
    order one, 0.5 below it (§II.B; the threshold 2.0 of its setup, §III)."""
    return 0.5 if r_norm < threshold else 0.1


def _derivative(system, u):
    """t = d/dlam R[rho + lam u] for one direction u: the single-point response
    (u of shape (nspin, N_g)) or the Brillouin-zone-sampled one (u of shape
    (N_g,), a KpointSystem)."""
    if isinstance(system, KpointSystem):
        return gateaux_kpoints(system, u[None])["F"][0]
    return gateaux(system, u[None])["F"][0]


def lrdm_krylov_step(system: System, R, s_tol=0.3, r_max=8, alpha=None, rho=None, rcond=1e-12):
    """One LRDM preconditioning step with adaptively chosen rank (§II.B):

      u_1 = R / ||R||;  for i = 1, 2, ...:
        t_i = d/dlam R[rho + lam u_i]            (gateaux, one direction)
        a = S^+ c, S_kl = <t_k, t_l>, c_k = <t_k, R>,
        s_rel = ||sum_k a_k t_k - R|| / ||R||    (Eqs. plowrank, relativeError)
        stop when s_rel < s_tol or i = r_max;
        u_{i+1} = t_i - sum_{k<=i} <t_i, u_k> u_k,  u_{i+1} /= ||u_{i+1}||
                                                 (Eq. krylovOrtho, classical
                                                  Gram-Schmidt as printed)
      Delta = sum_k a_k u_k,  rho_new = rho - alpha Delta (Eq. quasinewton);
      alpha None -> alpha_schedule(||R||).

    Directions and residuals have the shape (nspin, N_g) (a KpointSystem: (N_g,),
    the derivatives by gateaux_kpoints); for a spin pair the inner product sums
    the two channels (Eq. innerproductDirectsumHilbertspace).
    Returns the directions U (r, nspin, N_g), their derivatives T, the
    coefficients a, the rank r, s_rel after each rank, ||R||, alpha, Delta and
    rho_new when rho is given."""
    w = system.w
    Rm = np.asarray(R, dtype=np.float64)
    r_norm = float(np.sqrt(w * np.sum(Rm * Rm)))
    U = [Rm / r_norm]
    T = []
    s_hist = []
    while True:
        T.append(_derivative(system, U[-1]))
        ls = lrdm_apply(Rm, np.stack(U), np.stack(T), w, 0.0, rcond=rcond)
        s_hist.append(ls["s_rel"])
        if ls["s_rel"] < s_tol or len(U) == r_max:
            break
        t = T[-1]
        u = t - sum(w * float(np.sum(t * uk)) * uk for uk in U)
        U.append(u / np.sqrt(w * np.sum(u * u)))
    if alpha is None:
        alpha = alpha_schedule(r_norm)
    out = {"U": np.stack(U), "T": np.stack(T), "a": ls["a"], "rank": len(U), "s_rel": s_hist,
           "r_norm": r_norm, "alpha": alpha, "delta": ls["delta"]}
    if rho is not None:
        out["rho_new"] = np.asarray(rho, dtype=np.float64) - alpha * ls["delta"]
    return out


@dataclasses.dataclass
class LrdmaState:
    """History of the accumulated low-rank approximation (LRDMA, §II.B.1):
    the direction functions U and their Gateaux derivatives T kept since the
    last clearing, the linear prediction of the next residual (Eq.
    linearapprox) and a pending clearing (CT event)."""
    U: list = dataclasses.field(default_factory=list)
    T: list = dataclasses.field(default_factory=list)
    R_lin: Optional[np.ndarray] = None
    clear_next: bool = False


def _orthonormalise(x, U, w):
    """x - sum_k <x, u_k> u_k, normalised (classical Gram-Schmidt, Eq. krylovOrtho)."""
    u = x - sum(w * float(np.sum(x * uk)) * uk for uk in U)
    return u / np.sqrt(w * np.sum(u * u))


def lrdma_step(system: System, state: LrdmaState, R, rho=None, s_tol=0.3, beta_tol=0.1,
               r_norm_clear=1.0, r_max_iter=5, r_max=20, alpha=None, rcond=1e-12):
    """One SCF preconditioning step of the accumulated LRDM (LRDMA, §II.B.1),
    in the order the paper states its decisions:

    1. If a clearing is pending (CT) the history is cleared.  Otherwise, with a
       history, the linearity indicator beta = | ||R_lin|| / ||R|| - 1 | (Eq.
       linearityIndicator; R_lin = R_prev - alpha sum_k a_k t_k, Eq.
       linearapprox) decides: beta > beta_tol clears (CL); else the history's
       own s_rel on R is computed: below s_tol the history is used as it is
       (reuse); else ||R|| > r_norm_clear clears (CR); else the history is
       extended (accumulate).
    2. Without a history (first step or cleared) the rank is built afresh as in
       lrdm_krylov_step (up to r_max).  When accumulating, the first new
       direction is the normalised orthogonal complement of R to the history
       and each next one the Gram-Schmidt of the previous derivative against
       all directions (Eq. accum); at most r_max_iter new ones; if s_rel is
       still >= s_tol the next step clears (CT).
    3. a = S^+ c over all kept derivatives, Delta = sum_k a_k u_k,
       rho_new = rho - alpha Delta (alpha None -> alpha_schedule(||R||)) and
       R_lin = R - alpha sum_k a_k t_k for the next step's beta.
    Returns event ('fresh', 'reuse', 'accumulate', 'CL', 'CR', 'CT'), the
    total and new rank, s_rel, beta, ||R||, alpha, Delta (and rho_new).
    Pinned on an exactly linear residual map (tests/test_lrdma_pins.py): the
    closed forms of beta and of the reused fit, each clearing followed by a
    build equal to lrdm_krylov_step, and the span / orthogonality of the
    accumulated directions, with the CT flag."""
    w = system.w
    Rm = np.asarray(R, dtype=np.float64)
    r_norm = float(np.sqrt(w * np.sum(Rm * Rm)))
    beta = None
    if state.clear_next:
        event = "CT"
    elif state.U:
        beta = abs(float(np.sqrt(w * np.sum(state.R_lin * state.R_lin))) / r_norm - 1.0)
        if beta > beta_tol:
            event = "CL"
        else:
            s_hist = lrdm_apply(Rm, np.stack(state.U), np.stack(state.T), w, 0.0, rcond=rcond)["s_rel"]
            if s_hist < s_tol:
                event = "reuse"
            elif r_norm > r_norm_clear:
                event = "CR"
            else:
                event = "accumulate"
    else:
        event = "fresh"
    if event in ("CT", "CL", "CR"):
        state.U, state.T = [], []
    state.clear_next = False
    n_new = 0
    if event != "reuse":
        fresh = not state.U
        limit = r_max if fresh else max(1, min(r_max_iter, r_max - len(state.U)))
        u = Rm / r_norm if fresh else _orthonormalise(Rm, state.U, w)
        while True:
            state.U.append(u)
            state.T.append(_derivative(system, u))
            n_new += 1
            ls = lrdm_apply(Rm, np.stack(state.U), np.stack(state.T), w, 0.0, rcond=rcond)
            if ls["s_rel"] < s_tol or n_new == limit:
                break
            u = _orthonormalise(state.T[-1], state.U, w)
        if not fresh and ls["s_rel"] >= s_tol:
            state.clear_next = True
    if alpha is None:
        alpha = alpha_schedule(r_norm)
    ls = lrdm_apply(Rm, np.stack(state.U), np.stack(state.T), w, alpha, rcond=rcond,
                    rho=rho if rho is not None else None)
    state.R_lin = Rm - alpha * np.tensordot(ls["a"], np.stack(state.T), axes=1)
    out = {"event": event, "rank": len(state.U), "rank_new": n_new, "s_rel": ls["s_rel"],
           "beta": beta, "r_norm": r_norm, "alpha": alpha, "delta": ls["delta"], "a": ls["a"]}
    if rho is not None:
        out["rho_new"] = ls["rho_new"]
    return out


# ---------------------------------------------------------------------------
# Adjoint of v -> f and of the eigenvalue / occupation inputs
# ---------------------------------------------------------------------------

def backward(system: System, fbar, fwd=None, V=None):
    """Euclidean adjoint (gradients w.r.t. array entries) of the map
    v -> f = g diag(Psi (L o (X(v) - mu'(v) I)) Psi^T) - v, and of L's inputs.

    Steps, each the transpose of one forward step of gateaux():
      Gbar_k   = g Psi^T diag(fbar_k) Psi                 (of density_response)
      Ybar_k   = L o Gbar_k - diag(L) T_k / s,  T_k = sum L_mm Gbar_k,mm,
                 s = sum L_mm (all channels)            (of subspace_response+dmu)
      dVbar_k  = w diag(Psi Ybar_k Psi^T)                 (of project)
      vbar_k   = V_H[sum_s dVbar_k,s] + f_x dVbar_k - fbar_k
                 (of perturbation_potential; the periodic Hartree map is a
                  real symmetric circulant)
    and Lbar = sum_k Gbar_k o (X_k - mu'_k I) - diag(sum_k (T_k/s)(X_k,ii - mu'_k)),
    from which eps_bar (partial at fixed occupations) and occ_bar follow with
    the divided-difference derivatives: for |de| > tau,
    dL_ij/df_i = 1/(eps_i - eps_j), dL_ij/deps_i = -L_ij/(eps_i - eps_j);
    for near-degenerate pairs dL_ij/df_{i,j} = -(1 - 2 fbar)/(2 kT), no eps term;
    dL_ii/df_i = -(1 - 2 f_i)/kT.
    """
    if fwd is None:
        fwd = gateaux(system, V)
    fbar = np.asarray(fbar, dtype=np.float64)
    K = fbar.shape[0]
    ns = system.nspin
    g = system.occ_factor
    w = system.w
    L = fwd["L"]
    fx = fwd["fx"]
    s_sum = sum(float(np.sum(np.diag(Ls))) for Ls in L)
    vbar = np.zeros_like(fbar)
    Lbar = [np.zeros_like(Ls) for Ls in L]
    for k in range(K):
        Gbar = [project(system.psi[s], g * fbar[k, s]) for s in range(ns)]
        T = sum(float(np.dot(np.diag(L[s]), np.diag(Gbar[s]))) for s in range(ns))
        dVbar = []
        for s in range(ns):
            Ybar = L[s] * Gbar[s] - np.diag(np.diag(L[s])) * (T / s_sum)
            dVbar.append(w * np.einsum("ri,ri->r", system.psi[s] @ Ybar, system.psi[s]))
            X = fwd["X"][s][k]
            dmu = fwd["dmu"][k]
            Lbar[s] += Gbar[s] * (X - dmu * np.eye(X.shape[0]))
            Lbar[s] -= np.diag((T / s_sum) * (np.diag(X) - dmu))
        vh = hartree(sum(dVbar), system.n, system.h, system.poisson)
        for s in range(ns):
            vbar[k, s] = vh + fx[s] * dVbar[s] - fbar[k, s]
    occ = _occupations(system, fwd["mu"])
    eps_bar, occ_bar = [], []
    tau = system.degen_tol * system.kT
    for s in range(ns):
        e = np.asarray(system.eps[s], dtype=np.float64)
        f = occ[s]
        de = e[:, None] - e[None, :]
        offd = ~np.eye(len(e), dtype=bool)
        near = (np.abs(de) <= tau) & offd
        far = (np.abs(de) > tau) & offd
        sym = Lbar[s] + Lbar[s].T
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = np.where(far, 1.0 / np.where(far, de, 1.0), 0.0)
        fb = 0.5 * (f[:, None] + f[None, :])
        eb = np.sum(np.where(far, sym * (-L[s] * inv), 0.0), axis=1)
        ob = np.sum(np.where(far, sym * inv, 0.0), axis=1)
        ob += np.sum(np.where(near, sym * (-(1.0 - 2.0 * fb) / (2.0 * system.kT)), 0.0), axis=1)
        ob += np.diag(Lbar[s]) * (-(1.0 - 2.0 * f) / system.kT)
        eps_bar.append(eb)
        occ_bar.append(ob)
    return {"vbar": vbar, "eps_bar": eps_bar, "occ_bar": occ_bar, "Lbar": Lbar}


def total_eps_grad(system: System, eps_bar, occ_bar, mu):
    """Compose the total eps-gradient when occupations are Fermi-Dirac with mu
    fixed by the electron count: f_i = f(eps_i, mu(eps)), dmu/deps_j =
    f'_j / sum f' (from d/deps_j of g sum f = N_e), f' = df/deps."""
    fp = [-fermi(e, mu, system.kT) * (1.0 - fermi(e, mu, system.kT)) / system.kT
          for e in system.eps]
    sfp = sum(float(np.sum(x)) for x in fp)
    proj = sum(float(np.dot(ob, x)) for ob, x in zip(occ_bar, fp))
    return [eb + ob * x - x * proj / sfp for eb, ob, x in zip(eps_bar, occ_bar, fp)]
