"""Toy self-consistent Kohn-Sham driver: the LRDM preconditioner (§II.B) and its
accumulated variant (§II.B.1) inside an SCF loop whose subspace comes from
Chebyshev-filtered subspace iteration (ChFSI, §II.C), against simple, Kerker
and Anderson-Kerker mixing.  It demonstrates the library in the setting the
paper uses it; the Kohn-Sham model itself is a small finite-difference model,
not the paper's finite-element DFT.

Model (spin-restricted, atomic units): a periodic n0 x n1 x n2 grid with
spacing h, quadrature weight w = h0 h1 h2, and
    H[rho] = -1/2 Lap_FD + V_ext + V_H[rho] + V_x[rho]
with the second-order finite-difference Laplacian, the spectral Hartree
potential 4 pi / |G|^2 (G = 0 dropped) and LDA exchange
V_x = -(3/pi)^(1/3) rho^(1/3).  The fixed-point map is
rho_out = 2 sum_i f(eps_i, mu) psi_i^2 with Fermi-Dirac occupations and mu from
the electron count (Eq. kseqcont), its residual R[rho] = rho_out - rho.

Eigen-solver: one or more ChFSI passes per SCF step on the current subspace
X (N_g x N_s): a degree-m Chebyshev filter of H that damps the unwanted
interval [a, b] (the scaled three-term recurrence of Zhou and Saad, 2007),
w-orthonormalisation by Householder QR, and Rayleigh-Ritz on the N_s x N_s
projected Hamiltonian, whose eigenpairs are the subspace (Psi, eps) handed
to the library (Psi^T diag(w) Psi = I).

Mixers (rho_new from rho and R):
  simple          rho + alpha R
  kerker          rho + alpha F^-1[ |G|^2 / (|G|^2 + q0^2) F[R] ]
  anderson        Anderson mixing over the last m pairs (rho_i, R_i), with the
                  Kerker preconditioner on the mixed residual
  lrdm            lrdm_krylov_step (adaptive rank, s_tol, the paper's alpha
                  schedule 0.1 / 0.5 at ||R|| = 2)
  lrdma           lrdm_lrdma_step (beta_tol 0.1, r_max_iter 5, accumulation
                  only below ||R|| = 1)
The last two build a library context for every SCF step, since every step
has its own subspace.  All model arithmetic runs in torch on the given device.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np


def gaussian_wells(n, h, centres, depths, width=1.0):
    """V_ext(r) = -sum_a D_a exp(-d_min(r, R_a)^2 / (2 width^2)) on the periodic
    grid (minimum-image distances); centres in bohr, depths in Ha."""
    L = [n[d] * h[d] for d in range(3)]
    axes = [np.arange(n[d]) * h[d] for d in range(3)]
    X = np.meshgrid(*axes, indexing="ij")
    v = np.zeros(n)
    for c, D in zip(centres, depths):
        d2 = np.zeros(n)
        for d in range(3):
            dx = X[d] - c[d]
            dx -= L[d] * np.round(dx / L[d])
            d2 += dx * dx
        v -= D * np.exp(-d2 / (2.0 * width * width))
    return v.reshape(-1)


class KSModel:
    def __init__(self, n, h, v_ext, n_electrons, kT, ns, device="cuda", rho_floor=1e-12):
        import torch
        self.torch = torch
        self.n, self.h = tuple(int(x) for x in n), tuple(float(x) for x in h)
        self.ng = int(np.prod(self.n))
        self.w = float(np.prod(self.h))
        self.ne, self.kT, self.ns, self.g = float(n_electrons), float(kT), int(ns), 2.0
        self.device = device
        self.rho_floor = rho_floor
        dt = torch.float64
        self.v_ext = torch.as_tensor(np.asarray(v_ext, dtype=np.float64), device=device)
        # |G|^2 on the half-complex grid of rfftn
        ks = [2 * math.pi * torch.fft.fftfreq(self.n[d], d=self.h[d], dtype=dt, device=device)
              for d in range(2)]
        k2 = 2 * math.pi * torch.fft.rfftfreq(self.n[2], d=self.h[2], dtype=dt, device=device)
        G2 = ks[0][:, None, None] ** 2 + ks[1][None, :, None] ** 2 + k2[None, None, :] ** 2
        self.G2 = G2
        sym = torch.zeros_like(G2)
        nz = G2 > 0
        sym[nz] = 4 * math.pi / G2[nz]
        self.hartree_symbol = sym
        self.lap_max = sum(4.0 / (x * x) for x in self.h)      # ||Lap_FD|| (its largest |eigenvalue|)

    # ---- potentials ----------------------------------------------------------------
    def hartree(self, rho):
        torch = self.torch
        r = rho.reshape(self.n)
        return torch.fft.irfftn(torch.fft.rfftn(r) * self.hartree_symbol, s=self.n).reshape(-1)

    def vx(self, rho):
        return -((3.0 / math.pi) ** (1.0 / 3.0)) * self.torch.clamp(rho, min=self.rho_floor) ** (1.0 / 3.0)

    def v_eff(self, rho):
        return self.v_ext + self.hartree(rho) + self.vx(rho)

    # ---- Hamiltonian ---------------------------------------------------------------
    def apply_h(self, X, veff):
        """H X for X of shape (N_g, m): -1/2 Lap_FD X + veff X."""
        torch = self.torch
        m = X.shape[1]
        Y = X.reshape(self.n + (m,))
        lap = torch.zeros_like(Y)
        for d in range(3):
            lap += (torch.roll(Y, 1, dims=d) + torch.roll(Y, -1, dims=d) - 2.0 * Y) / (self.h[d] ** 2)
        return (-0.5 * lap).reshape(self.ng, m) + veff[:, None] * X

    def chebyshev_filter(self, X, veff, degree, a, b, a0):
        """T_m of H scaled so that [a, b] maps to [-1, 1], applied to X with the
        scaling that keeps the columns near unit size (a0 <= lowest eigenvalue)."""
        e = 0.5 * (b - a)
        c = 0.5 * (b + a)
        sigma = e / (a0 - c)
        tau = 2.0 / sigma
        Y = (self.apply_h(X, veff) - c * X) * (sigma / e)
        for _ in range(2, degree + 1):
            sigma_new = 1.0 / (tau - sigma)
            Y_new = (self.apply_h(Y, veff) - c * Y) * (2.0 * sigma_new / e) - (sigma * sigma_new) * X
            X, Y, sigma = Y, Y_new, sigma_new
        return Y

    def orthonormalise(self, X):
        """w-orthonormal basis of span(X): Householder QR of sqrt(w) X (the
        filtered columns can be nearly dependent, which Cholesky-QR would not
        survive), X -> Q / sqrt(w)."""
        Q, _ = self.torch.linalg.qr(X * math.sqrt(self.w), mode="reduced")
        return Q / math.sqrt(self.w)

    def rayleigh_ritz(self, X, veff):
        torch = self.torch
        Hs = self.w * (X.T @ self.apply_h(X, veff))
        eps, Q = torch.linalg.eigh(0.5 * (Hs + Hs.T))
        return eps, X @ Q

    def chfsi(self, X, veff, degree=16, passes=1, bounds=None):
        """ChFSI passes on the subspace X; returns (eps, Psi) of the last
        Rayleigh-Ritz step and the bounds used.  bounds = (a0, a): the lowest
        eigenvalue estimate and the top of the wanted interval (the largest
        Ritz value of the previous step); b bounds the spectrum from above."""
        b = 0.5 * self.lap_max + float(veff.max()) + 1e-3
        if bounds is None:
            eps, Psi = self.rayleigh_ritz(self.orthonormalise(X), veff)
            bounds = (float(eps[0]), float(eps[-1]))
        a0, a = bounds
        for _ in range(passes):
            Y = self.chebyshev_filter(X, veff, degree, a, b, a0 - 1e-3 * (b - a0))
            eps, Psi = self.rayleigh_ritz(self.orthonormalise(Y), veff)
            a0, a = float(eps[0]), float(eps[-1])
            X = Psi
        return eps, Psi, (a0, a)

    # ---- density ---------------------------------------------------------------------
    def fermi(self, eps, mu):
        return self.torch.special.expit(-(eps - mu) / self.kT)

    def chemical_potential(self, eps):
        """mu with g sum_i f(eps_i, mu) = N_e (bisection)."""
        lo = float(eps.min()) - 50 * self.kT
        hi = float(eps.max()) + 50 * self.kT
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if self.g * float(self.fermi(eps, mid).sum()) > self.ne:
                hi = mid
            else:
                lo = mid
        return 0.5 * (lo + hi)

    def density(self, Psi, eps):
        mu = self.chemical_potential(eps)
        return self.g * (Psi * Psi) @ self.fermi(eps, mu), mu

    def norm(self, x):
        return math.sqrt(self.w * float((x * x).sum()))

    def kerker(self, R, q0):
        torch = self.torch
        F = torch.fft.rfftn(R.reshape(self.n))
        return torch.fft.irfftn(F * (self.G2 / (self.G2 + q0 * q0)), s=self.n).reshape(-1)


# ---------------------------------------------------------------------------------------
# mixers
# ---------------------------------------------------------------------------------------

class SimpleMixer:
    name = "simple"

    def __init__(self, alpha=0.3):
        self.alpha = alpha

    def step(self, model, rho, R, Psi, eps):
        return rho + self.alpha * R, {}


class KerkerMixer:
    name = "kerker"

    def __init__(self, alpha=0.5, q0=1.0):
        self.alpha, self.q0 = alpha, q0

    def step(self, model, rho, R, Psi, eps):
        return rho + self.alpha * model.kerker(R, self.q0), {}


class AndersonKerkerMixer:
    """Anderson mixing of the last m (rho, R) pairs: coefficients c (sum 1)
    minimising ||sum_i c_i R_i||_w, then rho = sum_i c_i (rho_i + alpha K R_i)
    with K the Kerker preconditioner."""
    name = "anderson"

    def __init__(self, alpha=0.5, q0=1.0, m=6):
        self.alpha, self.q0, self.m = alpha, q0, m
        self.rhos: List = []
        self.res: List = []

    def step(self, model, rho, R, Psi, eps):
        torch = model.torch
        self.rhos.append(rho.clone())
        self.res.append(R.clone())
        self.rhos, self.res = self.rhos[-self.m:], self.res[-self.m:]
        k = len(self.res)
        if k == 1:
            c = torch.ones(1, dtype=rho.dtype, device=rho.device)
        else:
            # differences to the newest pair: min ||R_k + sum_j t_j (R_j - R_k)||
            D = torch.stack([r - self.res[-1] for r in self.res[:-1]], dim=1)
            A = model.w * (D.T @ D)
            bvec = -model.w * (D.T @ self.res[-1])
            t = torch.linalg.lstsq(A + 1e-12 * torch.trace(A) * torch.eye(k - 1, dtype=A.dtype,
                                                                              device=A.device), bvec).solution
            c = torch.cat([t, (1.0 - t.sum())[None]])
        rho_bar = sum(ci * r for ci, r in zip(c, self.rhos))
        R_bar = sum(ci * r for ci, r in zip(c, self.res))
        return rho_bar + self.alpha * model.kerker(R_bar, self.q0), {"coeff": c}


class LrdmMixer:
    """The LRDM step of the library (lrdm_krylov_step) on the step's subspace."""
    name = "lrdm"

    def __init__(self, prec="fp64", s_tol=0.3, r_max=20, alpha=-1.0):
        self.prec, self.s_tol, self.r_max, self.alpha = prec, s_tol, r_max, alpha

    def _context(self, model, rho, Psi, eps):
        import torch
        from .binding import Context
        io = torch.float64 if self.prec == "fp64" else torch.float32
        d = dict(n=model.n, h=model.h, psi=[Psi.to(io).contiguous()], eps=[eps.contiguous()],
                 rho=[rho.to(io).contiguous()], n_electrons=model.ne, kT=model.kT, g=model.g,
                 rho_floor=0.0, k_max=1)
        return Context([d], prec=self.prec, io_dtype=io, k_max=1), io

    def step(self, model, rho, R, Psi, eps):
        ctx, io = self._context(model, rho, Psi, eps)
        r = rho.to(io)[None].contiguous()
        out = ctx.krylov_step(R.to(io)[None].contiguous(), s_tol=self.s_tol, r_max=self.r_max,
                              alpha=self.alpha, rho=r)
        ctx.close()
        return r[0].to(rho.dtype), {"rank": out["rank"], "gateaux": out["rank"]}


class LrdmaMixer(LrdmMixer):
    """The accumulated LRDM step of the library (lrdm_lrdma_step)."""
    name = "lrdma"

    def __init__(self, prec="fp64", capacity=32, **params):
        super().__init__(prec=prec)
        self.capacity, self.params, self.hist = capacity, params, None

    def step(self, model, rho, R, Psi, eps):
        from .binding import Lrdma
        ctx, io = self._context(model, rho, Psi, eps)
        if self.hist is None:
            self.hist = Lrdma(model.ng, io, model.w, capacity=self.capacity)
        r = rho.to(io)[None].contiguous()
        rep = self.hist.step(ctx, R.to(io)[None].contiguous(), r, r_max=self.capacity, **self.params)
        ctx.close()
        return r[0].to(rho.dtype), {"rank": rep["rank"], "gateaux": rep["rank_new"], "event": rep["event"]}


# ---------------------------------------------------------------------------------------
# the SCF loop
# ---------------------------------------------------------------------------------------

@dataclass
class ScfResult:
    mixer: str
    converged: bool
    iterations: int
    residual_norms: List[float] = field(default_factory=list)
    gateaux: int = 0
    events: List[str] = field(default_factory=list)


def initial_subspace(model, seed=0):
    """Seeded random starting columns (run_scf filters them with its first
    step's ChFSI passes)."""
    torch = model.torch
    gen = torch.Generator(device="cpu")
    gen.manual_seed(int(seed))
    X = torch.randn(model.ng, model.ns, generator=gen, dtype=torch.float64).to(model.device)
    return X


def run_scf(model, mixer, rho0, X0, tol=1e-5, max_iter=100, degree=16, passes=1, warm_passes=8,
            diverge=1e3):
    """SCF iterations rho -> mixer(rho, R[rho]) until ||R||_w < tol; each
    step runs `passes` ChFSI passes on the subspace carried over from the
    previous step (the first step `warm_passes`)."""
    rho = rho0.clone()
    X = X0.clone()
    bounds = None
    res = ScfResult(mixer.name, False, 0)
    for it in range(max_iter):
        veff = model.v_eff(rho)
        eps, Psi, bounds = model.chfsi(X, veff, degree=degree, passes=warm_passes if it == 0 else passes,
                                       bounds=bounds)
        X = Psi
        rho_out, _ = model.density(Psi, eps)
        R = rho_out - rho
        rn = model.norm(R)
        res.residual_norms.append(rn)
        res.iterations = it
        if rn < tol:
            res.converged = True
            return res
        if not math.isfinite(rn) or rn > diverge:
            return res
        rho, info = mixer.step(model, rho, R, Psi, eps)
        res.gateaux += int(info.get("gateaux", 0))
        if "event" in info:
            res.events.append(info["event"])
    res.iterations = max_iter
    return res


def sloshing_model(device="cuda", n=(64, 6, 6), h=(0.5, 0.5, 0.5), wells=16, n_electrons=24.0,
                   kT=0.01, ns=28, seed=7):
    """An elongated cell (32 x 3 x 3 bohr) holding a chain of 16 Gaussian
    wells along x with varying spacing and depths (1-3 Ha) and 24 electrons:
    a metallic-like chain whose charge sloshes along the long axis.  N_s = 28
    states (12 occupied plus buffer states).  Start: the uniform density."""
    rng = np.random.default_rng(2211078940 + seed)
    Lx = n[0] * h[0]
    xs = (np.arange(wells) + 0.5) * Lx / wells + rng.uniform(-0.3, 0.3, wells)
    centres = [(x, 0.5 * n[1] * h[1] + rng.uniform(-0.2, 0.2), 0.5 * n[2] * h[2] + rng.uniform(-0.2, 0.2))
               for x in xs]
    depths = rng.uniform(1.0, 3.0, wells)
    v = gaussian_wells(n, h, centres, depths)
    model = KSModel(n, h, v, n_electrons, kT, ns, device=device)
    # starting density: uniform with the right electron count
    import torch
    rho0 = torch.full((model.ng,), n_electrons / (model.ng * model.w), dtype=torch.float64, device=device)
    return model, rho0


def compare(model, rho0, mixers, tol=1e-5, max_iter=100, seed=0, **kw) -> Dict[str, ScfResult]:
    """SCF iteration counts of several mixers from the same start."""
    X0 = initial_subspace(model, seed=seed)
    return {m.name: run_scf(model, m, rho0, X0, tol=tol, max_iter=max_iter, **kw) for m in mixers}
