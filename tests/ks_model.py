"""A tiny full-space Kohn-Sham model for SCF-level tests: the fixed-point map
F[rho] by dense diagonalisation of H = -1/2 Lap_FD + V_ext + V_H[rho] + V_x[rho]
(Eq. kseqcont) on a small periodic grid, with the lowest N_s eigenpairs as the
subspace of the response (the role the Chebyshev-filtered subspace plays in
the paper, occupied plus buffer states)."""

from __future__ import annotations

import numpy as np
from scipy.linalg import eigh

import oracle
import workloads


def scf_map(n, h, vext, lap, rho_channels, n_e, kT, g):
    """F[rho] per channel, all eigenvalues and eigenvectors (psi = v / sqrt(w))."""
    w = float(np.prod(h))
    nspin = len(rho_channels)
    vh = oracle.hartree(sum(rho_channels), n, h)
    eps, psi = [], []
    for s in range(nspin):
        veff = vext + vh + oracle.lda_vx(rho_channels[s], spin_polarized=(nspin == 2))
        H = -0.5 * lap + np.diag(veff)
        e, v = eigh(H)
        eps.append(e)
        psi.append(v / np.sqrt(w))
    mu = oracle.solve_mu(eps, n_e, kT, g)
    out = [oracle.density(p, oracle.fermi(e, mu, kT), g) for p, e in zip(psi, eps)]
    return out, eps, psi


class TinyModel:
    """Gaussian wells on an n^3 grid, restricted (g = 2)."""

    def __init__(self, n=(6, 6, 6), h=(0.5, 0.5, 0.5), wells=3, n_e=8.0, kT=0.05, ns=24, seed=0):
        self.n, self.h = tuple(n), tuple(h)
        rng = workloads.rng_for(91, seed)
        self.vext = workloads.gaussian_wells(self.n, self.h, wells, rng)
        self.lap = workloads.fd_laplacian_dense(self.n, self.h)
        self.w = float(np.prod(self.h))
        self.n_e, self.kT, self.ns, self.g = n_e, kT, ns, 2.0
        e0, p0 = workloads.lowest_eigenpairs(workloads.toy_hamiltonian(self.n, self.h, self.vext), ns,
                                             self.w)
        occ = oracle.fermi(e0, oracle.solve_mu([e0], n_e, kT, 2.0), kT)
        # a deliberately poor start: the non-interacting density, smoothed toward uniform
        rho = 2.0 * (p0 ** 2) @ occ
        self.rho0 = 0.5 * rho + 0.5 * rho.mean()

    def residual(self, rho):
        """R = F[rho] - rho and the subspace system at rho (oracle.System)."""
        out, eps, psi = scf_map(self.n, self.h, self.vext, self.lap, [rho], self.n_e, self.kT, self.g)
        sysm = oracle.System(n=self.n, h=self.h, psi=[psi[0][:, :self.ns]], eps=[eps[0][:self.ns]],
                             rho=[rho], n_electrons=self.n_e, kT=self.kT, g=self.g)
        return out[0] - rho, sysm

    def norm(self, x):
        return float(np.sqrt(self.w * np.sum(np.asarray(x) ** 2)))
