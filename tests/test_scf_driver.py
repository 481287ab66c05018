"""The toy SCF driver's own arithmetic (paper_2211_07894_gb300/scf.py), on the
CPU: the Hamiltonian, Hartree and exchange potentials against the pinned
oracle and a dense matrix; ChFSI against dense diagonalisation (the
Chebyshev-filtered subspace converges to the lowest eigenpairs); the density
and chemical potential; the Kerker filter and Anderson mixing.  The SCF
comparison with the library's LRDM / LRDMA steps is tests/test_gpu_scf.py."""

import numpy as np
import pytest
from scipy.linalg import eigh

import oracle
import workloads

torch = pytest.importorskip("torch")

from paper_2211_07894_gb300 import scf  # noqa: E402


@pytest.fixture(scope="module")
def small():
    n, h = (8, 6, 6), (0.5, 0.5, 0.5)
    v = scf.gaussian_wells(n, h, [(1.0, 1.5, 1.5), (3.0, 1.2, 1.7)], [2.0, 1.5])
    model = scf.KSModel(n, h, v, 4.0, 0.02, 10, device="cpu")
    rho = torch.as_tensor(0.05 + 0.02 * workloads.rng_for(92, 0).random(model.ng))
    return model, rho


def test_potentials_match_oracle(small):
    model, rho = small
    r = rho.numpy()
    assert np.allclose(model.hartree(rho).numpy(), oracle.hartree(r, model.n, model.h), rtol=0, atol=1e-12)
    assert np.allclose(model.vx(rho).numpy(), oracle.lda_vx(r), rtol=1e-14, atol=0)


def test_hamiltonian_matches_dense(small):
    model, rho = small
    veff = model.v_eff(rho)
    H = -0.5 * workloads.fd_laplacian_dense(model.n, model.h) + np.diag(veff.numpy())
    X = torch.as_tensor(workloads.rng_for(92, 1).standard_normal((model.ng, 3)))
    assert np.allclose(model.apply_h(X, veff).numpy(), H @ X.numpy(), rtol=0, atol=1e-11)


def test_chfsi_converges_to_lowest_eigenpairs(small):
    model, rho = small
    veff = model.v_eff(rho)
    H = -0.5 * workloads.fd_laplacian_dense(model.n, model.h) + np.diag(veff.numpy())
    e_ref, v_ref = eigh(H)
    X = scf.initial_subspace(model, seed=3)
    eps, Psi, _ = model.chfsi(X, veff, degree=16, passes=25)
    ns = model.ns
    # the 8 lowest (well separated from the subspace's top) converge fully
    assert np.max(np.abs(eps.numpy()[:8] - e_ref[:8])) < 1e-12
    P = Psi.numpy()
    assert np.max(np.abs(model.w * P.T @ P - np.eye(ns))) < 1e-12        # w-orthonormal
    # span: the lowest 8 eigenvectors lie in span(Psi) (vectors converge as the
    # square root of the eigenvalue error)
    Vl = v_ref[:, :8]
    Q = P * np.sqrt(model.w)
    assert np.linalg.norm(Vl - Q @ (Q.T @ Vl)) < 1e-6


def test_density_and_chemical_potential(small):
    model, rho = small
    eps = torch.as_tensor(np.sort(workloads.rng_for(92, 2).uniform(-1, 0.5, model.ns)))
    Psi = model.orthonormalise(torch.as_tensor(workloads.rng_for(92, 3).standard_normal((model.ng, model.ns))))
    rho_out, mu = model.density(Psi, eps)
    mu_ref = oracle.solve_mu([eps.numpy()], model.ne, model.kT, 2.0)
    assert abs(mu - mu_ref) < 1e-10
    ref = oracle.density(Psi.numpy(), oracle.fermi(eps.numpy(), mu_ref, model.kT), 2.0)
    assert np.allclose(rho_out.numpy(), ref, rtol=1e-9, atol=1e-14)
    assert abs(model.w * float(rho_out.sum()) - model.ne) < 1e-9


def test_kerker_and_anderson(small):
    model, rho = small
    R = torch.as_tensor(workloads.smooth_field(model.n, model.h, 0.1, workloads.rng_for(92, 4)))
    K = model.kerker(R, 1.0)
    # G = 0 removed, every other plane wave scaled by |G|^2 / (|G|^2 + q0^2) < 1
    assert abs(float(K.sum())) < 1e-12 * float(R.abs().sum())
    assert model.norm(K) < model.norm(R)
    # Anderson with one pair is Kerker mixing
    a = scf.AndersonKerkerMixer(alpha=0.5, q0=1.0, m=4)
    k = scf.KerkerMixer(alpha=0.5, q0=1.0)
    r1, _ = a.step(model, rho, R, None, None)
    r2, _ = k.step(model, rho, R, None, None)
    assert torch.allclose(r1, r2, rtol=0, atol=1e-15)
    # with a second pair, the mixed residual is the minimum-norm affine combination
    R2 = 0.5 * R + 0.01
    _, info = a.step(model, rho + 0.01, R2, None, None)
    c = info["coeff"].numpy()
    assert abs(c.sum() - 1.0) < 1e-14
    mix = c[0] * R.numpy() + c[1] * R2.numpy()
    for s in np.linspace(-1, 2, 13):
        other = s * R.numpy() + (1 - s) * R2.numpy()
        assert np.linalg.norm(mix) <= np.linalg.norm(other) + 1e-12


def test_scf_with_fixed_mixers_converges(small):
    """The SCF loop with Kerker and Anderson-Kerker mixing converges on the
    small model (the library's LRDM steps need a GPU)."""
    model, _ = small
    rho0 = torch.full((model.ng,), model.ne / (model.ng * model.w), dtype=torch.float64)
    res = scf.compare(model, rho0, [scf.KerkerMixer(0.5, 1.0), scf.AndersonKerkerMixer(0.5, 1.0)],
                      tol=1e-7, max_iter=120)
    for r in res.values():
        assert r.converged, (r.mixer, r.residual_norms[-3:])
