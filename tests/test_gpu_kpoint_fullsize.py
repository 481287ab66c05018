"""Parity of the k-point leg at the size the benchmark times it (48^3 grid,
4 k-points x N_s = 512 complex states, K = 8, split-BF16x3 on the stacked
operand; the benchmark's own input generator and seeds).

The oracle cannot run the whole path here in seconds, so the test checks
(a) sampled rows of drho_0 computed in FP64 from the definition
g sum_kappa w_kappa sum_ij psi_i(r) Gamma_ij conj(psi_j(r)) with
X_kappa = Psi_kappa^H diag(w dV_0) Psi_kappa and mu' from the BZ-averaged
traceless condition, dV_0 from the oracle's Hartree and xc kernel on the
device's density; and (b) properties that hold at any size: int drho_k = 0,
<dV_a, drho_b> = <dV_b, drho_a> and <dV_a, drho_a> <= 0.
"""

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kp():
    import bench
    from paper_2211_07894_gb300 import KpContext, build
    build.build()
    rng = workloads.rng_for(80, 0)
    pr, pi = [], []
    for q in range(bench.KP_NK):
        a, b = workloads.random_subspace_complex_torch(bench.KP_GRID, bench.H, bench.KP_NS,
                                                       2211078940 + 80 + q, "cuda")
        pr.append(a)
        pi.append(b)
    eps_h = [workloads.random_eigenvalues(bench.KP_NS, rng) + 0.02 * q for q in range(bench.KP_NK)]
    eps = [torch.as_tensor(e, device="cuda") for e in eps_h]
    kw = bench.kp_weights(bench.KP_NK)
    ctx = KpContext(bench.KP_GRID, bench.H, pr, pi, eps, kw, bench.KP_NE, bench.KP_KT, rho_floor=1e-3,
                    prec="bf16x3", io_dtype=torch.float32, k_max=bench.KP_K)
    V = torch.as_tensor(workloads.smooth_directions(bench.KP_GRID, bench.H, bench.KP_K, 1,
                                                    workloads.rng_for(80, 100))[:, 0],
                        dtype=torch.float32, device="cuda").contiguous()
    F, dmu = ctx.gateaux(V)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    rho = ctx.density().double().cpu().numpy()
    psi = [a.double().cpu().numpy() + 1j * b.double().cpu().numpy() for a, b in zip(pr, pi)]
    Vh = V.double().cpu().numpy()
    fx = oracle.lda_fx(rho)
    dV = np.stack([oracle.perturbation_potential([Vh[k]], [fx], bench.KP_GRID, bench.H)[0]
                   for k in range(bench.KP_K)])
    return dict(psi=psi, eps=eps_h, kw=kw, V=Vh, drho=F.double().cpu().numpy() + Vh, dV=dV,
                dmu=dmu.cpu().numpy(), mu=ctx.mu(), w=float(np.prod(bench.H)), g=2.0, kT=bench.KP_KT)


def test_sampled_response_rows(kp):
    w, g = kp["w"], kp["g"]
    a = w * kp["dV"][0]
    L = [oracle.loewner(e, kp["mu"], kp["kT"]) for e in kp["eps"]]
    X = [p.conj().T @ (a[:, None] * p) for p in kp["psi"]]
    X = [0.5 * (x + x.conj().T) for x in X]
    num = sum(wk * float(np.dot(np.diag(Lk), np.diag(Xk).real)) for wk, Lk, Xk in zip(kp["kw"], L, X))
    den = sum(wk * float(np.sum(np.diag(Lk))) for wk, Lk in zip(kp["kw"], L))
    dmu = num / den
    assert abs(kp["dmu"][0] - dmu) <= 1e-4 * max(abs(float(np.diag(x).real.max())) for x in X)
    rows = workloads.rng_for(80, 200).choice(kp["V"].shape[1], 64, replace=False)
    ref = np.zeros(len(rows))
    for p, wk, Lk, Xk in zip(kp["psi"], kp["kw"], L, X):
        G = Lk * (Xk - dmu * np.eye(Xk.shape[0]))
        ps = p[rows]
        ref += g * wk * np.einsum("ri,ri->r", ps @ G, ps.conj()).real
    got = kp["drho"][0][rows]
    scale = np.sqrt(np.mean(kp["drho"][0] ** 2))
    err = float(np.max(np.abs(got - ref)) / scale)
    print(f"k-point leg, sampled drho rows: max |err| / rms = {err:.2e}")
    assert err < 1e-4


def test_response_properties(kp):
    w = kp["w"]
    drho, dV = kp["drho"], kp["dV"]
    K = drho.shape[0]
    for k in range(K):
        assert abs(w * drho[k].sum()) <= 1e-5 * w * np.abs(drho[k]).sum()
        assert float(np.dot(dV[k], drho[k])) <= 0.0
    M = dV @ drho.T
    sym = np.abs(M - M.T).max() / np.abs(M).max()
    print(f"k-point leg: chi_0 symmetry {sym:.2e}")
    assert sym < 1e-4
