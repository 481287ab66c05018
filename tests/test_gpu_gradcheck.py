"""Finite-difference check of the hand-written adjoint on the GPU, FP64 path.

The loss J(v, eps, occ) = sum_k <fbar_k, f_k> (Euclidean) is evaluated by the
library's own FP64 forward (lrdm_gateaux_batch) with the occupations and the
density given, so that eps and occ enter only through the Loewner matrix
L(eps, occ) and v only through dV -- the inputs lrdm_backward differentiates.
Along 8 seeded probe directions (q_v, q_eps, q_occ) the central difference
(eta = 1e-4 of the probe scale, one Richardson step) must match
<vbar, q_v> + <eps_bar, q_eps> + <occ_bar, q_occ> from one backward call.
L_ij = (f_i - f_j) / (eps_i - eps_j) is a rational function of the gaps, so
the eigenvalue probe is scaled to move eigenvalues by at most ~1 % of the
smallest gap (1.7e-5 Ha here) per step; with steps of kT size the difference
quotient itself is off by up to 1e-4 (the FP64 oracle shows the same).
"""

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N = (20, 18, 16)
NS, K, NE, KT = 96, 3, 70.0, 0.01
ETA = 1e-4
PROBES = 8


@pytest.fixture(scope="module")
def setup():
    from paper_2211_07894_gb300 import build
    build.build()
    cfg = workloads.random_system(30, N, NS, NE, KT, K)
    eps = cfg["eps"][0]
    mu = oracle.solve_mu([eps], NE, KT, 2.0)
    occ = oracle.fermi(eps, mu, KT)
    rho = oracle.density(cfg["psi"][0], occ, 2.0, 1e-3)
    rng = workloads.rng_for(30, 7)
    fbar = rng.standard_normal(cfg["V"].shape)
    return cfg, eps, occ, rho, fbar


def _context(cfg, eps, occ, rho):
    from gpu_helpers import to_device_system
    from paper_2211_07894_gb300 import Context
    c = dict(cfg)
    c["eps"] = [eps]
    c["occ"] = [occ]
    d = to_device_system(c, torch.float64, pass_rho=[rho])
    return Context([d], prec="fp64", io_dtype=torch.float64, k_max=K)


def _loss(cfg, eps, occ, rho, V, fbar):
    ctx = _context(cfg, eps, occ, rho)
    (F,), _ = ctx.gateaux([torch.as_tensor(V, device="cuda")])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    J = float(np.sum(F.cpu().numpy() * fbar))
    ctx.close()
    return J


def test_adjoint_against_central_differences(setup):
    cfg, eps, occ, rho, fbar = setup
    V = cfg["V"]
    ctx = _context(cfg, eps, occ, rho)
    ctx.gateaux([torch.as_tensor(V, device="cuda")])
    vbar, eb, ob = ctx.backward([torch.as_tensor(fbar, device="cuda")])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    vbar = vbar[0].cpu().numpy()
    eb = eb[0].cpu().numpy()
    ob = ob[0].cpu().numpy()
    rng = workloads.rng_for(30, 8)
    gmin = float(np.diff(np.sort(eps)).min())
    worst = 0.0
    for p in range(PROBES):
        qv = workloads.smooth_directions(N, cfg["h"], K, 1, rng)
        qe = min(KT, 0.01 * gmin / ETA) * rng.standard_normal(NS)
        qo = 0.01 * rng.standard_normal(NS)
        pred = float(np.sum(vbar * qv) + eb @ qe + ob @ qo)

        def D(eta):
            jp = _loss(cfg, eps + eta * qe, occ + eta * qo, rho, V + eta * qv, fbar)
            jm = _loss(cfg, eps - eta * qe, occ - eta * qo, rho, V - eta * qv, fbar)
            return (jp - jm) / (2 * eta)

        fd = (4 * D(ETA / 2) - D(ETA)) / 3
        err = abs(fd - pred) / max(abs(pred), 1e-30)
        worst = max(worst, err)
    print(f"GPU FP64 adjoint vs central differences, {PROBES} probes: max rel err {worst:.2e}")
    assert worst < 1e-6


# --- at scale: 48^3 grid, N_s = 4096, K = 1 (FP64 path) ----------------------

N48 = (48, 48, 48)
NS48, NE48, KT48 = 4096, 3700.0, 0.005


@pytest.fixture(scope="module")
def setup48():
    from paper_2211_07894_gb300 import build
    build.build()
    h = (0.5, 0.5, 0.5)
    psi = workloads.random_subspace_torch(N48, h, NS48, seed=2211078940 + 57, device="cuda",
                                          dtype=torch.float64)
    eps = workloads.random_eigenvalues(NS48, workloads.rng_for(57, 0))
    mu = oracle.solve_mu([eps], NE48, KT48, 2.0)
    occ = oracle.fermi(eps, mu, KT48)
    # density from the occupations, on the device (g sum f psi^2 + floor)
    rho = (2.0 * (psi * psi) @ torch.as_tensor(occ, device="cuda") + 1e-3).cpu().numpy()
    V = workloads.smooth_directions(N48, h, 1, 1, workloads.rng_for(57, 1))
    fbar = workloads.rng_for(57, 2).standard_normal(V.shape)
    return dict(psi=psi, h=h, eps=eps, occ=occ, rho=rho, V=V, fbar=fbar)


def _context48(s, eps, occ):
    from paper_2211_07894_gb300 import Context
    d = dict(n=N48, h=s["h"], psi=[s["psi"]], eps=[torch.as_tensor(eps, device="cuda")],
             occ=[torch.as_tensor(occ, device="cuda")], rho=[torch.as_tensor(s["rho"], device="cuda")],
             n_electrons=NE48, kT=KT48, g=2.0, rho_floor=0.0, k_max=1)
    return Context([d], prec="fp64", io_dtype=torch.float64, k_max=1)


def _loss48(s, eps, occ, V):
    ctx = _context48(s, eps, occ)
    (F,), _ = ctx.gateaux([torch.as_tensor(V, device="cuda")])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    J = float(np.sum(F.cpu().numpy() * s["fbar"]))
    ctx.close()
    return J


def test_adjoint_central_differences_at_scale(setup48):
    """lrdm_backward at 48^3 / N_s = 4096 (K = 1, FP64) against central
    differences of the library's own forward, eta = 1e-4, along 8 seeded
    probes of one kind each: 3 in v and 2 in the occupations (f is linear in
    both, so the plain central difference is exact up to rounding) and 3 in
    the eigenvalues at fixed occupations (scaled to move each eigenvalue by at
    most 1 % of the smallest gap per step, with one Richardson step)."""
    s = setup48
    ctx = _context48(s, s["eps"], s["occ"])
    ctx.gateaux([torch.as_tensor(s["V"], device="cuda")])
    vbar, eb, ob = ctx.backward([torch.as_tensor(s["fbar"], device="cuda")])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    vbar, eb, ob = vbar[0].cpu().numpy(), eb[0].cpu().numpy(), ob[0].cpu().numpy()
    ctx.close()
    rng = workloads.rng_for(57, 3)
    gmin = float(np.diff(np.sort(s["eps"])).min())
    zero_e, zero_o, zero_v = np.zeros(NS48), np.zeros(NS48), np.zeros_like(s["V"])
    worst = {}
    for p, kind in enumerate(["v", "v", "v", "eps", "eps", "eps", "occ", "occ"]):
        qv, qe, qo = zero_v, zero_e, zero_o
        if kind == "v":
            qv = workloads.smooth_directions(N48, s["h"], 1, 1, rng)
            pred = float(np.sum(vbar * qv))
        elif kind == "eps":
            qe = 0.01 * gmin / ETA * rng.standard_normal(NS48)
            pred = float(eb @ qe)
        else:
            qo = 0.01 * rng.standard_normal(NS48)
            pred = float(ob @ qo)

        def D(eta):
            jp = _loss48(s, s["eps"] + eta * qe, s["occ"] + eta * qo, s["V"] + eta * qv)
            jm = _loss48(s, s["eps"] - eta * qe, s["occ"] - eta * qo, s["V"] - eta * qv)
            return (jp - jm) / (2 * eta)

        fd = (4 * D(ETA / 2) - D(ETA)) / 3 if kind == "eps" else D(ETA)
        err = abs(fd - pred) / max(abs(pred), 1e-30)
        worst[kind] = max(worst.get(kind, 0.0), err)
        print(f"probe {p} ({kind}): predicted {pred:.10e}, central difference {fd:.10e}, rel {err:.2e}")
    print(f"48^3 / 4096 FP64 adjoint vs central differences: {worst}")
    assert max(worst.values()) < 1e-6
