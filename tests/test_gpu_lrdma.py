"""The accumulated LRDM driver (lrdm_lrdma_step, §II.B.1) on the GPU against
the oracle's LRDMA step, along the oracle's own SCF trajectory on the
elongated sloshing model of test_scf_lrdm (FP64): at every step the same
event (fresh / reuse / accumulate / CL / CR / CT), the same kept and new
rank, and the same density update."""

import numpy as np
import pytest

import oracle
from ks_model import TinyModel

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_lrdma_driver_follows_oracle():
    from gpu_helpers import to_device_system
    from paper_2211_07894_gb300 import Context, Lrdma, build
    build.build()
    model = TinyModel(n=(32, 4, 4), n_e=16.0, kT=0.02, ns=40, wells=6, seed=1)
    gpu = Lrdma(int(np.prod(model.n)), torch.float64, model.w, capacity=16)
    state = oracle.LrdmaState()
    rho = model.rho0.copy()
    events, worst = [], 0.0
    for it in range(40):
        R, sysm = model.residual(rho)
        if model.norm(R) < 1e-8:
            break
        ref = oracle.lrdma_step(sysm, state, R[None], rho=rho[None], r_max=16)
        cfg = dict(n=model.n, h=model.h, psi=sysm.psi, eps=sysm.eps, n_electrons=model.n_e,
                   kT=model.kT, g=model.g, rho_floor=0.0, V=np.zeros((1, 1, 1)))
        ctx = Context([to_device_system(cfg, torch.float64, k_max=1, pass_rho=[rho])],
                      prec="fp64", io_dtype=torch.float64, k_max=1)
        rho_d = torch.as_tensor(rho[None], device="cuda").contiguous()
        rep = gpu.step(ctx, torch.as_tensor(R[None], device="cuda").contiguous(), rho_d, r_max=16)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        assert rep["event"] == ref["event"], (it, rep, ref["event"])
        assert (rep["rank"], rep["rank_new"]) == (ref["rank"], ref["rank_new"])
        assert abs(rep["s_rel"] - ref["s_rel"]) <= 1e-9 * max(ref["s_rel"], 1e-3)
        d_gpu = rho_d.cpu().numpy()[0] - rho
        d_ref = ref["rho_new"][0] - rho
        worst = max(worst, float(np.linalg.norm(d_gpu - d_ref) / np.linalg.norm(d_ref)))
        events.append(rep["event"])
        ctx.close()
        rho = ref["rho_new"][0]
    print(f"LRDMA driver vs oracle over {len(events)} SCF steps: max rel update diff {worst:.2e}; "
          f"events {events}")
    assert worst < 1e-9
    assert "reuse" in events and "accumulate" in events


def test_lrdma_history_checkpoint_resume(tmp_path):
    """The LRDMA history saved after three SCF steps (lrdm_lrdma_export) and
    restored into a new object (lrdm_lrdma_import) continues exactly as the
    original: same events, ranks and bit-identical density updates."""
    from gpu_helpers import to_device_system
    from paper_2211_07894_gb300 import Context, Lrdma, build
    build.build()
    model = TinyModel(n=(32, 4, 4), n_e=16.0, kT=0.02, ns=40, wells=6, seed=1)
    n = int(np.prod(model.n))
    a = Lrdma(n, torch.float64, model.w, capacity=16)
    rho = model.rho0.copy()

    def step(obj, rho):
        R, sysm = model.residual(rho)
        cfg = dict(n=model.n, h=model.h, psi=sysm.psi, eps=sysm.eps, n_electrons=model.n_e,
                   kT=model.kT, g=model.g, rho_floor=0.0, V=np.zeros((1, 1, 1)))
        ctx = Context([to_device_system(cfg, torch.float64, k_max=1, pass_rho=[rho])],
                      prec="fp64", io_dtype=torch.float64, k_max=1)
        rho_d = torch.as_tensor(rho[None], device="cuda").contiguous()
        rep = obj.step(ctx, torch.as_tensor(R[None], device="cuda").contiguous(), rho_d, r_max=16)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        ctx.close()
        return rep, rho_d.cpu().numpy()[0]

    for _ in range(3):
        _, rho = step(a, rho)
    path = str(tmp_path / "lrdma.npz")
    a.save(path)
    b = Lrdma(n, torch.float64, model.w, capacity=16)
    b.load(path)
    ra, rb = rho.copy(), rho.copy()
    for _ in range(3):
        rep_a, ra = step(a, ra)
        rep_b, rb = step(b, rb)
        assert rep_a == rep_b
        assert np.array_equal(ra, rb)
    a.close()
    b.close()


def test_lrdma_driver_closed_forms_on_linear_map(tmp_path):
    """The device driver's decisions on an exactly linear residual map (one
    fixed FP64 context, next residuals built from the driver's own linear
    prediction R_lin, read back by lrdm_lrdma_export), against the closed
    forms that pin the oracle's step: c R_lin gives beta = |1/c - 1| and a CL
    rebuild equal to a fresh step; R_lin gives beta = 0, the history's fit
    s / sqrt(s^2 + (1 - alpha)^2 (1 - s^2)) and the reused step
    (1 - alpha) Delta; alpha = 1 leaves nothing to reuse (CR); an accumulation
    stopped at r_max_iter short of s_tol schedules CT."""
    import workloads
    from gpu_helpers import to_device_system
    from paper_2211_07894_gb300 import Context, Lrdma, build
    build.build()
    cfg = workloads.random_system(71, (8, 7, 6), 24, 26.0, 0.02, 3)
    R0h = workloads.smooth_field(cfg["n"], cfg["h"], 0.1, workloads.rng_for(71, 1))[None]
    ng = int(np.prod(cfg["n"]))
    w = float(np.prod(cfg["h"]))
    ctx = Context([to_device_system(cfg, torch.float64, k_max=1)], prec="fp64", io_dtype=torch.float64,
                  k_max=1)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731

    def run(obj, R, **p):
        rho = torch.zeros(1, ng, dtype=torch.float64, device="cuda")
        rep = obj.step(ctx, dev(R), rho, **p)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        return rep, -rho.cpu().numpy() / rep["alpha"]            # Delta

    def r_lin(obj):
        obj.save(tmp_path / "h.npz")
        return np.load(tmp_path / "h.npz")["R_lin"].reshape(1, ng)

    def fresh(R, **p):
        f = Lrdma(ng, torch.float64, w, capacity=16)
        out = run(f, R, **p)
        f.close()
        return out

    # CL: beta = |1/c - 1| > beta_tol, then the same step as on an empty history
    a = Lrdma(ng, torch.float64, w, capacity=16)
    run(a, R0h, alpha=0.5)
    R1 = 2.0 * r_lin(a)
    rep, d = run(a, R1, alpha=0.5, r_norm_clear=1e9)
    rep_f, d_f = fresh(R1, alpha=0.5)
    assert rep["event"] == "CL" and abs(rep["beta"] - 0.5) < 1e-12
    assert rep["rank"] == rep_f["rank"] and np.abs(d - d_f).max() <= 1e-12 * np.abs(d_f).max()
    # reuse: the history's fit of R_lin in closed form, the step scaled by 1 - alpha
    for alpha in (0.5, 0.3):
        b = Lrdma(ng, torch.float64, w, capacity=16)
        rep0, d0 = run(b, R0h, alpha=alpha, s_tol=0.02)
        s = rep0["s_rel"]
        s_hist = s / np.sqrt(s * s + (1 - alpha) ** 2 * (1 - s * s))
        rep, d = run(b, r_lin(b), alpha=alpha, s_tol=0.3)
        assert rep["event"] == "reuse" and rep["rank_new"] == 0 and rep["beta"] < 1e-12
        assert abs(rep["s_rel"] - s_hist) < 1e-10
        assert np.linalg.norm(d - (1 - alpha) * d0) <= 1e-10 * np.linalg.norm(d0)
        b.close()
    # CR: alpha = 1 leaves R_lin outside the history's reach
    c = Lrdma(ng, torch.float64, w, capacity=16)
    run(c, R0h, alpha=1.0)
    R1 = r_lin(c)
    rn = float(np.sqrt(w * np.sum(R1 * R1)))
    rep, d = run(c, R1, alpha=0.5, r_norm_clear=0.5 * rn)
    rep_f, d_f = fresh(R1, alpha=0.5)
    assert rep["event"] == "CR" and rep["beta"] < 1e-12 and abs(rep["s_rel"] - rep_f["s_rel"]) < 1e-12
    assert np.abs(d - d_f).max() <= 1e-12 * np.abs(d_f).max()
    # accumulate to r_max_iter short of s_tol, then CT
    e = Lrdma(ng, torch.float64, w, capacity=16)
    run(e, R0h, alpha=1.0, r_max=2, s_tol=1e-9)
    rep, _ = run(e, r_lin(e), alpha=0.5, s_tol=1e-9, r_max_iter=3, r_norm_clear=1e9)
    assert rep["event"] == "accumulate" and (rep["rank"], rep["rank_new"]) == (5, 3)
    rep, _ = run(e, r_lin(e), alpha=0.5, s_tol=0.3, r_norm_clear=1e9)
    assert rep["event"] == "CT"
    for o in (a, c, e):
        o.close()
    ctx.close()
