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
