"""GPU parity of the Brillouin-zone-sampled response (lrdm_kp_create /
lrdm_kp_gateaux) against oracle.gateaux_kpoints (§II.C closing paragraphs,
Eq. tracelessCondition), through the C ABI.

Sizes: N_s = 150 (three 64-wide tiles, the last one ragged), N_g = 12*11*10 =
1320 (ragged against the 64-row blocks of the density contraction and padded
to 1408 rows for the tensor cores), nk = 3 k-points with unequal weights, K = 3
of k_max = 4 directions.  The tensor-core precisions run the real
contractions on the stacked operand [Re Psi, Im Psi] (2 N_s = 300 columns,
padded to three 128-column blocks).  Bounds are those of the real path: FP64
1e-10 (relative, per direction); FP32 (FP32 accumulation over row ranges of
N_g products of unit-scale values, error ~ sqrt(N_g) 2^-24 relative per entry,
with headroom) 1e-4; TF32 5e-3 (10-bit mantissas); BF16x3 1e-5 on f and 1e-4
on mu' (the bound of one FP32-accumulated projected entry).
"""

import numpy as np
import pytest

import oracle
import workloads
from gates import check, gate
from helpers import per_direction_rel_err, rel_err

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N = (12, 11, 10)
NS, NK, NE, KT, K = 150, 3, 110.0, 0.01, 3
DT = {"fp64": torch.float64, "fp32": torch.float32, "tf32": torch.float32, "bf16x3": torch.float32}


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def cfg():
    return workloads.kpoint_system(70, N, NS, NK, NE, KT, K)


def _oracle(cfg, psi):
    ks = oracle.KpointSystem(n=cfg["n"], h=cfg["h"], psi=psi, eps=cfg["eps"], k_weights=cfg["k_weights"],
                             rho=np.zeros(int(np.prod(cfg["n"]))), n_electrons=cfg["n_electrons"],
                             kT=cfg["kT"], g=cfg["g"])
    mu = oracle.solve_mu_kpoints(cfg["eps"], cfg["k_weights"], cfg["n_electrons"], cfg["kT"], cfg["g"])
    ks.rho = oracle.density_kpoints(ks, mu, cfg["rho_floor"])
    return ks, mu


def _device(cfg, prec, pass_rho=None, k_max=4, nk=None):
    from paper_2211_07894_gb300 import KpContext
    dt = DT[prec]
    nk = nk or len(cfg["psi"])
    pr = [torch.as_tensor(np.ascontiguousarray(p.real), dtype=dt, device="cuda") for p in cfg["psi"][:nk]]
    pi = [torch.as_tensor(np.ascontiguousarray(p.imag), dtype=dt, device="cuda") for p in cfg["psi"][:nk]]
    eps = [torch.as_tensor(e, dtype=torch.float64, device="cuda") for e in cfg["eps"][:nk]]
    rho = torch.as_tensor(pass_rho, dtype=dt, device="cuda") if pass_rho is not None else None
    ctx = KpContext(cfg["n"], cfg["h"], pr, pi, eps, cfg["k_weights"][:nk], cfg["n_electrons"], cfg["kT"],
                    g=cfg["g"], rho=rho, rho_floor=cfg["rho_floor"], prec=prec, io_dtype=dt, k_max=k_max)
    psi_seen = [(a.double().cpu().numpy() + 1j * b.double().cpu().numpy()) for a, b in zip(pr, pi)]
    return ctx, psi_seen


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_kpoint_gateaux_matches_oracle(lib, cfg, prec):
    ctx, psi_seen = _device(cfg, prec)
    ks, mu = _oracle(cfg, psi_seen)
    assert abs(ctx.mu() - mu) < 1e-12
    rho_d = ctx.density().double().cpu().numpy()
    assert rel_err(rho_d, ks.rho) < (1e-13 if prec == "fp64" else 1e-6)
    # two calls in a row give the same result (no state carried between calls)
    V = torch.as_tensor(cfg["V"], dtype=DT[prec], device="cuda")
    F0, _ = ctx.gateaux(V)
    F, dmu = ctx.gateaux(V)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert torch.equal(F0, F)
    # the oracle on the density the device computed (FP32: its rounded copy)
    ks.rho = rho_d
    Vh = V.double().cpu().numpy()
    ref = oracle.gateaux_kpoints(ks, Vh)
    Fd = F.double().cpu().numpy()
    err = per_direction_rel_err(Fd, ref["F"])
    derr = per_direction_rel_err(Fd + Vh, ref["drho"])
    dmu_d = dmu.cpu().numpy()
    scale = max(float(np.max(np.abs(np.diagonal(X, axis1=1, axis2=2)))) for X in ref["X"])
    print(f"k-point {prec}: f err {err:.2e}, drho err {derr:.2e}, "
          f"dmu err {np.max(np.abs(dmu_d - ref['dmu'])):.2e}")
    check(prec, "kpoint_gateaux_matches_oracle", err)
    check(prec, "kpoint_gateaux_matches_oracle", derr)
    check(prec, "kpoint_gateaux_matches_oracle", float(np.max(np.abs(dmu_d - ref["dmu"]))) / scale, "dmu")


def test_kpoint_given_density_single_point_and_fewer_directions(lib, cfg):
    one = dict(cfg)
    one["psi"] = cfg["psi"][:1]
    one["eps"] = cfg["eps"][:1]
    one["k_weights"] = np.array([1.0])
    ks, mu = _oracle(one, one["psi"])
    rho = ks.rho * 1.1
    ctx, _ = _device(one, "fp64", pass_rho=rho)
    assert rel_err(ctx.density().cpu().numpy(), rho) < 1e-15
    V = torch.as_tensor(cfg["V"], dtype=torch.float64, device="cuda")
    F, dmu = ctx.gateaux(V)
    torch.cuda.synchronize()
    ks.rho = rho
    ref = oracle.gateaux_kpoints(ks, cfg["V"])
    assert per_direction_rel_err(F.cpu().numpy(), ref["F"]) < 1e-10
    F1, _ = ctx.gateaux(V[1:2].contiguous())
    torch.cuda.synchronize()
    assert rel_err(F1.cpu().numpy()[0], ref["F"][1]) < 1e-10
    F0, _ = ctx.gateaux(V[:0].contiguous())
    assert F0.shape[0] == 0
    assert ctx.status() == 0


def test_kpoint_least_squares_step(lib, cfg):
    ctx, psi_seen = _device(cfg, "fp64")
    ks, _ = _oracle(cfg, psi_seen)
    V = torch.as_tensor(cfg["V"], dtype=torch.float64, device="cuda")
    F, _ = ctx.gateaux(V)
    R = torch.as_tensor(workloads.smooth_directions(N, cfg["h"], 1, 1, workloads.rng_for(70, 9))[0, 0],
                        device="cuda").contiguous()
    rho = torch.as_tensor(ks.rho, device="cuda").clone()
    coef, srel = ctx.apply(R, V, F, 0.5, rho=rho)
    torch.cuda.synchronize()
    ref = oracle.gateaux_kpoints(ks, cfg["V"])
    want = oracle.lrdm_apply(R.cpu().numpy()[None], cfg["V"][:, None], ref["F"][:, None], ks.w, 0.5,
                             rho=ks.rho[None])
    assert np.allclose(coef.cpu().numpy(), want["a"], rtol=1e-9, atol=1e-12)
    assert abs(srel.item() - want["s_rel"]) < 1e-9
    assert rel_err(rho.cpu().numpy(), want["rho_new"][0]) < 1e-10


def test_kpoint_rejections(lib, cfg):
    from paper_2211_07894_gb300 import LrdmError, binding
    with pytest.raises(LrdmError) as e:
        _device(cfg, "fp64", nk=2)                   # weights of 2 of the 3 points do not sum to 1
    assert e.value.code == 1
    with pytest.raises(LrdmError) as e:
        from paper_2211_07894_gb300 import KpContext
        p = torch.zeros((int(np.prod(N)), NS), dtype=torch.float32, device="cuda")
        KpContext(N, cfg["h"], [p], [p], [torch.as_tensor(cfg["eps"][0], device="cuda")], [1.0], NE, 0.0,
                  prec="bf16x3", io_dtype=torch.float32)          # kT = 0
    assert e.value.code == 1
    ctx, _ = _device(cfg, "fp64")
    V = torch.as_tensor(cfg["V"], dtype=torch.float64, device="cuda")
    F = torch.empty_like(V)
    # the real-subspace calls are refused for a k-point context
    assert binding.lrdm_gateaux_batch(ctx.handle, [V.data_ptr()], [K], [F.data_ptr()], 0) == 9
    assert binding.lrdm_get_projection(ctx.handle, 0, 0, 0, F.data_ptr()) == 9
    with pytest.raises(LrdmError):
        ctx.gateaux(torch.zeros((5, V.shape[1]), dtype=torch.float64, device="cuda"))   # K > k_max
    assert ctx.status() == 0


def test_kpoint_autotuned_shape_matches_default(lib, cfg):
    # the tuner picks among launch shapes of the same contractions: results agree
    ctx0, _ = _device(cfg, "bf16x3")
    from paper_2211_07894_gb300 import KpContext
    pr = [torch.as_tensor(np.ascontiguousarray(p.real), dtype=torch.float32, device="cuda") for p in cfg["psi"]]
    pi = [torch.as_tensor(np.ascontiguousarray(p.imag), dtype=torch.float32, device="cuda") for p in cfg["psi"]]
    eps = [torch.as_tensor(e, dtype=torch.float64, device="cuda") for e in cfg["eps"]]
    ctx1 = KpContext(cfg["n"], cfg["h"], pr, pi, eps, cfg["k_weights"], cfg["n_electrons"], cfg["kT"],
                     g=cfg["g"], rho_floor=cfg["rho_floor"], prec="bf16x3", io_dtype=torch.float32, k_max=4,
                     autotune=True)
    t = ctx1.tuning()
    assert t["g1_nb"] in (128, 256) and t["g2_bn"] in (128, 256) and t["g2_kgroup"] in (1, 2, 4)
    V = torch.as_tensor(cfg["V"], dtype=torch.float32, device="cuda")
    F0, d0 = ctx0.gateaux(V)
    F1, d1 = ctx1.gateaux(V)
    torch.cuda.synchronize()
    assert ctx1.status() == 0
    assert per_direction_rel_err(F1.double().cpu().numpy(), F0.double().cpu().numpy()) < 1e-5
    assert np.max(np.abs(d1.cpu().numpy() - d0.cpu().numpy())) < 1e-6


@pytest.mark.parametrize("prec,io", [("bf16x3", torch.float64), ("tf32", torch.float32)])
def test_kpoint_tensor_cores_edge_cases(lib, cfg, prec, io):
    """Tensor-core k-point path with FP64 io or TF32, one point with weight 1
    and a given density, K = 1 and K = 2 < k_max after a K = 3 call."""
    from paper_2211_07894_gb300 import KpContext
    one = dict(cfg)
    one["psi"] = cfg["psi"][1:2]
    one["eps"] = cfg["eps"][1:2]
    one["k_weights"] = np.array([1.0])
    ks, mu = _oracle(one, one["psi"])
    rho = ks.rho * 0.9
    pr = [torch.as_tensor(np.ascontiguousarray(p.real), dtype=io, device="cuda") for p in one["psi"]]
    pi = [torch.as_tensor(np.ascontiguousarray(p.imag), dtype=io, device="cuda") for p in one["psi"]]
    eps = [torch.as_tensor(e, dtype=torch.float64, device="cuda") for e in one["eps"]]
    ctx = KpContext(cfg["n"], cfg["h"], pr, pi, eps, [1.0], cfg["n_electrons"], cfg["kT"], g=cfg["g"],
                    rho=torch.as_tensor(rho, dtype=io, device="cuda"), prec=prec, io_dtype=io, k_max=4)
    psi_seen = [a.double().cpu().numpy() + 1j * b.double().cpu().numpy() for a, b in zip(pr, pi)]
    ks.psi = psi_seen
    ks.rho = ctx.density().double().cpu().numpy()
    V = torch.as_tensor(cfg["V"], dtype=io, device="cuda")
    ref = oracle.gateaux_kpoints(ks, V.double().cpu().numpy())
    case = "kpoint_tensor_cores_edge_cases"
    F3, _ = ctx.gateaux(V)
    F1, d1 = ctx.gateaux(V[2:3].contiguous())
    F2, _ = ctx.gateaux(V[:2].contiguous())
    torch.cuda.synchronize()
    assert ctx.status() == 0
    check(prec, case, per_direction_rel_err(F3.double().cpu().numpy(), ref["F"]))
    check(prec, case, rel_err(F1.double().cpu().numpy()[0], ref["F"][2]))
    check(prec, case, per_direction_rel_err(F2.double().cpu().numpy(), ref["F"][:2]))
    # the same direction gives the same result in a batch of 3 or alone
    assert torch.equal(F1[0], F3[2]) or rel_err(F1.double().cpu().numpy()[0], F3.double().cpu().numpy()[2]) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_kpoint_krylov_step(lib, cfg, prec):
    """lrdm_krylov_step on a k-point context against the oracle's LRDM step
    with the k-point derivative: same rank, directions, derivatives,
    coefficients and density update."""
    ctx, psi_seen = _device(cfg, prec, k_max=1)
    ks, _ = _oracle(cfg, psi_seen)
    ks.rho = ctx.density().double().cpu().numpy()
    io = DT[prec]
    R = workloads.smooth_field(cfg["n"], cfg["h"], 0.1, workloads.rng_for(70, 11))
    R = torch.as_tensor(R, dtype=io).double().numpy()           # the values the device sees
    ref = oracle.lrdm_krylov_step(ks, R, s_tol=1e-12, r_max=4)
    s_tol = 0.5 * (ref["s_rel"][1] + ref["s_rel"][2])           # stop at rank 3
    ref = oracle.lrdm_krylov_step(ks, R, s_tol=s_tol, r_max=4, rho=ks.rho)
    rho = torch.as_tensor(ks.rho, dtype=io, device="cuda")
    out = ctx.krylov_step(torch.as_tensor(R, dtype=io, device="cuda"), s_tol=s_tol, r_max=4, rho=rho)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert out["rank"] == ref["rank"] == 3
    tol = gate(prec, "kpoint_krylov_step")
    assert np.allclose(out["s_rel"], ref["s_rel"], rtol=10 * tol, atol=0)
    assert per_direction_rel_err(out["U"].double().cpu().numpy(), ref["U"]) < 10 * tol
    assert per_direction_rel_err(out["T"].double().cpu().numpy(), ref["T"]) < 10 * tol
    assert np.allclose(out["a"].cpu().numpy(), ref["a"], rtol=100 * tol, atol=0)
    assert rel_err(rho.double().cpu().numpy() - ks.rho, ref["rho_new"] - ks.rho) < 100 * tol


def test_kpoint_lrdma_steps_follow_oracle(lib, cfg):
    """Three accumulated-LRDM steps (lrdm_lrdma_step) on one k-point context
    along a residual sequence R_{n+1} = R_lin,n + a small smooth change: the
    same event, kept and new rank, s_rel and density update as the oracle."""
    from paper_2211_07894_gb300 import Lrdma
    ctx, psi_seen = _device(cfg, "fp64", k_max=1)
    ks, _ = _oracle(cfg, psi_seen)
    ks.rho = ctx.density().cpu().numpy()
    gpu = Lrdma(int(np.prod(N)), torch.float64, ks.w, capacity=8)
    state = oracle.LrdmaState()
    rng = workloads.rng_for(70, 12)
    R = workloads.smooth_field(N, cfg["h"], 0.1, rng)
    rho = ks.rho.copy()
    events = []
    for it in range(3):
        ref = oracle.lrdma_step(ks, state, R, rho=rho, r_max=8)
        rho_d = torch.as_tensor(rho, device="cuda").clone()
        rep = gpu.step(ctx, torch.as_tensor(R, device="cuda").contiguous(), rho_d, r_max=8)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        assert rep["event"] == ref["event"], (it, rep, ref["event"])
        assert (rep["rank"], rep["rank_new"]) == (ref["rank"], ref["rank_new"])
        assert abs(rep["s_rel"] - ref["s_rel"]) <= 1e-9 * max(ref["s_rel"], 1e-3)
        d_ref = ref["rho_new"] - rho
        assert rel_err(rho_d.cpu().numpy() - rho, d_ref) < 1e-9
        events.append(rep["event"])
        rho = ref["rho_new"]
        R = state.R_lin + workloads.smooth_field(N, cfg["h"], 0.002, rng)
    print(f"k-point LRDMA events {events}")
    gpu.close()


def test_kpoint_many_points_split_launches(lib):
    """20 k-points (more than the 16 problems of one grouped tensor-core
    launch: two launches per contraction) and the 32-point maximum, small
    sizes; 33 points are refused."""
    from paper_2211_07894_gb300 import KpContext, LrdmError
    for nk, prec in ((20, "bf16x3"), (32, "fp64")):
        c = workloads.kpoint_system(71, (8, 7, 6), 20, nk, 22.0, 0.02, 2)
        ctx, psi_seen = _device(c, prec, k_max=2)
        ks, mu = _oracle(c, psi_seen)
        assert abs(ctx.mu() - mu) < 1e-12
        ks.rho = ctx.density().double().cpu().numpy()
        V = torch.as_tensor(c["V"], dtype=DT[prec], device="cuda")
        F, _ = ctx.gateaux(V)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        ref = oracle.gateaux_kpoints(ks, V.double().cpu().numpy())
        err = per_direction_rel_err(F.double().cpu().numpy(), ref["F"])
        print(f"{nk} k-points {prec}: f err {err:.2e}")
        check(prec, "kpoint_many_points_split_launches", err)
        ctx.close()
    c = workloads.kpoint_system(72, (6, 6, 6), 8, 33, 8.0, 0.02, 1)
    p = [torch.as_tensor(np.ascontiguousarray(x.real), device="cuda") for x in c["psi"]]
    e = [torch.as_tensor(x, device="cuda") for x in c["eps"]]
    with pytest.raises(LrdmError) as ex:
        KpContext(c["n"], c["h"], p, p, e, c["k_weights"], 8.0, 0.02)
    assert ex.value.code == 1


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_kpoint_backward_matches_oracle(lib, cfg, prec):
    """lrdm_backward on a k-point context (v_bar of the last forward call)
    against oracle.backward_kpoints, and the dot-product identity on the
    device's own forward and adjoint."""
    ctx, psi_seen = _device(cfg, prec)
    ks, _ = _oracle(cfg, psi_seen)
    ks.rho = ctx.density().double().cpu().numpy()
    io = DT[prec]
    V = torch.as_tensor(cfg["V"], dtype=io, device="cuda")
    fbar = torch.as_tensor(workloads.rng_for(70, 13).standard_normal(cfg["V"].shape), dtype=io, device="cuda")
    F, _ = ctx.gateaux(V)
    vbar = ctx.backward(fbar)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = oracle.backward_kpoints(ks, fbar.double().cpu().numpy())
    err = per_direction_rel_err(vbar.double().cpu().numpy(), ref)
    lhs = float((fbar.double() * F.double()).sum())
    rhs = float((vbar.double() * V.double()).sum())
    print(f"k-point adjoint {prec}: v_bar err {err:.2e}, dot-product rel {abs(lhs - rhs) / abs(lhs):.2e}")
    check(prec, "kpoint_backward_matches_oracle", err)
    assert abs(lhs - rhs) <= 10 * gate(prec, "kpoint_backward_matches_oracle") * abs(lhs)
    from paper_2211_07894_gb300 import binding
    e = torch.empty(NS, dtype=torch.float64, device="cuda")
    assert binding.lrdm_backward(ctx.handle, [fbar.data_ptr()], [vbar.data_ptr()], [e.data_ptr(), 0],
                                 None) == 9       # no eigenvalue gradients for k-point contexts


def test_kpoint_autograd_function(lib, cfg):
    """gateaux_function on a k-point context: torch autograd through the
    hand-written adjoint satisfies <fbar, F> = <V.grad, V> (F linear in V)."""
    from paper_2211_07894_gb300 import gateaux_function
    ctx, _ = _device(cfg, "fp64")
    V = torch.as_tensor(cfg["V"], dtype=torch.float64, device="cuda").requires_grad_(True)
    fbar = torch.as_tensor(workloads.rng_for(70, 14).standard_normal(cfg["V"].shape), device="cuda")
    F = gateaux_function().apply(ctx, V)
    (F * fbar).sum().backward()
    lhs = float((fbar * F.detach()).sum())
    rhs = float((V.grad * V.detach()).sum())
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_kpoint_split_row_ranges(lib):
    """A 24^3 grid (432 reduction stages) where the tensor-core projection
    splits the grid into row ranges (3 for 45 items per range on 152 SMs):
    the summed partials give the oracle's response."""
    c = workloads.kpoint_system(73, (24, 24, 24), NS, NK, NE, KT, K)
    for prec in ("bf16x3", "fp64"):
        ctx, psi_seen = _device(c, prec)
        ks, _ = _oracle(c, psi_seen)
        ks.rho = ctx.density().double().cpu().numpy()
        V = torch.as_tensor(c["V"], dtype=DT[prec], device="cuda")
        F, dmu = ctx.gateaux(V)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        ref = oracle.gateaux_kpoints(ks, V.double().cpu().numpy())
        err = per_direction_rel_err(F.double().cpu().numpy(), ref["F"])
        print(f"k-point 24^3 {prec}: f err {err:.2e}")
        check(prec, "kpoint_split_row_ranges", err)
        ctx.close()


def test_kpoint_graph_replay_equals_eager(lib, cfg):
    """use_graph on a k-point context (bf16x3): the captured call replayed on
    a side stream gives bit-identical results to the eager call; a different
    K is captured anew; the adjoint after a replay uses that call's K."""
    from paper_2211_07894_gb300 import KpContext
    eager, _ = _device(cfg, "bf16x3")
    pr = [torch.as_tensor(np.ascontiguousarray(p.real), dtype=torch.float32, device="cuda") for p in cfg["psi"]]
    pi = [torch.as_tensor(np.ascontiguousarray(p.imag), dtype=torch.float32, device="cuda") for p in cfg["psi"]]
    eps = [torch.as_tensor(e, dtype=torch.float64, device="cuda") for e in cfg["eps"]]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = KpContext(cfg["n"], cfg["h"], pr, pi, eps, cfg["k_weights"], cfg["n_electrons"], cfg["kT"],
                      g=cfg["g"], rho_floor=cfg["rho_floor"], prec="bf16x3", io_dtype=torch.float32, k_max=4,
                      use_graph=True)
        V = torch.as_tensor(cfg["V"], dtype=torch.float32, device="cuda")
        F = torch.empty_like(V)
        ref, _ = eager.gateaux(V)
        for _ in range(3):
            g.gateaux(V, out=F)                       # capture, then replays
        V2 = V[:2].contiguous()
        F2 = torch.empty_like(V2)
        g.gateaux(V2, out=F2)
        fbar = torch.ones_like(V2)
        vbar = g.backward(fbar)
    st.synchronize()
    ref2, _ = eager.gateaux(V2)
    vref = eager.backward(fbar)
    torch.cuda.synchronize()
    assert g.status() == 0
    assert torch.equal(F, ref) and torch.equal(F2, ref2) and torch.equal(vbar, vref)
