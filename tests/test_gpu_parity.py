"""GPU parity: the CUDA path through the C ABI against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances (relative w-norm error per direction) are those of tests/gates.py:
FP64 1e-10; split-BF16x3 1e-5 on f (1e-4 on the intermediates X, drho, mu');
FP32 CUDA-core 1e-4; TF32 per case at about three times its measured error,
each check printing whether it meets the 1e-5 target.
"""

import numpy as np
import pytest

import oracle
import workloads
from gates import TOL, check, gate
from helpers import oracle_system, per_direction_rel_err, rel_err

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

IO = {"fp64": torch.float64, "fp32": torch.float32, "tf32": torch.float32,
      "bf16x3": torch.float32}


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build, binding
    build.build()
    return binding.load()


def _ragged(cfg_id=20, n=(20, 18, 22), ns=200, K=5, ne=150, kT=0.01, stream=0):
    return workloads.random_system(cfg_id, n, ns, ne, kT, K, stream=stream)


def _run(cfgs, prec, **kw):
    from gpu_helpers import directions, make_context
    io = IO[prec]
    ctx, systems = make_context(cfgs, prec, io, **kw)
    V = [directions(c, io) for c in cfgs]
    F, dmu = ctx.gateaux(V)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return ctx, V, [f.double().cpu().numpy() for f in F], dmu.cpu().numpy()


def _check_dmu(dmu, ref, prec, case):
    """mu'_k is a weighted mean of the X_k,ii, so its error is bounded by the
    error of those entries: |dmu - ref| < gate(X) * max_i |X_k,ii|."""
    worst = 0.0
    for k in range(len(dmu)):
        scale = max(np.max(np.abs(np.diag(X[k]))) for X in ref["X"])
        worst = max(worst, abs(dmu[k] - ref["dmu"][k]) / scale)
    check(prec, case, worst, "dmu")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_projection_ragged_tiles(lib, prec):
    """X_k = Psi^T diag(w dV_k) Psi alone (the first contraction)."""
    cfg = _ragged()
    ctx, V, F, dmu = _run([cfg], prec)
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    errs = []
    for k in range(cfg["V"].shape[0]):
        X = ctx.projection(k).cpu().numpy()
        errs.append(rel_err(X, ref["X"][0][k]))
    print(f"projection {prec}: max rel err {max(errs):.3e}")
    check(prec, "projection_ragged_tiles", max(errs), "X")


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_projection_and_forward_odd_block_count(lib, prec):
    """N_s = 300 pads to 384 states, three 128-blocks: the last 256-wide
    projection tile and the last response j-tile are half outside the matrix
    (their missing rows come from the TMA zero fill and are never stored)."""
    cfg = _ragged(cfg_id=24, n=(18, 16, 20), ns=300, K=3, ne=230)
    ctx, V, F, dmu = _run([cfg], prec)
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    errs = [rel_err(ctx.projection(k).cpu().numpy(), ref["X"][0][k]) for k in range(3)]
    err = per_direction_rel_err(F[0], ref["F"])
    print(f"odd block count {prec}: X err {max(errs):.2e}, f err {err:.2e}")
    check(prec, "projection_and_forward_odd_block_count", max(errs), "X")
    check(prec, "projection_and_forward_odd_block_count", err)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_small_k_row_range_split(lib, prec):
    """A one-direction call (the Krylov steps' unit) splits the projection's
    grid reduction into row ranges (40^3 rows, N_s = 512: 8 ranges); the
    partial X are summed by every consumer: X, mu', f and the adjoint meet
    the oracle tolerance, and the direction agrees with the same direction
    computed unsplit inside an 8-direction call."""
    from gpu_helpers import directions, make_context
    cfg = _ragged(cfg_id=25, n=(40, 40, 40), ns=512, K=8, ne=400)
    io = IO[prec]
    ctx, _ = make_context([cfg], prec, io)
    V = directions(cfg, io)
    F8, _ = ctx.gateaux([V])
    F8 = F8[0].double().cpu().numpy()
    one = V[2:3].contiguous()
    (F1,), dmu1 = ctx.gateaux([one])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"][2:3])
    X1 = ctx.projection(0).cpu().numpy()
    check(prec, "small_k_row_range_split", rel_err(X1, ref["X"][0][0]), "X")
    err = per_direction_rel_err(F1.double().cpu().numpy(), ref["F"])
    _check_dmu(dmu1.cpu().numpy(), ref, prec, "small_k_row_range_split")
    check(prec, "small_k_row_range_split", err)
    check(prec, "small_k_row_range_split", rel_err(F1.double().cpu().numpy()[0], F8[2]))
    fbar = workloads.rng_for(25, 9).standard_normal((1,) + cfg["V"].shape[1:])
    vbar, eb, ob = ctx.backward([torch.as_tensor(fbar, dtype=io, device="cuda")])
    torch.cuda.synchronize()
    bref = oracle.backward(oracle_system(cfg), fbar, ref)
    print(f"K=1 split {prec}: f err {err:.2e}, vbar err "
          f"{per_direction_rel_err(vbar[0].double().cpu().numpy(), bref['vbar']):.2e}")
    check(prec, "small_k_row_range_split", per_direction_rel_err(vbar[0].double().cpu().numpy(), bref["vbar"]))
    check(prec, "small_k_row_range_split", rel_err(eb[0].cpu().numpy(), bref["eps_bar"][0]), "eps_bar")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_forward_toy16(lib, cfg1, prec):
    ctx, V, F, dmu = _run([cfg1], prec)
    ref = oracle.gateaux(oracle_system(cfg1), cfg1["V"])
    err = per_direction_rel_err(F[0], ref["F"])
    print(f"toy16 {prec}: max rel err {err:.3e}")
    check(prec, "forward_toy16", err)
    _check_dmu(dmu, ref, prec, "forward_toy16")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_forward_ragged_tiles(lib, prec):
    cfg = _ragged()
    ctx, V, F, dmu = _run([cfg], prec)
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    err = per_direction_rel_err(F[0], ref["F"])
    drho_err = per_direction_rel_err(F[0] + cfg["V"], ref["drho"])
    print(f"ragged {prec}: f err {err:.3e}  drho err {drho_err:.3e}")
    check(prec, "forward_ragged_tiles", err)
    check(prec, "forward_ragged_tiles", drho_err, "X")
    _check_dmu(dmu, ref, prec, "forward_ragged_tiles")


def test_density_mu_and_given_rho(lib, cfg1):
    from gpu_helpers import directions, make_context
    ctx, _ = make_context([cfg1], "fp64", torch.float64)
    osys = oracle_system(cfg1)
    mu = oracle.solve_mu(osys.eps, osys.n_electrons, osys.kT, osys.occ_factor)
    assert abs(ctx.mu() - mu) < 1e-12
    rho = ctx.density().cpu().numpy()
    assert rel_err(rho, osys.rho[0]) < 1e-13
    # same results when the oracle's density is passed in
    from paper_2211_07894_gb300 import Context
    from gpu_helpers import to_device_system
    ctx2 = Context([to_device_system(cfg1, torch.float64, pass_rho=osys.rho)], prec="fp64",
                   io_dtype=torch.float64)
    V = directions(cfg1, torch.float64)
    F1, _ = ctx.gateaux([V])
    F2, _ = ctx2.gateaux([V])
    assert rel_err(F1[0].cpu().numpy(), F2[0].cpu().numpy()) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_spin_pair(lib, prec):
    cfg = workloads.spin_pair_system(21, (12, 12, 12), 60, 52, 50, 0.01, 3)
    ctx, V, F, dmu = _run([cfg], prec)
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    err = max(rel_err(F[0][k], ref["F"][k]) for k in range(3))
    print(f"spin {prec}: {err:.3e}")
    check(prec, "spin_pair", err)
    _check_dmu(dmu, ref, prec, "spin_pair")


def test_occupation_mode_near_degenerate(lib):
    d = workloads.config4(scale=8)      # 9^3 grid, 256 states, 5 % near-degenerate pairs
    d["V"] = d["V"][:3]
    osys = oracle_system(d, occ_mode=True)
    d["occ"] = osys.occ
    ctx, V, F, dmu = _run([d], "fp64", k_max=3)
    ref = oracle.gateaux(osys, d["V"])
    assert per_direction_rel_err(F[0], ref["F"]) < 1e-10


def test_near_degenerate_default_mode(lib):
    d = workloads.config4(scale=8)
    d["V"] = d["V"][:3]
    ctx, V, F, dmu = _run([d], "fp64", k_max=3)
    ref = oracle.gateaux(oracle_system(d), d["V"])
    assert per_direction_rel_err(F[0], ref["F"]) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16x3"])
def test_batched_uneven_equals_separate(lib, prec):
    """Systems of different sizes and K in one call (one grouped launch per
    contraction on the tensor-core paths) give bit-for-bit the results of
    separate contexts, and each meets the oracle tolerance."""
    cfgs = workloads.config3(scale=8)
    from gpu_helpers import directions, make_context
    io = IO[prec]
    ctx, _ = make_context(cfgs, prec, io)
    V = [directions(c, io) for c in cfgs]
    F, dmu = ctx.gateaux(V)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    off = 0
    for i, c in enumerate(cfgs):
        one, _ = make_context([c], prec, io)
        Fi, dmui = one.gateaux([V[i]])
        assert torch.equal(Fi[0], F[i])
        assert torch.equal(dmui, dmu[off:off + len(dmui)])
        off += len(dmui)
        ref = oracle.gateaux(oracle_system(c), c["V"])
        err = per_direction_rel_err(F[i].double().cpu().numpy(), ref["F"])
        print(f"batched system {i} {prec}: f rel err {err:.2e}")
        check(prec, "batched_uneven_equals_separate", err)


def _tune_key(cfgs, prec_code):
    """The autotuner's cache key of a problem set (device, precision, every
    (N_g, N_s padded to 128, k_max)); each system's k_max is its K."""
    props = torch.cuda.get_device_properties(0)
    major, minor = torch.cuda.get_device_capability(0)
    k = f"sm{major}{minor}x{props.multi_processor_count};prec{prec_code}"
    for c in cfgs:
        ng = int(np.prod(c["n"]))
        for p in c["psi"]:
            k += f";{ng},{(p.shape[1] + 127) // 128 * 128},{c['V'].shape[0]}"
    return k


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_forced_launch_shapes(lib, prec, tmp_path, monkeypatch):
    """Launch shapes forced through the tuning cache (128 x 128 projection
    tiles with one or two directions, 128 x 256 tiles, 256 x 256 pair tiles,
    128- and 256-wide response j-tiles, direction groups 1, 2, 4): every
    shape meets the oracle
    tolerance on X and f; shapes that differ only in how work items are
    grouped reproduce each other bit for bit."""
    from gpu_helpers import directions, make_context
    cfgs = workloads.config3(scale=8)[:3]
    io = IO[prec]
    base, _ = make_context(cfgs, prec, io)          # default shape: pair tiles for both, group 4
    V = [directions(c, io) for c in cfgs]
    F0, _ = base.gateaux(V)
    X0 = base.projection(1, sys=1)
    X_square = None
    code = {"tf32": 2, "bf16x3": 3}[prec]
    Xr = oracle.gateaux(oracle_system(cfgs[1]), cfgs[1]["V"][1:2])["X"][0][0]
    for nb, dpt, bn, kg in [(128, 1, 128, 1), (128, 2, 128, 4), (128, 1, 256, 4), (256, 1, 256, 4),
                            (512, 1, 256, 2), (512, 1, 512, 4)]:
        cache = tmp_path / f"tune_{nb}_{dpt}_{bn}_{kg}.jsonl"
        cache.write_text('{"key": "%s", "g1_nb": %d, "g1_dpt": %d, "g2_bn": %d, "g2_kgroup": %d}\n'
                         % (_tune_key(cfgs, code), nb, dpt, bn, kg))
        monkeypatch.setenv("LRDM_TUNE_CACHE", str(cache))
        ctx, _ = make_context(cfgs, prec, io, autotune=True)
        assert ctx.tuning() == {"g1_nb": nb, "g1_dpt": dpt, "g2_bn": bn, "g2_kgroup": kg}
        F, _ = ctx.gateaux(V)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        X = ctx.projection(1, sys=1)
        check(prec, "forced_launch_shapes", rel_err(X.cpu().numpy(), Xr), "X")
        if nb == 512:
            assert torch.equal(X, X0)          # same tiles as the default
        elif nb == 256:
            pass                               # 128 x 256 tiles: checked against the oracle above
        elif X_square is None:
            X_square = X
        else:
            assert torch.equal(X, X_square)    # 1 or 2 directions per square tile: same sums
        for i, c in enumerate(cfgs):
            ref = oracle.gateaux(oracle_system(c), c["V"])
            err = per_direction_rel_err(F[i].double().cpu().numpy(), ref["F"])
            check(prec, "forced_launch_shapes", err)
            if bn in (256, 512) and nb == 512:
                # the direction group only reorders items, and the pair response
                # sums each row in the single-CTA kernel's order
                assert torch.equal(F[i], F0[i])
        assert len(cache.read_text().splitlines()) == 1     # read, not re-tuned


def test_autotune_batched(lib, tmp_path, monkeypatch):
    """The autotuner on the uneven batch: a valid choice, results within the
    oracle tolerance, and the choice cached and reused."""
    from gpu_helpers import directions, make_context
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("LRDM_TUNE_CACHE", str(cache))
    cfgs = workloads.config3(scale=8)
    ctx, _ = make_context(cfgs, "bf16x3", torch.float32, autotune=True)
    t = ctx.tuning()
    print("autotuned launch shape (uneven batch):", t)
    assert t["g1_nb"] in (128, 256, 512) and t["g1_dpt"] in (1, 2)
    assert t["g2_bn"] in (128, 256, 512) and t["g2_kgroup"] in (1, 2, 4)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and '"key": "sm' in lines[0]
    V = [directions(c, torch.float32) for c in cfgs]
    F, _ = ctx.gateaux(V)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    for i, c in enumerate(cfgs):
        ref = oracle.gateaux(oracle_system(c), c["V"])
        assert per_direction_rel_err(F[i].double().cpu().numpy(), ref["F"]) < TOL["bf16x3"]
    again, _ = make_context(cfgs, "bf16x3", torch.float32, autotune=True)
    assert again.tuning() == t
    assert len(cache.read_text().splitlines()) == 1


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_graph_replay(lib, cfg1, prec):
    """use_graph: the first call on a stream captures the forward path, later
    calls with the same buffers replay it and see new values written into
    them; a new K (or new buffers) captures again."""
    from gpu_helpers import directions, make_context
    io = IO[prec]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plain, _ = make_context([cfg1], prec, io)
        ctx, _ = make_context([cfg1], prec, io, use_graph=True)
        V = directions(cfg1, io)
        ref, ref_dmu = plain.gateaux([V])
        out = [torch.empty_like(V)]
        dmu = torch.empty(V.shape[0], dtype=torch.float64, device="cuda")
        for _ in range(3):
            out[0].fill_(float("nan"))
            ctx.gateaux([V], out=out, dmu=dmu)
            st.synchronize()
            assert torch.equal(out[0], ref[0])
            assert torch.equal(dmu, ref_dmu)
        # new values in the same buffer: the replay reads them
        V.mul_(-0.5)
        ref2, _ = plain.gateaux([V])
        ctx.gateaux([V], out=out, dmu=dmu)
        st.synchronize()
        assert torch.equal(out[0], ref2[0])
        # fewer directions: captured again
        V3 = V[:2].contiguous()
        ref3, _ = plain.gateaux([V3])
        F3, _ = ctx.gateaux([V3])
        st.synchronize()
        assert torch.equal(F3[0], ref3[0])
        assert ctx.status() == 0
        # backward after a replayed forward uses that forward's state
        fbar = [torch.randn_like(V3)]
        vb_p, eb_p, _ = plain.backward(fbar)
        vb_g, eb_g, _ = ctx.backward(fbar)
        st.synchronize()
        assert torch.equal(vb_p[0], vb_g[0])
        assert torch.equal(eb_p[0], eb_g[0])


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_apply_step(lib, cfg1, prec):
    io = IO[prec]
    # the least-squares step alone, on the oracle's derivatives
    ctx, V, _, _ = _run([cfg1], prec)
    osys = oracle_system(cfg1)
    Fref = oracle.gateaux(osys, cfg1["V"])["F"]
    Fd = torch.as_tensor(Fref, dtype=io, device="cuda")
    Vd = V[0]
    R = torch.as_tensor(cfg1["R"], dtype=io, device="cuda")
    rho = torch.as_tensor(np.stack(osys.rho), dtype=io, device="cuda")
    coef, srel = ctx.apply(0, R, Vd, Fd, 0.5, rho=rho)
    torch.cuda.synchronize()
    want = oracle.lrdm_apply(cfg1["R"], cfg1["V"], Fref, osys.w, 0.5, rho=np.stack(osys.rho))
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert np.allclose(coef.cpu().numpy(), want["a"], rtol=tol * 10, atol=1e-12)
    assert abs(srel.item() - want["s_rel"]) < tol * 10
    assert rel_err(rho.double().cpu().numpy(), want["rho_new"]) < tol


@pytest.mark.parametrize("K", [1, 2, 3, 7, 16, 33, 64])
def test_apply_solver_odd_and_large_k(lib, K):
    """The K x K solve (parallel Jacobi rounds: an odd K pairs one index with
    a dummy each round) on seeded derivatives whose singular values spread
    over four decades, against the oracle's LS step and numpy's lstsq, FP64."""
    cfg = _ragged(cfg_id=22, n=(12, 10, 14), ns=70, K=64, ne=50)
    from gpu_helpers import make_context
    ctx, _ = make_context([cfg], "fp64", torch.float64)
    rng = workloads.rng_for(22, 40 + K)
    ng = int(np.prod(cfg["n"]))
    w = float(np.prod(cfg["h"]))
    Fm = rng.standard_normal((K, ng)) * np.logspace(0, -4, K)[:, None]
    Vm = rng.standard_normal((K, ng))
    R = rng.standard_normal(ng)
    rho = 1.0 + 0.1 * rng.random(ng)
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    rho_d = dev(rho[None, :])
    coef, srel = ctx.apply(0, dev(R[None, :]), dev(Vm), dev(Fm), 0.5, rho=rho_d)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    want = oracle.lrdm_apply(R[None, :], Vm, Fm, w, 0.5, rho=rho[None, :])
    a_ls = np.linalg.lstsq(np.sqrt(w) * Fm.T, np.sqrt(w) * R, rcond=None)[0]
    a = coef.cpu().numpy()
    print(f"K = {K}: coefficient error vs oracle {rel_err(a, want['a']):.2e}, vs lstsq "
          f"{rel_err(a, a_ls):.2e}")
    # cond(S) = 1e8: the coefficients carry cond(S) times the rounding of S
    assert rel_err(a, want["a"]) < 1e-7
    assert rel_err(a, a_ls) < 1e-7
    assert abs(srel.item() - want["s_rel"]) < 1e-10
    assert rel_err(rho_d.cpu().numpy(), want["rho_new"]) < 1e-10


def test_apply_singular_flag_and_nonfinite(lib, cfg1):
    ctx, V, _, _ = _run([cfg1], "fp64")
    Fh = oracle.gateaux(oracle_system(cfg1), cfg1["V"])["F"]
    Fh[3] = Fh[1]
    Fd = torch.as_tensor(Fh, dtype=torch.float64, device="cuda")
    R = torch.as_tensor(cfg1["R"], dtype=torch.float64, device="cuda")
    coef, srel = ctx.apply(0, R, V[0], Fd, 0.0)
    assert ctx.status() == 6          # LRDM_ERR_SINGULAR
    w = float(np.prod(cfg1["h"]))
    a_ref = np.linalg.lstsq(np.sqrt(w) * Fh.reshape(4, -1).T, np.sqrt(w) * cfg1["R"].ravel(), rcond=1e-10)[0]
    assert np.allclose(coef.cpu().numpy(), a_ref, rtol=1e-8)
    R[0, 5] = float("nan")
    ctx.apply(0, R, V[0], Fd, 0.0)
    assert ctx.status() == 8          # LRDM_ERR_NONFINITE
    assert ctx.status() == 0          # cleared


def test_argument_errors(lib, cfg1):
    from paper_2211_07894_gb300 import LrdmError
    from gpu_helpers import directions, make_context
    ctx, _ = make_context([cfg1], "fp64", torch.float64)
    V = directions(cfg1, torch.float64)
    big = torch.zeros((5,) + tuple(V.shape[1:]), dtype=torch.float64, device="cuda")
    with pytest.raises(LrdmError) as e:
        ctx.gateaux([big])
    assert e.value.code == 1
    bad = dict(cfg1)
    bad["n_electrons"] = 1000.0
    with pytest.raises(LrdmError) as e:
        make_context([bad], "fp64", torch.float64)
    assert e.value.code == 5
    # K = 0 is a no-op
    F, dmu = ctx.gateaux([V[:0]])
    assert F[0].shape[0] == 0


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_backward_vs_oracle(lib, prec):
    cfg = _ragged(cfg_id=22, n=(12, 10, 14), ns=70, K=3, ne=50)
    io = IO[prec]
    ctx, V, F, dmu = _run([cfg], prec)
    rng = workloads.rng_for(22, 9)
    fbar = rng.standard_normal(cfg["V"].shape)
    vbar, eb, ob = ctx.backward([torch.as_tensor(fbar, dtype=io, device="cuda")])
    torch.cuda.synchronize()
    osys = oracle_system(cfg)
    ref = oracle.backward(osys, fbar, V=cfg["V"])
    tol = gate(prec, "backward_vs_oracle")
    assert per_direction_rel_err(vbar[0].double().cpu().numpy(), ref["vbar"]) < tol
    assert rel_err(eb[0].cpu().numpy(), ref["eps_bar"][0]) < tol * 10
    assert rel_err(ob[0].cpu().numpy(), ref["occ_bar"][0]) < tol * 10


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_recursive_fermi_response(lib, prec):
    """fermi_T = 8: the device's closed-form Loewner matrix of f_T against the
    oracle's perturbed recursion (Eq. recursiveFermiOperator), forward and the
    v-adjoint; eigenvalue / occupation gradients are refused in this mode."""
    from gpu_helpers import directions, make_context
    from paper_2211_07894_gb300 import LrdmError
    cfg = _ragged(cfg_id=23, n=(16, 18, 14), ns=150, K=4, ne=110, kT=0.01)
    io = IO[prec]
    ctx, _ = make_context([cfg], prec, io, fermi_T=8)
    V = directions(cfg, io)
    (F,), dmu = ctx.gateaux([V])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    osys = oracle_system(cfg)
    osys.fermi_T = 8
    ref = oracle.gateaux(osys, cfg["V"])
    err = per_direction_rel_err(F.double().cpu().numpy(), ref["F"])
    print(f"fermi_T=8 {prec}: f rel err {err:.2e}")
    check(prec, "recursive_fermi_response", err)
    # the recursion at depth 8 differs from Fermi-Dirac by far more than the tolerance
    full = oracle.gateaux(oracle_system(cfg), cfg["V"])
    assert per_direction_rel_err(ref["F"], full["F"]) > 100 * TOL["fp64"]
    fbar = workloads.rng_for(23, 9).standard_normal(cfg["V"].shape)
    vbar, _, _ = ctx.backward([torch.as_tensor(fbar, dtype=io, device="cuda")], want_eps=False)
    torch.cuda.synchronize()
    bref = oracle.backward(osys, fbar, ref)
    check(prec, "recursive_fermi_response", per_direction_rel_err(vbar[0].double().cpu().numpy(), bref["vbar"]))
    with pytest.raises(LrdmError) as e:
        ctx.backward([torch.as_tensor(fbar, dtype=io, device="cuda")], want_eps=True)
    assert e.value.code == 9          # LRDM_ERR_UNSUPPORTED
    # eigenvalues outside the recursion's window |eps - mu| < kT 2^(T+1) are refused
    with pytest.raises(LrdmError) as e:
        make_context([cfg], prec, io, fermi_T=3)
    assert e.value.code == 1


@pytest.mark.parametrize("prec,spin", [("fp64", False), ("fp64", True), ("bf16x3", False)])
def test_krylov_step(lib, cfg1, prec, spin):
    """lrdm_krylov_step against the oracle's LRDM step (§II.B): same rank,
    directions, derivatives, coefficients and updated density."""
    from gpu_helpers import make_context
    io = IO[prec]
    if spin:
        cfg = workloads.spin_pair_system(98, (10, 9, 8), 40, 36, 60.0, 0.01, 1)
    else:
        cfg = cfg1
    osys = oracle_system(cfg)
    R = np.asarray(cfg["R"], dtype=np.float64)
    ref = oracle.lrdm_krylov_step(osys, R, s_tol=1e-12, r_max=4)
    # a tolerance between the s_rel of ranks 2 and 3 makes the adaptive stop at 3
    s_tol = 0.5 * (ref["s_rel"][1] + ref["s_rel"][2])
    ref = oracle.lrdm_krylov_step(osys, R, s_tol=s_tol, r_max=4, rho=np.stack(osys.rho))
    ctx, _ = make_context([cfg], prec, io, k_max=1)
    rho = torch.as_tensor(np.stack(osys.rho), dtype=io, device="cuda")
    out = ctx.krylov_step(torch.as_tensor(R, dtype=io, device="cuda"), s_tol=s_tol, r_max=4, rho=rho)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert out["rank"] == ref["rank"] == 3
    tol = gate(prec, "krylov_step")
    # ||R|| of the io-dtype copy of R (FP32 rounding of R in the mixed modes)
    assert abs(out["r_norm"] - ref["r_norm"]) <= (1e-12 if io == torch.float64 else 1e-6) * ref["r_norm"]
    assert np.allclose(out["s_rel"], ref["s_rel"], rtol=10 * tol, atol=0)
    assert per_direction_rel_err(out["U"].double().cpu().numpy(), ref["U"]) < 10 * tol
    assert per_direction_rel_err(out["T"].double().cpu().numpy(), ref["T"]) < 10 * tol
    assert np.allclose(out["a"].cpu().numpy(), ref["a"], rtol=100 * tol, atol=0)
    assert rel_err(rho.double().cpu().numpy() - np.stack(osys.rho),
                   ref["rho_new"] - np.stack(osys.rho)) < 100 * tol


def test_autograd_function_dot_product(lib, cfg1):
    from gpu_helpers import directions, make_context
    from paper_2211_07894_gb300 import gateaux_function
    ctx, _ = make_context([cfg1], "fp64", torch.float64)
    V = directions(cfg1, torch.float64).requires_grad_(True)
    fbar = torch.randn_like(V)
    F = gateaux_function().apply(ctx, V)
    (F * fbar).sum().backward()
    lhs = float((fbar * F.detach()).sum())
    rhs = float((V.grad * V.detach()).sum())
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16x3"])
def test_maximum_directions(lib, prec):
    """K = k_max = 64 (the largest batch a call takes) on a ragged system:
    forward, the least-squares step over all 64 derivatives and the adjoint
    against the oracle."""
    cfg = _ragged(cfg_id=23, n=(12, 10, 14), ns=70, K=64, ne=50)
    io = IO[prec]
    ctx, V, F, dmu = _run([cfg], prec)
    osys = oracle_system(cfg)
    ref = oracle.gateaux(osys, cfg["V"])
    err = per_direction_rel_err(F[0], ref["F"])
    print(f"K = 64 {prec}: f err {err:.3e}")
    check(prec, "maximum_directions", err)
    _check_dmu(dmu, ref, prec, "maximum_directions")
    Fd = torch.as_tensor(ref["F"], dtype=io, device="cuda")
    R = torch.as_tensor(cfg["R"], dtype=io, device="cuda")
    coef, srel = ctx.apply(0, R, V[0], Fd, 0.5)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    want = oracle.lrdm_apply(cfg["R"], cfg["V"], ref["F"], osys.w, 0.5)
    tol = 1e-10 if prec == "fp64" else 1e-5
    # a = S^+ c with cond(S) ~ 1e4: the coefficients carry the io rounding times cond(S)
    assert rel_err(coef.cpu().numpy(), want["a"]) < (1e-8 if prec == "fp64" else 1e-2)
    assert abs(srel.item() - want["s_rel"]) < tol * 10
    if prec != "tf32":
        fbar = workloads.rng_for(23, 9).standard_normal(cfg["V"].shape)
        vbar, _, _ = ctx.backward([torch.as_tensor(fbar, dtype=io, device="cuda")])
        torch.cuda.synchronize()
        assert ctx.status() == 0
        vref = oracle.backward(osys, fbar, V=cfg["V"])["vbar"]
        check(prec, "maximum_directions", per_direction_rel_err(vbar[0].double().cpu().numpy(), vref))


@pytest.mark.parametrize("prec,bn", [("bf16x3", 256), ("bf16x3", 128), ("tf32", 256)])
def test_response_split_over_j_tiles(lib, prec, bn, tmp_path, monkeypatch):
    """N_s = 2048 on a ragged grid (2464 rows): with K = 1 the response
    items are split into 4 parts over their j-tiles, whose FP64 part sums a
    second kernel adds in order; K = 2 and 4 run unsplit.  All three against
    the oracle, and K = 1 and 2 against the same directions of K = 4."""
    from gpu_helpers import directions, make_context
    cfg = _ragged(cfg_id=24, n=(16, 14, 11), ns=2048, K=4, ne=1800)
    io = IO[prec]
    code = {"tf32": 2, "bf16x3": 3}[prec]
    cache = tmp_path / "tune.jsonl"
    cache.write_text('{"key": "%s", "g1_nb": 256, "g1_dpt": 1, "g2_bn": %d, "g2_kgroup": 4}\n'
                     % (_tune_key([cfg], code), bn))
    monkeypatch.setenv("LRDM_TUNE_CACHE", str(cache))
    ctx, _ = make_context([cfg], prec, io, autotune=True)
    assert ctx.tuning()["g2_bn"] == bn
    V = directions(cfg, io)
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    out = {}
    for K in (1, 2, 4):
        F, _ = ctx.gateaux([V[:K].contiguous()])
        torch.cuda.synchronize()
        assert ctx.status() == 0
        out[K] = F[0].double().cpu().numpy()
        err = per_direction_rel_err(out[K], ref["F"][:K])
        print(f"N_s 2048 {prec} bn {bn} K = {K}: f err {err:.3e}")
        check(prec, "response_split_over_j_tiles", err)
    # same projections up to FP32 rounding of the grid reduction: the split
    # response agrees with the unsplit one far inside the tolerance
    for K in (1, 2):
        d = per_direction_rel_err(out[K], out[4][:K])
        print(f"response split {prec} K = {K} vs the same directions at K = 4: {d:.2e}")
        assert d < 0.1 * gate(prec, "response_split_over_j_tiles")


# --- projection on CTA pairs (256 x 256 tiles, pair MMAs) -------------------

PAIR_CASES = {
    # (cfg_id, grid, N_s, K, N_e): padded N_s 256 (one pair tile), 384 (three
    # 128-blocks: the odd CTA of the last tile row and column reads zero fill),
    # 640 (five blocks, three 256-columns)
    "ns200": (30, (20, 18, 22), 200, 5, 150),
    "ns300": (31, (18, 16, 20), 300, 3, 230),
    "ns640": (32, (24, 22, 20), 640, 4, 500),
}


@pytest.mark.parametrize("case", sorted(PAIR_CASES))
@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_pair_projection_tiles(lib, prec, case):
    """The pair-tile projection (lrdm_set_tuning g1_nb = 512) against the
    oracle on X_k (every entry) and f_k, on tile counts that leave the odd CTA
    of a pair outside the matrix; the single-CTA 128 x 256 form on the same
    context gives the same X within the precision's tolerance."""
    from gpu_helpers import directions, make_context
    cid, n, ns, K, ne = PAIR_CASES[case]
    cfg = _ragged(cfg_id=cid, n=n, ns=ns, K=K, ne=ne)
    io = IO[prec]
    ctx, _ = make_context([cfg], prec, io)
    ctx.set_tuning(g1_nb=512, g1_dpt=1)
    assert ctx.tuning()["g1_nb"] == 512
    V = directions(cfg, io)
    (F,), dmu = ctx.gateaux([V])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    Xp = [ctx.projection(k).cpu().numpy() for k in range(K)]
    errs = [rel_err(Xp[k], ref["X"][0][k]) for k in range(K)]
    err = per_direction_rel_err(F.double().cpu().numpy(), ref["F"])
    print(f"pair tiles {prec} {case}: X err {max(errs):.2e}, f err {err:.2e}")
    check(prec, "pair_projection_tiles", max(errs), "X")
    check(prec, "pair_projection_tiles", err)
    _check_dmu(dmu.cpu().numpy(), ref, prec, "pair_projection_tiles")
    ctx.set_tuning(g1_nb=256, g1_dpt=1)
    ctx.gateaux([V])
    torch.cuda.synchronize()
    for k in range(K):
        Xs = ctx.projection(k).cpu().numpy()
        assert np.max(np.abs(Xs - Xp[k])) <= gate(prec, "pair_projection_tiles", "X") * np.max(np.abs(Xs))


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_pair_projection_small_k_and_batch(lib, prec):
    """Pair tiles with a one-direction call (grid-row ranges chosen over CTA
    pairs, partial X summed by the consumers) and in one grouped launch over
    the uneven batch with its spin pair: oracle tolerance, and the batch equals
    separate calls bit for bit."""
    from gpu_helpers import directions, make_context
    io = IO[prec]
    cfg = _ragged(cfg_id=33, n=(40, 40, 40), ns=512, K=8, ne=400)
    ctx, _ = make_context([cfg], prec, io)
    ctx.set_tuning(g1_nb=512, g1_dpt=1)
    one = directions(cfg, io)[2:3].contiguous()
    (F1,), dmu1 = ctx.gateaux([one])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"][2:3])
    check(prec, "pair_projection_small_k_and_batch", rel_err(ctx.projection(0).cpu().numpy(), ref["X"][0][0]), "X")
    check(prec, "pair_projection_small_k_and_batch", per_direction_rel_err(F1.double().cpu().numpy(), ref["F"]))
    cfgs = workloads.config3(scale=8)
    bctx, _ = make_context(cfgs, prec, io)
    bctx.set_tuning(g1_nb=512, g1_dpt=1)
    V = [directions(c, io) for c in cfgs]
    F, _ = bctx.gateaux(V)
    torch.cuda.synchronize()
    assert bctx.status() == 0
    for i, c in enumerate(cfgs):
        sep, _ = make_context([c], prec, io)
        sep.set_tuning(g1_nb=512, g1_dpt=1)
        (Fi,), _ = sep.gateaux([V[i]])
        assert torch.equal(Fi, F[i])
        ref = oracle.gateaux(oracle_system(c), c["V"])
        err = per_direction_rel_err(F[i].double().cpu().numpy(), ref["F"])
        print(f"pair tiles batched system {i} {prec}: f err {err:.2e}")
        check(prec, "pair_projection_small_k_and_batch", err)


def test_set_tuning_rejects_bad_shapes(lib, cfg1):
    from gpu_helpers import make_context
    from paper_2211_07894_gb300 import binding
    ctx, _ = make_context([cfg1], "bf16x3", torch.float32)
    for bad in [(384, 1, 256, 4), (256, 2, 256, 4), (512, 2, 256, 4), (256, 1, 192, 4), (256, 1, 256, 3),
                (256, 1, 1024, 4)]:
        assert binding.lrdm_set_tuning(ctx.handle, *bad) == 1      # LRDM_ERR_INVALID_ARG
    f64, _ = make_context([cfg1], "fp64", torch.float64)
    assert binding.lrdm_set_tuning(f64.handle, 256, 1, 256, 4) == 9   # LRDM_ERR_UNSUPPORTED


# --- response on CTA pairs (256-row blocks, 256-wide j-tiles) ---------------

@pytest.mark.parametrize("case", sorted(PAIR_CASES))
@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_pair_response_tiles(lib, prec, case):
    """The pair-tile response (lrdm_set_tuning g2_bn = 512) against the
    oracle on f and drho: grids whose row blocks are odd in number (the odd
    CTA of the last pair reads zero fill) and padded N_s = 384 (the odd
    CTA's half of the last j-tile lies outside the matrix); the single-CTA
    response on the same context agrees within the precision's tolerance."""
    from gpu_helpers import directions, make_context
    cid, n, ns, K, ne = PAIR_CASES[case]
    cfg = _ragged(cfg_id=cid, n=n, ns=ns, K=K, ne=ne)
    io = IO[prec]
    ctx, _ = make_context([cfg], prec, io)
    ctx.set_tuning(g1_nb=512, g2_bn=512)
    V = directions(cfg, io)
    (F,), dmu = ctx.gateaux([V])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    Fh = F.double().cpu().numpy()
    check(prec, "pair_response_tiles", per_direction_rel_err(Fh, ref["F"]))
    check(prec, "pair_response_tiles", per_direction_rel_err(Fh + cfg["V"], ref["drho"]), "X")
    ctx.set_tuning(g2_bn=256)
    (F2,), _ = ctx.gateaux([V])
    torch.cuda.synchronize()
    d = per_direction_rel_err(F2.double().cpu().numpy(), Fh)
    print(f"pair response {prec} {case}: vs single-CTA response {d:.2e}")
    assert d < gate(prec, "pair_response_tiles")


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_pair_response_split_and_batch(lib, prec):
    """The pair response with one direction at N_s = 2048 (items split into
    j-tile parts, FP64 part sums added by the combine kernel) and over the
    uneven batch with its spin pair (grouped launch); oracle tolerance, and
    the batch equals separate calls bit for bit."""
    from gpu_helpers import directions, make_context
    io = IO[prec]
    cfg = _ragged(cfg_id=24, n=(16, 14, 11), ns=2048, K=2, ne=1800)
    ctx, _ = make_context([cfg], prec, io)
    ctx.set_tuning(g2_bn=512)
    V = directions(cfg, io)
    (F1,), _ = ctx.gateaux([V[:1].contiguous()])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"][:1])
    check(prec, "pair_response_split_and_batch", per_direction_rel_err(F1.double().cpu().numpy(), ref["F"]))
    cfgs = workloads.config3(scale=8)
    bctx, _ = make_context(cfgs, prec, io)
    bctx.set_tuning(g2_bn=512)
    Vb = [directions(c, io) for c in cfgs]
    F, _ = bctx.gateaux(Vb)
    torch.cuda.synchronize()
    assert bctx.status() == 0
    for i, c in enumerate(cfgs):
        sep, _ = make_context([c], prec, io)
        sep.set_tuning(g2_bn=512)
        (Fi,), _ = sep.gateaux([Vb[i]])
        assert torch.equal(Fi, F[i])
        refc = oracle.gateaux(oracle_system(c), c["V"])
        check(prec, "pair_response_split_and_batch", per_direction_rel_err(F[i].double().cpu().numpy(), refc["F"]))
