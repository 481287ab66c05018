"""Grid-row-sharded contexts (lrdm_create_rows) on one GPU: two "ranks" in two
host threads, each holding a slab of the grid's rows of Psi in its own
context and stream, with the library's collective steps summed by a host-side
rendezvous of the two threads (the kernels of the two contexts never wait on
each other; only the host threads meet between launches).

Checked against one unsharded context on the same system, and against the
FP64 oracle: the forward (Eq. densityResponse per row, with X_k the sum of
the slabs' projections), the least-squares step (Eqs. plowrank,
relativeError: the same coefficients and s_rel on every rank) and the
adjoint, and the drivers (the adaptive-rank LRDM step and LRDMA) whose
norms, Gram-Schmidt inner products and least-squares sums run over the
ranks; a failing collective returns LRDM_ERR_COLLECTIVE.
"""

import threading

import numpy as np
import pytest

import oracle
import workloads
from gates import TOL
from helpers import oracle_system, per_direction_rel_err

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

IO = {"fp64": torch.float64, "bf16x3": torch.float32}


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build
    build.build()


class ThreadSum:
    """In-place sum over `n` host threads (one per rank): each rank's buffer is
    complete on its stream, both are read after a first rendezvous, the sum
    (rank 0's buffer plus rank 1's, the same order for both) is written back
    after a second one."""

    def __init__(self, n):
        self.bar = threading.Barrier(n, timeout=120)
        self.slots = [None] * n
        self.calls = [0] * n

    def member(self, r):
        def fn(t, st):
            st.synchronize()
            self.slots[r] = t
            self.calls[r] += 1
            self.bar.wait()
            total = self.slots[0].clone()
            for x in self.slots[1:]:
                total += x
            torch.cuda.current_stream().synchronize()
            self.bar.wait()
            t.copy_(total)
            torch.cuda.current_stream().synchronize()
        return fn


def _system(cfg, io, rows=None):
    from gpu_helpers import to_device_system
    c = dict(cfg)
    if rows is not None:
        r0, r1 = rows
        c["psi"] = [p[r0:r1] for p in cfg["psi"]]
    return to_device_system(c, io)


def _run_ranks(fns):
    """Runs fns[r]() on its own thread; returns their results (re-raises)."""
    out, err = [None] * len(fns), []

    def work(r):
        try:
            out[r] = fns[r]()
        except Exception as e:          # noqa: BLE001
            err.append(e)

    th = [threading.Thread(target=work, args=(r,)) for r in range(len(fns))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    return out


@pytest.mark.parametrize("prec,cut", [("fp64", 3001), ("bf16x3", 3001), ("bf16x3", 3960)])
def test_row_sharded_step_matches_unsharded(lib, prec, cut):
    from paper_2211_07894_gb300 import Context
    io = IO[prec]
    cfg = workloads.random_system(71, (20, 18, 22), 200, 150, 0.01, 5)
    ng = int(np.prod(cfg["n"]))
    bounds = [(0, cut), (cut, ng)]
    V = torch.as_tensor(cfg["V"], dtype=io, device="cuda")
    R = torch.as_tensor(cfg["R"], dtype=io, device="cuda")
    fbar = torch.as_tensor(workloads.rng_for(71, 9).standard_normal(cfg["V"].shape), dtype=io,
                           device="cuda")
    # the unsharded reference on the same system
    full = Context([_system(cfg, io)], prec=prec, io_dtype=io, k_max=5)
    (F,), dmu = full.gateaux([V])
    vbar, eb, ob = full.backward([fbar])
    torch.cuda.synchronize()
    assert full.status() == 0
    F_ref = F.double().cpu().numpy()
    vbar_ref = vbar[0].double().cpu().numpy()
    eb_ref = eb[0].cpu().numpy()
    rho0 = torch.full_like(R, 0.01)

    ts = ThreadSum(2)

    def rank(r):
        r0, r1 = bounds[r]
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = Context([_system(cfg, io, (r0, r1))], prec=prec, io_dtype=io, k_max=5,
                          rows=dict(row_begin=r0, n_rows=r1 - r0, allreduce=ts.member(r)))
            Vs = V[:, :, r0:r1].contiguous()
            Rs = R[:, r0:r1].contiguous()
            (Fs,), dmus = ctx.gateaux([Vs])
            rho_s = rho0[:, r0:r1].clone()      # a copy (the slice of one row is contiguous)
            c_s, s_s = ctx.apply(0, Rs, Vs, Fs, 0.5, rho=rho_s)
            vb_s, eb_s, ob_s = ctx.backward([fbar[:, :, r0:r1].contiguous()])
            st.synchronize()
            code = ctx.status()
            ctx.close()
        return dict(F=Fs.double().cpu().numpy(), dmu=dmus.cpu().numpy(), coef=c_s.cpu().numpy(),
                    srel=float(s_s.item()), rho=rho_s.double().cpu().numpy(),
                    vbar=vb_s[0].double().cpu().numpy(), eb=eb_s[0].cpu().numpy(),
                    ob=ob_s[0].cpu().numpy(), code=code)

    out = _run_ranks([lambda: rank(0), lambda: rank(1)])
    assert [o["code"] for o in out] == [0, 0]
    assert ts.calls[0] == ts.calls[1] == 6    # forward 2, least squares 2, adjoint 2
    # quantities reduced over the ranks come out identical on both
    for key in ("dmu", "coef", "eb", "ob"):
        assert np.array_equal(out[0][key], out[1][key]), key
    assert out[0]["srel"] == out[1]["srel"]
    Fs = np.concatenate([o["F"] for o in out], axis=-1)
    vbs = np.concatenate([o["vbar"] for o in out], axis=-1)
    rhos = np.concatenate([o["rho"] for o in out], axis=-1)
    tol = 1e-12 if prec == "fp64" else 1e-6
    err_f = per_direction_rel_err(Fs, F_ref)
    err_vb = per_direction_rel_err(vbs, vbar_ref)
    print(f"rows {prec} cut {cut}: f vs unsharded {err_f:.2e}, vbar {err_vb:.2e}")
    assert err_f < tol and err_vb < tol
    dmu_ref = dmu.cpu().numpy()    # mu' is a weighted mean of X_ii: its error scales with max |mu'|
    assert np.allclose(out[0]["dmu"], dmu_ref, rtol=tol * 10, atol=tol * 10 * np.abs(dmu_ref).max())
    assert np.allclose(out[0]["eb"], eb_ref, rtol=tol * 100, atol=tol * np.abs(eb_ref).max())
    # the least-squares step on the same derivatives (the sharded ones), unsharded:
    # the ranks' sums differ from it only in the order of the FP64 grid sums
    rho_ref = rho0.clone()
    coef, srel = full.apply(0, R, V, torch.as_tensor(Fs, dtype=io, device="cuda"), 0.5, rho=rho_ref)
    torch.cuda.synchronize()
    assert np.allclose(out[0]["coef"], coef.cpu().numpy(), rtol=1e-9, atol=1e-12)
    assert abs(out[0]["srel"] - srel.item()) < 1e-10
    assert np.allclose(rhos, rho_ref.double().cpu().numpy(), rtol=1e-9, atol=1e-14)
    # and the sharded forward against the FP64 oracle at the stated tolerance
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    assert per_direction_rel_err(Fs, ref["F"]) < TOL[prec]


def test_row_sharded_failures(lib):
    from paper_2211_07894_gb300 import Context, LrdmError
    cfg = workloads.random_system(72, (12, 10, 14), 70, 50, 0.01, 3)
    ng = int(np.prod(cfg["n"]))
    V = torch.as_tensor(cfg["V"], dtype=torch.float64, device="cuda")

    def failing(t, st):
        raise RuntimeError("collective failed (test)")

    ctx = Context([_system(cfg, torch.float64, (0, ng))], prec="fp64", io_dtype=torch.float64,
                  k_max=3, rows=dict(row_begin=0, n_rows=ng, allreduce=failing))
    with pytest.raises(LrdmError) as e:
        ctx.gateaux([V])
    assert e.value.code == 10                 # LRDM_ERR_COLLECTIVE
    torch.cuda.synchronize()
    # a one-rank group (the callback leaves the buffer as it is) equals the plain
    # context up to the order of the grid sums (one partial X against the
    # plain context's row ranges)
    solo = Context([_system(cfg, torch.float64, (0, ng))], prec="fp64", io_dtype=torch.float64,
                   k_max=3, rows=dict(row_begin=0, n_rows=ng, allreduce=lambda t, st: None))
    plain = Context([_system(cfg, torch.float64)], prec="fp64", io_dtype=torch.float64, k_max=3)
    (F1,), _ = solo.gateaux([V])
    (F2,), _ = plain.gateaux([V])
    torch.cuda.synchronize()
    assert per_direction_rel_err(F1.cpu().numpy(), F2.cpu().numpy()) < 1e-13
    # rows outside the grid are refused before anything is allocated
    with pytest.raises(LrdmError) as e:
        Context([_system(cfg, torch.float64, (0, 10))], prec="fp64", io_dtype=torch.float64,
                k_max=3, rows=dict(row_begin=ng - 5, n_rows=10, allreduce=lambda t, st: None))
    assert e.value.code == 2                  # LRDM_ERR_SHAPE
    for c in (ctx, solo, plain):
        c.close()


def test_row_sharded_drivers_match_unsharded(lib):
    """lrdm_krylov_step and lrdm_lrdma_step on two row slabs (FP64): rank,
    s_rel, coefficients, directions and the density update against one
    unsharded context."""
    from paper_2211_07894_gb300 import Context, Lrdma
    io = torch.float64
    cfg = workloads.random_system(73, (20, 18, 22), 200, 150, 0.01, 1)
    ng = int(np.prod(cfg["n"]))
    w = float(np.prod(cfg["h"]))
    cut = 3001
    bounds = [(0, cut), (cut, ng)]
    R = torch.as_tensor(cfg["R"], dtype=io, device="cuda")
    rho0 = torch.full_like(R, 0.01)
    full = Context([_system(cfg, io)], prec="fp64", io_dtype=io, k_max=8)
    rho_k = rho0.clone()
    ref = full.krylov_step(R, s_tol=0.05, r_max=6, alpha=0.5, rho=rho_k)
    la = Lrdma(n=ng, io_dtype=io, w=w, capacity=8)
    rho_l = rho0.clone()
    rep = la.step(full, R, rho_l, s_tol=0.05, r_max=6)
    torch.cuda.synchronize()
    ts = ThreadSum(2)

    def rank(r):
        r0, r1 = bounds[r]
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = Context([_system(cfg, io, (r0, r1))], prec="fp64", io_dtype=io, k_max=8,
                          rows=dict(row_begin=r0, n_rows=r1 - r0, allreduce=ts.member(r)))
            Rs = R[:, r0:r1].clone()
            rk = rho0[:, r0:r1].clone()
            step = ctx.krylov_step(Rs, s_tol=0.05, r_max=6, alpha=0.5, rho=rk)
            lr = Lrdma(n=r1 - r0, io_dtype=io, w=w, capacity=8)
            rl = rho0[:, r0:r1].clone()
            rp = lr.step(ctx, Rs, rl, s_tol=0.05, r_max=6)
            st.synchronize()
            code = ctx.status()
            ctx.close()
        return dict(rank=step["rank"], a=step["a"].cpu().numpy(), U=step["U"].cpu().numpy(),
                    s_rel=np.asarray(step["s_rel"]), rho_k=rk.cpu().numpy(), rep=rep_dict(rp),
                    rho_l=rl.cpu().numpy(), code=code)

    def rep_dict(x):
        return {k: x[k] for k in ("event", "rank", "s_rel")} if isinstance(x, dict) else x

    out = _run_ranks([lambda: rank(0), lambda: rank(1)])
    assert [o["code"] for o in out] == [0, 0]
    for o in out:
        assert o["rank"] == ref["rank"]
        assert np.allclose(o["a"], ref["a"].cpu().numpy(), rtol=1e-9, atol=1e-12)
        assert np.allclose(o["s_rel"], np.asarray(ref["s_rel"]), rtol=1e-9, atol=1e-12)
    assert np.array_equal(out[0]["a"], out[1]["a"])
    U = np.concatenate([o["U"] for o in out], axis=-1)
    assert np.allclose(U, ref["U"].cpu().numpy(), rtol=1e-9, atol=1e-10)
    rho = np.concatenate([o["rho_k"] for o in out], axis=-1)
    assert np.allclose(rho, rho_k.cpu().numpy(), rtol=1e-10, atol=1e-14)
    # LRDMA's first step (a fresh build) and its density update
    assert out[0]["rep"] == out[1]["rep"]
    ref_rep = rep_dict(rep)
    assert out[0]["rep"]["event"] == ref_rep["event"] and out[0]["rep"]["rank"] == ref_rep["rank"]
    assert abs(out[0]["rep"]["s_rel"] - ref_rep["s_rel"]) < 1e-10
    rho = np.concatenate([o["rho_l"] for o in out], axis=-1)
    assert np.allclose(rho, rho_l.cpu().numpy(), rtol=1e-10, atol=1e-14)
    full.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_row_sharded_spin_pair(lib, prec):
    """A collinear spin pair (two channels sharing mu and the Hartree term)
    on two row slabs: f, mu' and the least-squares step against one
    unsharded context and the oracle."""
    from paper_2211_07894_gb300 import Context
    io = IO[prec]
    cfg = workloads.spin_pair_system(74, (16, 14, 18), 120, 100, 90, 0.01, 3)
    ng = int(np.prod(cfg["n"]))
    bounds = [(0, 1501), (1501, ng)]
    V = torch.as_tensor(cfg["V"], dtype=io, device="cuda")
    R = torch.as_tensor(cfg["R"], dtype=io, device="cuda")
    full = Context([_system(cfg, io)], prec=prec, io_dtype=io, k_max=3)
    (F,), dmu = full.gateaux([V])
    torch.cuda.synchronize()
    ts = ThreadSum(2)

    def rank(r):
        r0, r1 = bounds[r]
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = Context([_system(cfg, io, (r0, r1))], prec=prec, io_dtype=io, k_max=3,
                          rows=dict(row_begin=r0, n_rows=r1 - r0, allreduce=ts.member(r)))
            Vs = V[:, :, r0:r1].contiguous()
            (Fs,), dmus = ctx.gateaux([Vs])
            c_s, s_s = ctx.apply(0, R[:, r0:r1].contiguous(), Vs, Fs, 0.0)
            st.synchronize()
            code = ctx.status()
            ctx.close()
        return dict(F=Fs.double().cpu().numpy(), dmu=dmus.cpu().numpy(), coef=c_s.cpu().numpy(),
                    srel=float(s_s.item()), code=code)

    out = _run_ranks([lambda: rank(0), lambda: rank(1)])
    assert [o["code"] for o in out] == [0, 0]
    assert np.array_equal(out[0]["coef"], out[1]["coef"]) and out[0]["srel"] == out[1]["srel"]
    Fs = np.concatenate([o["F"] for o in out], axis=-1)
    tol = 1e-12 if prec == "fp64" else 1e-6
    err = per_direction_rel_err(Fs, F.double().cpu().numpy())
    print(f"rows spin {prec}: f vs unsharded {err:.2e}")
    assert err < tol
    dmu_ref = dmu.cpu().numpy()
    assert np.allclose(out[0]["dmu"], dmu_ref, rtol=tol * 10, atol=tol * 10 * np.abs(dmu_ref).max())
    coef, srel = full.apply(0, R, V, torch.as_tensor(Fs, dtype=io, device="cuda"), 0.0)
    torch.cuda.synchronize()
    assert np.allclose(out[0]["coef"], coef.cpu().numpy(), rtol=1e-9, atol=1e-12)
    assert abs(out[0]["srel"] - srel.item()) < 1e-10
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    assert per_direction_rel_err(Fs, ref["F"]) < TOL[prec]
    full.close()
