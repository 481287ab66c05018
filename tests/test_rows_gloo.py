"""Grid-row partition of one system over two CPU ranks (gloo), with the FP64
oracle's steps on each rank's rows: the steps a row-sharded context
(lrdm_create_rows) takes on the device, in the same order, with the same
exchanges.  Each rank holds rows [r0, r1) of Psi; the directions' rows are
written into a zeroed full-grid buffer and summed over the ranks (the
all-gather the replicated Poisson solve needs); the slabs' projections
X_k = Psi_slab^T diag(w dV_k) Psi_slab are summed over the ranks; mu'_k and
the subspace response follow from the summed X_k on every rank; drho_k and
f_k are row-local (Eq. densityResponse); the least-squares sums S, c and
||R||^2 and the residual sum behind s_rel are summed over the ranks (Eqs.
plowrank, relativeError).  The gathered result must equal the oracle on the
whole grid."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

# restricted: seed, grid, N_s, N_e, kT, K; spin pair: seed, grid, N_s up / down, N_e, kT, K
CASES = {"restricted": ("random", 41, (8, 8, 9), 30, 20.0, 0.02, 4),
         "spin": ("spin", 42, (8, 8, 8), (24, 20), 22.0, 0.02, 3)}
CUTS = {"restricted": [0, 229, 576], "spin": [0, 301, 512]}     # ragged slabs of the rows


def _case(name):
    import workloads
    kind, seed, n, ns, ne, kT, K = CASES[name]
    if kind == "random":
        return workloads.random_system(seed, n, ns, ne, kT, K)
    return workloads.spin_pair_system(seed, n, ns[0], ns[1], ne, kT, K)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sum(x):
    t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _worker(rank, world, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        here = os.path.dirname(os.path.abspath(__file__))
        sys.path.insert(0, here)
        sys.path.insert(0, os.path.dirname(here))
        import oracle
        from helpers import oracle_system
        cfg = _case(name)
        osys = oracle_system(cfg)
        n = cfg["n"]
        ng = int(np.prod(n))
        nspin = osys.nspin
        K = cfg["V"].shape[0]
        r0, r1 = CUTS[name][rank], CUTS[name][rank + 1]
        psi = [p[r0:r1] for p in osys.psi]             # this rank's rows of Psi per channel
        w, g = osys.w, osys.occ_factor
        v = cfg["V"][:, :, r0:r1]                      # this rank's rows of the directions
        R = cfg["R"][:, r0:r1]
        mu = oracle.solve_mu(osys.eps, osys.n_electrons, osys.kT, g)
        L = [oracle.loewner(e, mu, osys.kT) for e in osys.eps]
        fx = [oracle.lda_fx(rh[r0:r1], spin_polarized=nspin == 2) for rh in osys.rho]
        # the spin-summed directions on the whole grid: each rank's rows into zeros, summed
        full = np.zeros((K, ng))
        full[:, r0:r1] = v.sum(axis=1)
        full = _sum(full)
        F = np.zeros_like(v)
        dmu = np.zeros(K)
        for k in range(K):
            vh = oracle.hartree(full[k], n, osys.h)       # replicated Poisson solve
            X = [_sum(oracle.project(psi[c], w * (vh[r0:r1] + fx[c] * v[k, c])))
                 for c in range(nspin)]                  # the slabs' projections, summed
            dmu[k] = oracle.dmu_shift(L, X)
            for c in range(nspin):
                Xp = oracle.subspace_response(L[c], X[c], dmu[k])
                F[k, c] = oracle.density_response(psi[c], Xp, g) - v[k, c]
        # least squares: grid sums (both channels) over the ranks, the same K x K solve on each
        Fm, Rm, Vm = F.reshape(K, -1), R.ravel(), v.reshape(K, -1)
        S = _sum(w * Fm @ Fm.T)
        c_ = _sum(w * Fm @ Rm)
        r2 = float(_sum(np.array([w * Rm @ Rm]))[0])
        lam, Q = np.linalg.eigh(S)
        keep = lam > 1e-12 * lam.max()
        a = Q[:, keep] @ ((Q[:, keep].T @ c_) / lam[keep])
        res = Fm.T @ a - Rm
        s_rel = float(np.sqrt(_sum(np.array([w * res @ res]))[0] / r2))
        rho = np.stack([rh[r0:r1] for rh in osys.rho])
        rho_new = rho - 0.5 * (Vm.T @ a).reshape(rho.shape)
        out[rank] = (F, dmu, a, s_rel, rho_new)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["restricted", "spin"])
def test_row_partition_matches_whole_grid(name):
    import oracle
    from helpers import oracle_system
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, name, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    cfg = _case(name)
    osys = oracle_system(cfg)
    ref = oracle.gateaux(osys, cfg["V"])
    step = oracle.lrdm_apply(cfg["R"], cfg["V"], ref["F"], osys.w, 0.5, rho=np.stack(osys.rho))
    F = np.concatenate([res[r][0] for r in range(world)], axis=-1)
    assert np.allclose(F, ref["F"], rtol=0, atol=1e-12 * np.abs(ref["F"]).max())
    for r in range(world):
        _, dmu, a, s_rel, _ = res[r]
        assert np.allclose(dmu, ref["dmu"], rtol=1e-12, atol=1e-14)
        assert np.allclose(a, step["a"], rtol=1e-10)
        assert abs(s_rel - step["s_rel"]) < 1e-12
    # the ranks' reduced quantities agree exactly
    assert np.array_equal(res[0][2], res[1][2]) and res[0][3] == res[1][3]
    rho = np.concatenate([res[r][4] for r in range(world)], axis=-1)
    assert np.allclose(rho, step["rho_new"], rtol=1e-12)
