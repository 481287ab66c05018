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
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

CFG = (41, (8, 8, 9), 30, 20.0, 0.02, 4)       # seed, grid, N_s, N_e, kT, K
CUTS = {2: [0, 229, 576]}                      # ragged slabs of the 576 rows


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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        here = os.path.dirname(os.path.abspath(__file__))
        sys.path.insert(0, here)
        sys.path.insert(0, os.path.dirname(here))
        import oracle
        import workloads
        from helpers import oracle_system
        seed, n, ns, ne, kT, K = CFG
        cfg = workloads.random_system(seed, n, ns, ne, kT, K)
        osys = oracle_system(cfg)
        ng = int(np.prod(n))
        r0, r1 = CUTS[world][rank], CUTS[world][rank + 1]
        psi = osys.psi[0][r0:r1]                       # this rank's rows of Psi
        rho = osys.rho[0][r0:r1]
        w, g = osys.w, osys.occ_factor
        v = cfg["V"][:, 0, r0:r1]                      # this rank's rows of the directions
        R = cfg["R"][0, r0:r1]
        mu = oracle.solve_mu(osys.eps, osys.n_electrons, osys.kT, g)
        L = oracle.loewner(osys.eps[0], mu, osys.kT)
        fx = oracle.lda_fx(rho)
        # the directions on the whole grid: each rank's rows into zeros, summed
        full = np.zeros((K, ng))
        full[:, r0:r1] = v
        full = _sum(full)
        F = np.zeros((K, r1 - r0))
        dmu = np.zeros(K)
        for k in range(K):
            vh = oracle.hartree(full[k], n, osys.h)       # replicated Poisson solve
            dV = vh[r0:r1] + fx * v[k]
            X = _sum(oracle.project(psi, w * dV))         # the slabs' projections, summed
            dmu[k] = oracle.dmu_shift([L], [X])
            Xp = oracle.subspace_response(L, X, dmu[k])
            F[k] = oracle.density_response(psi, Xp, g) - v[k]
        # least squares: grid sums over the ranks, then the same K x K solve on each
        S = _sum(w * F @ F.T)
        c = _sum(w * F @ R)
        r2 = float(_sum(np.array([w * R @ R]))[0])
        lam, Q = np.linalg.eigh(S)
        keep = lam > 1e-12 * lam.max()
        a = Q[:, keep] @ ((Q[:, keep].T @ c) / lam[keep])
        res = F.T @ a - R
        s_rel = float(np.sqrt(_sum(np.array([w * res @ res]))[0] / r2))
        rho_new = rho - 0.5 * (v.T @ a)
        out[rank] = (F, dmu, a, s_rel, rho_new)
    finally:
        dist.destroy_process_group()


def test_row_partition_matches_whole_grid():
    import oracle
    import workloads
    from helpers import oracle_system
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    seed, n, ns, ne, kT, K = CFG
    cfg = workloads.random_system(seed, n, ns, ne, kT, K)
    osys = oracle_system(cfg)
    ref = oracle.gateaux(osys, cfg["V"])
    step = oracle.lrdm_apply(cfg["R"], cfg["V"], ref["F"], osys.w, 0.5, rho=np.stack(osys.rho))
    F = np.concatenate([res[r][0] for r in range(world)], axis=1)
    assert np.allclose(F, ref["F"][:, 0], rtol=0, atol=1e-12 * np.abs(ref["F"]).max())
    for r in range(world):
        _, dmu, a, s_rel, _ = res[r]
        assert np.allclose(dmu, ref["dmu"], rtol=1e-12)
        assert np.allclose(a, step["a"], rtol=1e-10)
        assert abs(s_rel - step["s_rel"]) < 1e-12
    # the ranks' reduced quantities agree exactly
    assert np.array_equal(res[0][2], res[1][2]) and res[0][3] == res[1][3]
    rho = np.concatenate([res[r][4] for r in range(world)])
    assert np.allclose(rho, step["rho_new"][0], rtol=1e-12)
