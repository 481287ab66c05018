"""Direction-sharded evaluation on two CPU ranks (gloo): each rank evaluates
its slice of the directions, the slices are all-gathered and the
least-squares step on the gathered set must equal the single-process one.
The FP64 oracle stands in for the per-rank GPU evaluation: directly, and as
a context-shaped object driven by the library's own sharded_step (slice,
forward, all-gather, least-squares step on every rank)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_07894_gb300.sharding import gather_directions, shard_bounds, sharded_step


def test_shard_bounds_cover_exactly():
    for K in range(0, 20):
        for world in range(1, 6):
            spans = [shard_bounds(K, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == K
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c and b >= a
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


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
        cfg = workloads.random_system(40, (8, 8, 8), 24, 16, 0.02, 5)
        osys = oracle_system(cfg)
        K = cfg["V"].shape[0]
        a, b = shard_bounds(K, world, rank)
        Fl = oracle.gateaux(osys, cfg["V"][a:b])["F"]
        F = gather_directions(torch.as_tensor(Fl), K).numpy()
        V = gather_directions(torch.as_tensor(cfg["V"][a:b]), K).numpy()
        step = oracle.lrdm_apply(cfg["R"], V, F, osys.w, 0.5, rho=np.stack(osys.rho))
        out[rank] = (F, step["a"], step["s_rel"])
    finally:
        dist.destroy_process_group()


def test_direction_sharded_step_matches_single_process():
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
    cfg = workloads.random_system(40, (8, 8, 8), 24, 16, 0.02, 5)
    osys = oracle_system(cfg)
    F = oracle.gateaux(osys, cfg["V"])["F"]
    step = oracle.lrdm_apply(cfg["R"], cfg["V"], F, osys.w, 0.5, rho=np.stack(osys.rho))
    for r in range(world):
        Fr, ar, sr = res[r]
        assert np.array_equal(Fr, F)
        assert np.allclose(ar, step["a"], rtol=1e-12)
        assert abs(sr - step["s_rel"]) < 1e-12


class _OracleContext:
    """What sharded_step needs of a Context (gateaux over the systems' lists,
    apply with an in-place density update), evaluated by the FP64 oracle on
    CPU tensors."""

    nsys = 1

    def __init__(self, osys):
        self.osys = osys
        self.calls = []

    def gateaux(self, V):
        import oracle
        (v,) = V
        self.calls.append(int(v.shape[0]))
        if v.shape[0] == 0:
            return [v.clone()], torch.zeros(0, dtype=torch.float64)
        r = oracle.gateaux(self.osys, v.numpy())
        return [torch.as_tensor(r["F"])], torch.as_tensor(r["dmu"])

    def apply(self, sys, R, V, F, alpha, rho=None):
        import oracle
        out = oracle.lrdm_apply(R.numpy(), V.numpy(), F.numpy(), self.osys.w, alpha,
                                rho=None if rho is None else rho.numpy().copy())
        if rho is not None:
            rho.copy_(torch.as_tensor(out["rho_new"]))
        return torch.as_tensor(out["a"]), torch.as_tensor([out["s_rel"]])


def _worker_step(rank, world, port, out, K):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        here = os.path.dirname(os.path.abspath(__file__))
        sys.path.insert(0, here)
        sys.path.insert(0, os.path.dirname(here))
        import workloads
        from helpers import oracle_system
        cfg = workloads.random_system(41, (8, 8, 8), 24, 16, 0.02, K)
        osys = oracle_system(cfg)
        ctx = _OracleContext(osys)
        rho = torch.as_tensor(np.stack(osys.rho))
        F, a, s_rel = sharded_step(ctx, torch.as_tensor(cfg["V"]), torch.as_tensor(cfg["R"]), 0.5, rho=rho)
        out[rank] = (F.numpy(), a.numpy(), float(s_rel[0]), rho.numpy(), ctx.calls)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("K", [5, 1])
def test_sharded_step_matches_single_process(K):
    """sharded_step on 2 ranks (K = 5: slices of 3 and 2 directions; K = 1:
    one rank evaluates nothing) gives every rank the single-process
    derivatives, coefficients, s_rel and density update."""
    import oracle
    import workloads
    from helpers import oracle_system
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker_step, args=(world, port, out, K), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    cfg = workloads.random_system(41, (8, 8, 8), 24, 16, 0.02, K)
    osys = oracle_system(cfg)
    F = oracle.gateaux(osys, cfg["V"])["F"]
    step = oracle.lrdm_apply(cfg["R"], cfg["V"], F, osys.w, 0.5, rho=np.stack(osys.rho))
    assert [res[r][4] for r in range(world)] == [[b - a] for a, b in
                                                  (shard_bounds(K, world, r) for r in range(world))]
    for r in range(world):
        Fr, ar, sr, rho_r, _ = res[r]
        assert np.array_equal(Fr, F)
        assert np.allclose(ar, step["a"], rtol=1e-12)
        assert abs(sr - step["s_rel"]) < 1e-12
        assert np.allclose(rho_r, step["rho_new"], rtol=1e-13, atol=1e-15)
