"""Direction-sharded evaluation on two CPU ranks (gloo): each rank evaluates
its slice of the directions, the slices are all-gathered and the
least-squares step on the gathered set must equal the single-process one.
The FP64 oracle stands in for the per-rank GPU evaluation."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_07894_gb300.sharding import gather_directions, shard_bounds


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
