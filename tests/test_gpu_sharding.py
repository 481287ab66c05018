"""Direction-sharded step (sharding.sharded_step) on the GPU with the real
library context: with no process group and with a one-rank NCCL group (the
all-gather runs on device tensors), it equals the unsharded forward and
least-squares step bit for bit.  Several ranks are covered on the CPU
(tests/test_sharding_gloo.py); each rank needs a GPU of its own."""

import socket

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build
    build.build()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_sharded_step_one_rank(lib):
    import torch.distributed as dist
    from gpu_helpers import directions, make_context
    from paper_2211_07894_gb300.sharding import sharded_step
    cfg = workloads.random_system(42, (20, 18, 16), 160, 120, 0.01, 6)
    io = torch.float32
    ctx, _ = make_context([cfg], "bf16x3", io)
    V = directions(cfg, io)
    R = torch.as_tensor(cfg["R"], dtype=io, device="cuda")
    rho0 = torch.full_like(R, 0.1)
    (F_ref,), _ = ctx.gateaux([V])
    rho_ref = rho0.clone()
    a_ref, s_ref = ctx.apply(0, R, V, F_ref, 0.5, rho=rho_ref)
    rho1 = rho0.clone()
    F1, a1, s1 = sharded_step(ctx, V, R, 0.5, rho=rho1)        # no process group
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        rho2 = rho0.clone()
        F2, a2, s2 = sharded_step(ctx, V, R, 0.5, rho=rho2)
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    assert ctx.status() == 0
    for F, a, s, rho in ((F1, a1, s1, rho1), (F2, a2, s2, rho2)):
        assert torch.equal(F, F_ref)
        assert torch.equal(a, a_ref) and torch.equal(s, s_ref)
        assert torch.equal(rho, rho_ref)
    assert float(s_ref) < 1.0 and np.isfinite(a_ref.cpu().numpy()).all()
