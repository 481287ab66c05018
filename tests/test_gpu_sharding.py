"""Direction-sharded step (sharding.sharded_step) on the GPU with the real
library context: with no process group and with a one-rank NCCL group (the
all-gather runs on device tensors), it equals the unsharded forward and
least-squares step bit for bit; and a grid-row-sharded context whose
exchanges go through torch_allreduce on a one-rank NCCL group.  Several
ranks are covered on the CPU (tests/test_sharding_gloo.py,
tests/test_rows_gloo.py) and as host threads on one GPU
(tests/test_gpu_rows.py); NCCL ranks need a GPU each."""

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


def test_row_sharded_context_one_rank_nccl(lib):
    """A grid-row-sharded context holding all rows, its exchanges through
    torch_allreduce over a one-rank NCCL group (the library's buffers summed
    in place as torch tensors on the library's stream): the forward, the
    least-squares step and the adjoint equal the plain context's up to the
    order of the grid sums (one partial X against row ranges)."""
    import torch.distributed as dist
    from gpu_helpers import directions, to_device_system
    from helpers import per_direction_rel_err
    from paper_2211_07894_gb300 import Context, torch_allreduce
    cfg = workloads.random_system(43, (20, 18, 16), 160, 120, 0.01, 4)
    io = torch.float32
    ng = int(np.prod(cfg["n"]))
    V = directions(cfg, io)
    R = torch.as_tensor(cfg["R"], dtype=io, device="cuda")
    fbar = torch.randn_like(V)
    plain = Context([to_device_system(cfg, io)], prec="bf16x3", io_dtype=io, k_max=4)
    (F0,), _ = plain.gateaux([V])
    a0, s0 = plain.apply(0, R, V, F0, 0.5)
    vb0, eb0, _ = plain.backward([fbar])
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        rows = Context([to_device_system(cfg, io)], prec="bf16x3", io_dtype=io, k_max=4,
                       rows=dict(row_begin=0, n_rows=ng, allreduce=torch_allreduce()))
        (F1,), _ = rows.gateaux([V])
        a1, s1 = rows.apply(0, R, V, F1, 0.5)
        vb1, eb1, _ = rows.backward([fbar])
        torch.cuda.synchronize()
        assert rows.status() == 0
    finally:
        dist.destroy_process_group()
    assert per_direction_rel_err(F1.double().cpu().numpy(), F0.double().cpu().numpy()) < 1e-6
    assert per_direction_rel_err(vb1[0].double().cpu().numpy(), vb0[0].double().cpu().numpy()) < 1e-6
    assert np.allclose(a1.cpu().numpy(), a0.cpu().numpy(), rtol=1e-4, atol=1e-9)
    assert abs(float(s1) - float(s0)) < 1e-5
    rows.close()
    plain.close()
