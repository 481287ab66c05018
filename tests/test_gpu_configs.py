"""Parity at the full sizes of the single-system and batched workloads,
against the FP64 oracle on every direction.

* 48^3 grid (110,592 points), N_s = 512, N_e = 460, kT = 0.005, K = 8
  (random subspace under a smooth envelope, uniform eigenvalues): every
  precision, FP64 <= 1e-10, FP32 <= 1e-4, split-BF16x3 <= 1e-5, TF32 at its
  gate (tests/gates.py).
* Six uneven systems (32^3 / 256 / K 4 up to 64^3 / 1024 / K 16) and one spin
  pair (64^3, 768 / 704 states, K = 8 shared): 64 Gateaux derivatives in one
  call, split-BF16x3, one grouped launch per contraction (counted by the
  library's profiling) and replayed from a captured CUDA graph; every
  derivative <= 1e-5 against the oracle.
"""

import numpy as np
import pytest

import oracle
import workloads
from gates import check
from helpers import oracle_system, per_direction_rel_err

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def single():
    cfg = workloads.config2()
    ref = oracle.gateaux(oracle_system(cfg), cfg["V"])
    return cfg, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_single_system_48cube(lib, single, prec):
    from gpu_helpers import directions, make_context
    cfg, ref = single
    io = torch.float64 if prec == "fp64" else torch.float32
    ctx, _ = make_context([cfg], prec, io)
    V = directions(cfg, io)
    (F,), dmu = ctx.gateaux([V])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    err = per_direction_rel_err(F.double().cpu().numpy(), ref["F"])
    check(prec, "single_system_48cube", err)
    scale = float(np.max(np.abs(np.diagonal(ref["X"][0], axis1=1, axis2=2))))
    check(prec, "single_system_48cube", float(np.max(np.abs(dmu.cpu().numpy() - ref["dmu"]))) / scale, "dmu")


@pytest.fixture(scope="module")
def batch():
    cfgs = workloads.config3()
    refs = [oracle.gateaux(oracle_system(c), c["V"]) for c in cfgs]
    return cfgs, refs


def test_uneven_batch_one_launch(lib, batch):
    from gpu_helpers import directions, make_context
    cfgs, refs = batch
    assert sum(c["V"].shape[0] for c in cfgs) == 64
    io = torch.float32
    ctx, _ = make_context(cfgs, "bf16x3", io, use_graph=True)
    V = [directions(c, io) for c in cfgs]
    F = [torch.empty_like(v) for v in V]
    ctx.profile(True)
    ctx.profile_read(reset=True)
    ctx.gateaux(V, out=F)
    torch.cuda.synchronize()
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    assert ctx.status() == 0
    assert prof["gemm1_launches"] == 1 and prof["gemm2_launches"] == 1
    eager = [f.clone() for f in F]
    side = torch.cuda.Stream()     # graphs are captured on a stream other than the legacy default
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.gateaux(V, out=F)      # captured into a graph
        ctx.gateaux(V, out=F)      # replayed
    torch.cuda.synchronize()
    assert ctx.status() == 0
    worst = 0.0
    for i, (c, ref) in enumerate(zip(cfgs, refs)):
        assert torch.equal(F[i], eager[i])
        err = per_direction_rel_err(F[i].double().cpu().numpy(), ref["F"])
        print(f"uneven batch system {i} ({c['name']}, K = {c['V'].shape[0]}): f err {err:.2e}")
        worst = max(worst, err)
    check("bf16x3", "uneven_batch_one_launch", worst)
