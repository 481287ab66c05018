"""Failure detection on the GPU without a GPU fault.

Every wait inside the tensor-core contractions is bounded (4 s by the global
timer).  With the test-only flag LRDM_DEBUG_STALL_PROJECTION the next
projection launch leaves one weighted stage of its first CTA unpublished: the
MMA thread's wait expires, the kernel records LRDM_ERR_TIMEOUT in the
context's status word, waits for its own copies and MMAs, frees its tensor
memory and returns.  The test checks the status, that the call returned
after the bound (not a hang, not a trap), and that the next call on the same
context gives exactly the result of a clean context.
"""

import time

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N = (16, 16, 16)
NS, K, NE, KT = 256, 2, 200.0, 0.01


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build
    build.build()


def _ctx(cfg, **kw):
    from gpu_helpers import to_device_system
    from paper_2211_07894_gb300 import Context
    d = to_device_system(cfg, torch.float32)
    return Context([d], prec="bf16x3", io_dtype=torch.float32, k_max=K, **kw)


def test_projection_timeout_is_reported_and_recovered(lib):
    from paper_2211_07894_gb300 import binding
    cfg = workloads.random_system(90, N, NS, NE, KT, K)
    V = torch.as_tensor(cfg["V"], dtype=torch.float32, device="cuda")
    clean = _ctx(cfg)
    (Fc,), _ = clean.gateaux([V])
    torch.cuda.synchronize()
    assert clean.status() == 0

    ctx = _ctx(cfg, debug_flags=binding.DEBUG_STALL_PROJECTION)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.gateaux([V])
    code = ctx.status()                       # synchronises
    dt = time.perf_counter() - t0
    print(f"stalled projection: status {code}, returned after {dt:.2f} s")
    assert code == 7                          # LRDM_ERR_TIMEOUT
    assert 3.5 < dt < 60.0
    # the flag applies once; the context and the device stay usable
    (F2,), _ = ctx.gateaux([V])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert torch.equal(F2, Fc)
    ctx.close()
    clean.close()
