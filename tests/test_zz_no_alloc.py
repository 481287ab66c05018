"""lrdm_apply_static: the least-squares step for callers that cannot allocate
device memory (their memory is owned by another allocator, or cudaMalloc's
implicit synchronisation is not acceptable on their path).  It must give the
same result as lrdm_apply, which runs the same step on a context's
workspaces, and it must not keep anything from one call to the next that
changes the result.  Collected last on purpose."""

import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import oracle_system

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build, binding
    build.build()
    return binding.load()


def _inputs(cfg, K, io):
    F = oracle.gateaux(oracle_system(cfg), cfg["V"][:K])["F"]
    dev = dict(device="cuda", dtype=io)
    return (torch.as_tensor(cfg["R"], **dev), torch.as_tensor(cfg["V"][:K], **dev),
            torch.as_tensor(F, **dev))


@pytest.mark.parametrize("io", [torch.float64, torch.float32])
def test_static_apply_matches_context_apply(lib, cfg1, io):
    from gpu_helpers import make_context
    from paper_2211_07894_gb300 import binding
    prec = "fp64" if io == torch.float64 else "fp32"
    tol = 1e-10 if io == torch.float64 else 1e-5
    ctx, _ = make_context([cfg1], prec, io)
    w = float(np.prod(cfg1["h"]))
    dtype_code = binding.DTYPE_F64 if io == torch.float64 else binding.DTYPE_F32
    rng = np.random.default_rng(7)
    # two calls in a row with different inputs: each must equal lrdm_apply's result
    for call, (K, alpha) in enumerate([(4, 0.5), (3, 0.0)]):
        R, V, F = _inputs(cfg1, K, io)
        R = R * (1.0 + 0.1 * call)
        rho0 = torch.as_tensor(rng.standard_normal((1, R.shape[1])) * 0.01 + 0.1, dtype=io,
                               device="cuda")
        rho_ref = rho0.clone()
        coef_ref, srel_ref = ctx.apply(0, R, V, F, alpha, rho=rho_ref)
        rho_new = rho0.clone()
        coef = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
        srel = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        code = binding.lrdm_apply_static(R.data_ptr(), V.data_ptr(), F.data_ptr(), dtype_code, K,
                                         R.numel(), w, alpha, 1e-12, rho_new.data_ptr(),
                                         coef.data_ptr(), srel.data_ptr(), status.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
        assert code == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        c, cr = coef.cpu().numpy(), coef_ref.cpu().numpy()
        assert np.max(np.abs(c - cr)) <= tol * np.max(np.abs(cr))
        assert abs(srel.item() - srel_ref.item()) <= tol * max(srel_ref.item(), 1e-30)
        d = (rho_new - rho_ref).double().norm() / rho_ref.double().norm()
        assert float(d) <= tol


def test_static_apply_rejects_oversized_k(lib):
    from paper_2211_07894_gb300 import binding
    n = 64
    x = torch.zeros((17, n), dtype=torch.float64, device="cuda")
    code = binding.lrdm_apply_static(x.data_ptr(), x.data_ptr(), x.data_ptr(), binding.DTYPE_F64,
                                     17, n, 1.0, 0.5, 1e-12, 0, 0, 0, 0,
                                     torch.cuda.current_stream().cuda_stream)
    assert code == 1      # LRDM_ERR_INVALID_ARG: K above the static limit of 16


def _call_static(R, V, F, K, w, alpha, rho, coef, srel, status, io):
    from paper_2211_07894_gb300 import binding
    dtype_code = binding.DTYPE_F64 if io == torch.float64 else binding.DTYPE_F32
    return binding.lrdm_apply_static(R.data_ptr(), V.data_ptr(), F.data_ptr(), dtype_code, K, R.numel(), w,
                                     alpha, 1e-12, rho.data_ptr(), coef.data_ptr(), srel.data_ptr(),
                                     status.data_ptr(), torch.cuda.current_stream().cuda_stream)


def test_static_apply_status_bits(lib, cfg1):
    """The status word the call reports: a singular S (two equal derivatives)
    sets the singular bit and gives lrdm_apply's minimum-norm coefficients; a
    non-finite residual sets the non-finite bit; the next clean call reports
    0, since the word is cleared at the start of every call."""
    from gpu_helpers import make_context
    io = torch.float64
    ctx, _ = make_context([cfg1], "fp64", io)
    w = float(np.prod(cfg1["h"]))
    R, V, F = _inputs(cfg1, 3, io)
    F2 = F.clone()
    F2[1] = F2[0]
    rho = torch.zeros_like(R)
    coef = torch.empty(3, dtype=torch.float64, device="cuda")
    srel = torch.empty(1, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert _call_static(R, V, F2, 3, w, 0.0, rho, coef, srel, status, io) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 4
    coef_ref, _ = ctx.apply(0, R, V, F2, 0.0, rho=torch.zeros_like(R))
    torch.cuda.synchronize()
    assert torch.allclose(coef, coef_ref, rtol=1e-10, atol=1e-14)
    Rn = R.clone()
    Rn[0, 5] = float("nan")
    assert _call_static(Rn, V, F, 3, w, 0.0, rho, coef, srel, status, io) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 2
    assert _call_static(R, V, F, 3, w, 0.0, rho, coef, srel, status, io) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_static_apply_allocates_nothing(lib, cfg1):
    """After a first call on the device (which looks the scratch array up),
    further calls leave torch's allocator and the device's free memory as
    they were."""
    io = torch.float32
    w = float(np.prod(cfg1["h"]))
    R, V, F = _inputs(cfg1, 4, io)
    rho = torch.zeros_like(R)
    coef = torch.empty(4, dtype=torch.float64, device="cuda")
    srel = torch.empty(1, dtype=torch.float64, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    assert _call_static(R, V, F, 4, w, 0.5, rho, coef, srel, status, io) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert _call_static(R, V, F, 4, w, 0.5, rho, coef, srel, status, io) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert int(status.item()) == 0
