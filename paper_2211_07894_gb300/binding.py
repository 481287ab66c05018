"""ctypes binding of liblrdm.so: the C-ABI calls under the same names, plus a
small torch-facing ``Context`` that marshals tensors into them.

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  There is no fallback -- if the compiled library is
missing, loading raises.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_void_p
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "liblrdm.so")

LRDM_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "shape", 3: "out of memory", 4: "cuda",
                5: "mu not converged", 6: "singular", 7: "timeout", 8: "non-finite",
                9: "unsupported", 10: "collective"}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3}
DTYPE_F64, DTYPE_F32 = 0, 1
DEBUG_STALL_PROJECTION = 1      # lrdm_options.debug_flags bit (tests only)


class LrdmError(RuntimeError):
    def __init__(self, call, code):
        super().__init__(f"{call} failed: {STATUS_NAMES.get(code, code)} ({code})")
        self.code = code


class lrdm_system(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("h", c_double * 3), ("nspin", c_int), ("ns", c_int * 2),
                ("ld_psi", c_int * 2), ("psi", c_void_p * 2), ("eps", c_void_p * 2),
                ("occ", c_void_p * 2), ("rho", c_void_p * 2), ("n_electrons", c_double),
                ("kT", c_double), ("occ_factor", c_double), ("rho_floor", c_double),
                ("k_max", c_int)]


class lrdm_options(ctypes.Structure):
    _fields_ = [("prec", c_int), ("io_dtype", c_int), ("k_max", c_int),
                ("pinv_rcond", c_double), ("degen_tol", c_double), ("poisson_symbol", c_int),
                ("use_graph", c_int), ("autotune", c_int), ("debug_flags", c_int),
                ("fermi_T", c_int)]


# int (*)(void* user, void* buf, long long count, int dtype, void* stream)
ALLREDUCE_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_void_p, ctypes.c_longlong, c_int, c_void_p)


class lrdm_rows(ctypes.Structure):
    _fields_ = [("row_begin", ctypes.c_longlong), ("n_rows", ctypes.c_longlong),
                ("allreduce", ALLREDUCE_FN), ("user", c_void_p)]


class lrdm_kpoint_system(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("h", c_double * 3), ("nk", c_int), ("ns", c_int),
                ("ld_psi", c_int), ("psi_re", POINTER(c_void_p)), ("psi_im", POINTER(c_void_p)),
                ("eps", POINTER(c_void_p)), ("k_weights", POINTER(c_double)), ("rho", c_void_p),
                ("n_electrons", c_double), ("kT", c_double), ("occ_factor", c_double),
                ("rho_floor", c_double), ("k_max", c_int)]


_lib = None

EXPORTS = ["lrdm_default_options", "lrdm_create", "lrdm_gateaux_batch", "lrdm_apply",
           "lrdm_apply_static",
           "lrdm_backward", "lrdm_status_query", "lrdm_get_mu", "lrdm_get_density",
           "lrdm_get_projection", "lrdm_profile_enable", "lrdm_profile_read", "lrdm_destroy", "lrdm_status_string",
           "lrdm_get_tuning", "lrdm_krylov_step", "lrdm_lrdma_default_params", "lrdm_lrdma_create",
           "lrdm_lrdma_step", "lrdm_lrdma_clear", "lrdm_lrdma_destroy", "lrdm_kp_create",
           "lrdm_kp_gateaux", "lrdm_lrdma_get_state", "lrdm_lrdma_export", "lrdm_lrdma_import",
           "lrdm_kp_get_split", "lrdm_set_tuning", "lrdm_create_rows"]


class lrdm_lrdma_params(ctypes.Structure):
    _fields_ = [("s_tol", c_double), ("beta_tol", c_double), ("r_norm_clear", c_double),
                ("alpha", c_double), ("r_max_iter", c_int), ("r_max", c_int)]


class lrdm_lrdma_report(ctypes.Structure):
    _fields_ = [("event", c_int), ("rank", c_int), ("rank_new", c_int), ("s_rel", c_double),
                ("beta", c_double), ("r_norm", c_double), ("alpha", c_double)]


LRDMA_EVENTS = {0: "fresh", 1: "reuse", 2: "accumulate", 3: "CL", 4: "CR", 5: "CT"}


def load(path: Optional[str] = None):
    """Loads liblrdm.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"liblrdm.so not built at {p}; run paper_2211_07894_gb300.build.build()")
    lib = ctypes.CDLL(p)
    lib.lrdm_default_options.argtypes = [POINTER(lrdm_options)]
    lib.lrdm_default_options.restype = None
    lib.lrdm_create.argtypes = [POINTER(c_void_p), POINTER(lrdm_system), c_int,
                                POINTER(lrdm_options), c_void_p]
    lib.lrdm_create.restype = c_int
    lib.lrdm_create_rows.argtypes = [POINTER(c_void_p), POINTER(lrdm_system), POINTER(lrdm_rows),
                                     POINTER(lrdm_options), c_void_p]
    lib.lrdm_create_rows.restype = c_int
    lib.lrdm_gateaux_batch.argtypes = [c_void_p, POINTER(c_void_p), POINTER(c_int),
                                       POINTER(c_void_p), c_void_p, c_void_p]
    lib.lrdm_gateaux_batch.restype = c_int
    lib.lrdm_apply.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_double,
                               c_void_p, c_void_p, c_void_p, c_void_p]
    lib.lrdm_apply.restype = c_int
    lib.lrdm_apply_static.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int,
                                      ctypes.c_longlong, c_double, c_double, c_double, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p]
    lib.lrdm_apply_static.restype = c_int
    lib.lrdm_backward.argtypes = [c_void_p, POINTER(c_void_p), POINTER(c_void_p),
                                  POINTER(c_void_p), POINTER(c_void_p), c_void_p]
    lib.lrdm_backward.restype = c_int
    lib.lrdm_status_query.argtypes = [c_void_p, c_int]
    lib.lrdm_status_query.restype = c_int
    lib.lrdm_get_mu.argtypes = [c_void_p, c_int, POINTER(c_double)]
    lib.lrdm_get_mu.restype = c_int
    lib.lrdm_get_density.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p]
    lib.lrdm_get_density.restype = c_int
    lib.lrdm_get_projection.argtypes = [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]
    lib.lrdm_get_projection.restype = c_int
    lib.lrdm_profile_enable.argtypes = [c_void_p, c_int]
    lib.lrdm_profile_enable.restype = c_int
    lib.lrdm_profile_read.argtypes = [c_void_p, POINTER(c_double), POINTER(ctypes.c_longlong),
                                      POINTER(c_double), POINTER(ctypes.c_longlong),
                                      POINTER(c_double), POINTER(ctypes.c_longlong),
                                      POINTER(ctypes.c_longlong), c_int]
    lib.lrdm_profile_read.restype = c_int
    lib.lrdm_krylov_step.argtypes = [c_void_p, c_int, c_void_p, c_double, c_int, c_double, c_void_p,
                                     c_void_p, c_void_p, c_void_p, POINTER(c_double), POINTER(c_int),
                                     POINTER(c_double), c_void_p]
    lib.lrdm_krylov_step.restype = c_int
    lib.lrdm_lrdma_default_params.argtypes = [POINTER(lrdm_lrdma_params)]
    lib.lrdm_lrdma_default_params.restype = None
    lib.lrdm_lrdma_create.argtypes = [POINTER(c_void_p), ctypes.c_longlong, c_int, c_double, c_int]
    lib.lrdm_lrdma_create.restype = c_int
    lib.lrdm_lrdma_step.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                    POINTER(lrdm_lrdma_params), POINTER(lrdm_lrdma_report), c_void_p]
    lib.lrdm_lrdma_step.restype = c_int
    lib.lrdm_lrdma_clear.argtypes = [c_void_p]
    lib.lrdm_lrdma_clear.restype = c_int
    lib.lrdm_lrdma_get_state.argtypes = [c_void_p, POINTER(c_int), POINTER(c_int)]
    lib.lrdm_lrdma_get_state.restype = c_int
    lib.lrdm_lrdma_export.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.lrdm_lrdma_export.restype = c_int
    lib.lrdm_lrdma_import.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.lrdm_lrdma_import.restype = c_int
    lib.lrdm_lrdma_destroy.argtypes = [c_void_p]
    lib.lrdm_lrdma_destroy.restype = None
    lib.lrdm_get_tuning.argtypes = [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                    POINTER(c_int)]
    lib.lrdm_get_tuning.restype = c_int
    lib.lrdm_set_tuning.argtypes = [c_void_p, c_int, c_int, c_int, c_int]
    lib.lrdm_set_tuning.restype = c_int
    lib.lrdm_kp_create.argtypes = [POINTER(c_void_p), POINTER(lrdm_kpoint_system),
                                   POINTER(lrdm_options), c_void_p]
    lib.lrdm_kp_create.restype = c_int
    lib.lrdm_kp_gateaux.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    lib.lrdm_kp_gateaux.restype = c_int
    lib.lrdm_kp_get_split.argtypes = [c_void_p, c_int, POINTER(c_int)]
    lib.lrdm_kp_get_split.restype = c_int
    lib.lrdm_destroy.argtypes = [c_void_p]
    lib.lrdm_destroy.restype = None
    lib.lrdm_status_string.argtypes = [c_int]
    lib.lrdm_status_string.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def _check(call, code):
    if code != LRDM_OK:
        raise LrdmError(call, code)


def _ptr_array(ptrs):
    arr = (c_void_p * max(1, len(ptrs)))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


# ---------------------------------------------------------------------------
# C-ABI calls under their own names (plain pointers in, status code out)
# ---------------------------------------------------------------------------

def lrdm_default_options() -> lrdm_options:
    o = lrdm_options()
    load().lrdm_default_options(ctypes.byref(o))
    return o


def lrdm_create(systems: Sequence[lrdm_system], options: lrdm_options, stream: int = 0):
    arr = (lrdm_system * len(systems))(*systems)
    h = c_void_p()
    code = load().lrdm_create(ctypes.byref(h), arr, len(systems), ctypes.byref(options),
                              c_void_p(stream))
    return code, h


def lrdm_create_rows(system: lrdm_system, rows: lrdm_rows, options: lrdm_options, stream: int = 0):
    h = c_void_p()
    code = load().lrdm_create_rows(ctypes.byref(h), ctypes.byref(system), ctypes.byref(rows),
                                   ctypes.byref(options), c_void_p(stream))
    return code, h


class _DeviceArray:
    """A device buffer of the library seen by torch (zero copy)."""

    def __init__(self, ptr, count, dtype):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": (int(count),),
                                         "typestr": "<f8" if dtype == DTYPE_F64 else "<f4",
                                         "version": 3, "strides": None}


def rows_callback(fn):
    """The C callback of a row-sharded context around fn(tensor, stream):
    tensor is the library's buffer as a 1-D torch tensor (summed in place over
    the ranks by fn), stream the torch stream the library enqueued its work on."""
    import torch

    def cb(user, buf, count, dtype, stream):
        try:
            t = torch.as_tensor(_DeviceArray(buf, count, dtype), device="cuda")
            st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                fn(t, st)
            return 0
        except Exception as e:          # reported to the library as a failed collective
            import sys
            print(f"lrdm rows allreduce failed: {e!r}", file=sys.stderr)
            return 1

    return ALLREDUCE_FN(cb)


def torch_allreduce(group=None):
    """fn(tensor, stream) for rows_callback: an in-place sum over the ranks of
    `group` by torch.distributed (NCCL), ordered on the library's stream."""
    import torch.distributed as dist

    def fn(t, st):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

    return fn


def lrdm_gateaux_batch(ctx, v_ptrs, K, f_ptrs, dmu_ptr, stream: int = 0) -> int:
    Ks = (c_int * len(K))(*K)
    return load().lrdm_gateaux_batch(ctx, _ptr_array(v_ptrs), Ks, _ptr_array(f_ptrs),
                                     c_void_p(dmu_ptr or 0), c_void_p(stream))


def lrdm_apply(ctx, sys, R, v, f, K, alpha, rho, coeff, s_rel, stream: int = 0) -> int:
    return load().lrdm_apply(ctx, sys, c_void_p(R), c_void_p(v), c_void_p(f), K, alpha,
                             c_void_p(rho or 0), c_void_p(coeff or 0), c_void_p(s_rel or 0),
                             c_void_p(stream))


def lrdm_apply_static(R, v, f, io_dtype, K, n, w, alpha, pinv_rcond, rho, coeff, s_rel,
                      status, stream: int = 0) -> int:
    return load().lrdm_apply_static(c_void_p(R), c_void_p(v), c_void_p(f), io_dtype, K, n, w,
                                    alpha, pinv_rcond, c_void_p(rho or 0), c_void_p(coeff or 0),
                                    c_void_p(s_rel or 0), c_void_p(status or 0), c_void_p(stream))


def lrdm_backward(ctx, fbar_ptrs, vbar_ptrs, eps_bar_ptrs=None, occ_bar_ptrs=None,
                  stream: int = 0) -> int:
    eb = _ptr_array(eps_bar_ptrs) if eps_bar_ptrs is not None else None
    ob = _ptr_array(occ_bar_ptrs) if occ_bar_ptrs is not None else None
    return load().lrdm_backward(ctx, _ptr_array(fbar_ptrs), _ptr_array(vbar_ptrs),
                                eb, ob, c_void_p(stream))


def lrdm_status_query(ctx, synchronize: int = 1) -> int:
    return load().lrdm_status_query(ctx, synchronize)


def lrdm_get_mu(ctx, sys: int) -> float:
    mu = c_double()
    _check("lrdm_get_mu", load().lrdm_get_mu(ctx, sys, ctypes.byref(mu)))
    return mu.value


def lrdm_get_density(ctx, sys, spin, out_ptr, stream: int = 0) -> int:
    return load().lrdm_get_density(ctx, sys, spin, c_void_p(out_ptr), c_void_p(stream))


def lrdm_get_projection(ctx, sys, spin, k, out_ptr, stream: int = 0) -> int:
    return load().lrdm_get_projection(ctx, sys, spin, k, c_void_p(out_ptr), c_void_p(stream))


def lrdm_profile_enable(ctx, on: int) -> int:
    return load().lrdm_profile_enable(ctx, on)


def lrdm_profile_read(ctx, reset: int = 1):
    t1, t2, t3 = c_double(), c_double(), c_double()
    n1, n2, n3, nk = (ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong(),
                      ctypes.c_longlong())
    _check("lrdm_profile_read", load().lrdm_profile_read(ctx, ctypes.byref(t1), ctypes.byref(n1),
                                                         ctypes.byref(t2), ctypes.byref(n2),
                                                         ctypes.byref(t3), ctypes.byref(n3),
                                                         ctypes.byref(nk), reset))
    return dict(gemm1_ms=t1.value, gemm1_launches=n1.value, gemm2_ms=t2.value,
                gemm2_launches=n2.value, poisson_ms=t3.value, poisson_calls=n3.value,
                kernel_launches=nk.value)


def lrdm_krylov_step(ctx, sys, R_ptr, s_tol, r_max, alpha, rho_ptr, U_ptr, T_ptr, coeff_ptr,
                     stream: int = 0):
    """Returns (status, rank, s_rel list, ||R||)."""
    s_rel = (c_double * max(1, r_max))()
    rank = c_int(0)
    rn = c_double(0.0)
    code = load().lrdm_krylov_step(ctx, sys, c_void_p(R_ptr), float(s_tol), int(r_max), float(alpha),
                                   c_void_p(rho_ptr), c_void_p(U_ptr), c_void_p(T_ptr),
                                   c_void_p(coeff_ptr), s_rel, ctypes.byref(rank), ctypes.byref(rn),
                                   c_void_p(stream))
    return code, rank.value, [s_rel[i] for i in range(rank.value)], rn.value


def lrdm_get_tuning(ctx):
    z, a, b, c = c_int(), c_int(), c_int(), c_int()
    _check("lrdm_get_tuning", load().lrdm_get_tuning(ctx, ctypes.byref(z), ctypes.byref(a),
                                                     ctypes.byref(b), ctypes.byref(c)))
    return dict(g1_nb=z.value, g1_dpt=a.value, g2_bn=b.value, g2_kgroup=c.value)


def lrdm_set_tuning(ctx, g1_nb, g1_dpt, g2_bn, g2_kgroup) -> int:
    return load().lrdm_set_tuning(ctx, g1_nb, g1_dpt, g2_bn, g2_kgroup)


def lrdm_kp_create(system: lrdm_kpoint_system, options: lrdm_options, stream: int = 0):
    h = c_void_p()
    code = load().lrdm_kp_create(ctypes.byref(h), ctypes.byref(system), ctypes.byref(options),
                                 c_void_p(stream))
    return code, h


def lrdm_kp_gateaux(ctx, v_ptr, K, f_ptr, dmu_ptr, stream: int = 0) -> int:
    return load().lrdm_kp_gateaux(ctx, c_void_p(v_ptr), int(K), c_void_p(f_ptr),
                                  c_void_p(dmu_ptr or 0), c_void_p(stream))


def lrdm_destroy(ctx) -> None:
    load().lrdm_destroy(ctx)


def lrdm_status_string(code: int) -> str:
    return load().lrdm_status_string(code).decode()


# ---------------------------------------------------------------------------
# torch-facing context
# ---------------------------------------------------------------------------

class Context:
    """Owns one lrdm_ctx.  ``systems`` is a list of dicts with keys

      n, h, psi (list of (N_g, N_s) tensors on the device), eps (list of
      float64 tensors), optional occ, optional rho, n_electrons, kT, g,
      rho_floor, k_max.

    Direction / result tensors are (K, nspin, N_g) in the io dtype.

    rows = dict(row_begin, n_rows, allreduce) makes a grid-row-sharded
    context (lrdm_create_rows) of the one system given, whose psi (and rho)
    hold those grid rows only; every row-wise tensor is then (.., n_rows).
    allreduce(tensor, stream) sums the library's buffer in place over the
    ranks (torch_allreduce(group) for torch.distributed); all ranks make the
    same calls in the same order.
    """

    def __init__(self, systems, prec="bf16x3", io_dtype=None, k_max=16, pinv_rcond=1e-12,
                 degen_tol=1e-5, poisson="spectral", use_graph=False, stream=None, fermi_T=0,
                 autotune=False, debug_flags=0, rows=None):
        import torch
        self.torch = torch
        self.io_dtype = io_dtype or torch.float32
        self.prec = prec
        o = lrdm_default_options()
        o.prec = PRECISIONS[prec]
        o.io_dtype = DTYPE_F64 if self.io_dtype == torch.float64 else DTYPE_F32
        o.k_max = int(k_max)
        o.pinv_rcond = float(pinv_rcond)
        o.degen_tol = float(degen_tol)
        o.poisson_symbol = 1 if poisson == "fd" else 0
        o.use_graph = 1 if use_graph else 0
        o.fermi_T = int(fermi_T)
        o.autotune = 1 if autotune else 0
        o.debug_flags = int(debug_flags)
        self.options = o
        keep = []
        cs = []
        self.meta = []
        for d in systems:
            s = lrdm_system()
            nspin = len(d["psi"])
            s.nspin = nspin
            for i in range(3):
                s.n[i] = int(d["n"][i])
                s.h[i] = float(d["h"][i])
            for c in range(nspin):
                psi = d["psi"][c]
                assert psi.is_cuda and psi.dtype == self.io_dtype and psi.dim() == 2
                assert psi.stride(1) == 1
                eps = d["eps"][c]
                assert eps.is_cuda and eps.dtype == torch.float64 and eps.is_contiguous()
                s.ns[c] = psi.shape[1]
                s.ld_psi[c] = psi.stride(0)
                s.psi[c] = psi.data_ptr()
                s.eps[c] = eps.data_ptr()
                keep += [psi, eps]
                if d.get("occ") is not None:
                    occ = d["occ"][c].contiguous()
                    s.occ[c] = occ.data_ptr()
                    keep.append(occ)
                if d.get("rho") is not None:
                    rho = d["rho"][c].to(self.io_dtype).contiguous()
                    s.rho[c] = rho.data_ptr()
                    keep.append(rho)
            s.n_electrons = float(d["n_electrons"])
            s.kT = float(d["kT"])
            s.occ_factor = float(d.get("g", 0.0) or 0.0)
            s.rho_floor = float(d.get("rho_floor", 0.0))
            s.k_max = int(d.get("k_max", 0))
            cs.append(s)
            ng = int(rows["n_rows"]) if rows is not None else int(np.prod(d["n"]))
            self.meta.append(dict(nspin=nspin, Ng=ng, ns=[int(p.shape[1]) for p in d["psi"]],
                                  k_max=int(d.get("k_max", 0)) or int(k_max)))
        self.nsys = len(self.meta)
        st = self._stream(stream)
        if rows is not None:
            # one system whose grid rows [row_begin, row_begin + n_rows) this
            # rank holds; rows["allreduce"] is fn(tensor, stream) (rows_callback)
            assert len(cs) == 1
            self._rows_cb = rows_callback(rows["allreduce"])
            r = lrdm_rows(int(rows["row_begin"]), int(rows["n_rows"]), self._rows_cb, None)
            code, h = lrdm_create_rows(cs[0], r, o, st)
            _check("lrdm_create_rows", code)
        else:
            code, h = lrdm_create(cs, o, st)
            _check("lrdm_create", code)
        self.handle = h
        del keep

    def _stream(self, stream):
        if stream is None:
            return self.torch.cuda.current_stream().cuda_stream
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def close(self):
        if getattr(self, "handle", None):
            lrdm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mu(self, sys=0):
        return lrdm_get_mu(self.handle, sys)

    def density(self, sys=0, spin=0, stream=None):
        out = self.torch.empty(self.meta[sys]["Ng"], dtype=self.io_dtype, device="cuda")
        _check("lrdm_get_density", lrdm_get_density(self.handle, sys, spin, out.data_ptr(),
                                                    self._stream(stream)))
        return out

    def gateaux(self, V: List, out: Optional[List] = None, dmu=None, stream=None):
        torch = self.torch
        assert len(V) == len(self.meta)
        K = [int(v.shape[0]) if v is not None else 0 for v in V]
        if out is None:
            out = [torch.empty_like(v) if v is not None else None for v in V]
        if dmu is None:
            dmu = torch.empty(max(1, sum(K)), dtype=torch.float64, device="cuda")
        for v, f in zip(V, out):
            if v is not None:
                assert v.is_contiguous() and v.dtype == self.io_dtype and f.is_contiguous()
        code = lrdm_gateaux_batch(self.handle, [v.data_ptr() if v is not None else 0 for v in V],
                                  K, [f.data_ptr() if f is not None else 0 for f in out],
                                  dmu.data_ptr(), self._stream(stream))
        _check("lrdm_gateaux_batch", code)
        return out, dmu[: sum(K)]

    def apply(self, sys, R, V, F, alpha, rho=None, coeff=None, s_rel=None, stream=None):
        torch = self.torch
        K = int(V.shape[0])
        coeff = coeff if coeff is not None else torch.empty(K, dtype=torch.float64, device="cuda")
        s_rel = s_rel if s_rel is not None else torch.empty(1, dtype=torch.float64, device="cuda")
        code = lrdm_apply(self.handle, sys, R.data_ptr(), V.data_ptr(), F.data_ptr(), K,
                          float(alpha), rho.data_ptr() if rho is not None else 0,
                          coeff.data_ptr(), s_rel.data_ptr(), self._stream(stream))
        _check("lrdm_apply", code)
        return coeff, s_rel

    def backward(self, fbar: List, want_eps=True, stream=None, out=None):
        """Adjoint of the most recent gateaux call.  ``out`` = (vbar, eps_bar,
        occ_bar) from an earlier call may be passed back to reuse its buffers."""
        torch = self.torch
        if out is not None:
            vbar, eb, ob = out
            code = lrdm_backward(self.handle, [f.data_ptr() if f is not None else 0 for f in fbar],
                                 [v.data_ptr() if v is not None else 0 for v in vbar],
                                 [e.data_ptr() if e is not None else 0 for e in eb] if want_eps else None,
                                 [o.data_ptr() if o is not None else 0 for o in ob] if want_eps else None,
                                 self._stream(stream))
            _check("lrdm_backward", code)
            return vbar, eb, ob
        vbar = [torch.empty_like(f) if f is not None else None for f in fbar]
        eb, ob = [], []
        ebp, obp = [], []
        for m in self.meta:
            for c in range(2):
                if want_eps and c < m["nspin"]:
                    e = torch.empty(m["ns"][c], dtype=torch.float64, device="cuda")
                    o = torch.empty(m["ns"][c], dtype=torch.float64, device="cuda")
                    eb.append(e)
                    ob.append(o)
                    ebp.append(e.data_ptr())
                    obp.append(o.data_ptr())
                else:
                    eb.append(None)
                    ob.append(None)
                    ebp.append(0)
                    obp.append(0)
        code = lrdm_backward(self.handle, [f.data_ptr() if f is not None else 0 for f in fbar],
                             [v.data_ptr() if v is not None else 0 for v in vbar],
                             ebp if want_eps else None, obp if want_eps else None,
                             self._stream(stream))
        _check("lrdm_backward", code)
        return vbar, eb, ob

    def projection(self, k, sys=0, spin=0, stream=None):
        """X_k (FP64, (N_s, N_s)) of the most recent gateaux call."""
        ns = self.meta[sys]["ns"][spin]
        out = self.torch.empty((ns, ns), dtype=self.torch.float64, device="cuda")
        _check("lrdm_get_projection", lrdm_get_projection(self.handle, sys, spin, k,
                                                          out.data_ptr(), self._stream(stream)))
        return out

    def krylov_step(self, R, s_tol=0.3, r_max=8, alpha=-1.0, rho=None, sys=0, stream=None):
        """One LRDM step with adaptive rank (lrdm_krylov_step).  R: (nspin, N_g)
        in the io dtype; rho (same shape) is updated in place when given;
        alpha < 0 selects the paper's schedule.  Returns dict(U, T, a, rank,
        s_rel, r_norm) with U, T (rank, nspin, N_g)."""
        torch = self.torch
        assert R.is_contiguous() and R.dtype == self.io_dtype
        U = torch.empty((r_max,) + tuple(R.shape), dtype=self.io_dtype, device="cuda")
        T = torch.empty_like(U)
        a = torch.zeros(r_max, dtype=torch.float64, device="cuda")
        code, rank, s_rel, rn = lrdm_krylov_step(self.handle, sys, R.data_ptr(), s_tol, r_max, alpha,
                                                 rho.data_ptr() if rho is not None else 0,
                                                 U.data_ptr(), T.data_ptr(), a.data_ptr(),
                                                 self._stream(stream))
        _check("lrdm_krylov_step", code)
        return dict(U=U[:rank], T=T[:rank], a=a[:rank], rank=rank, s_rel=s_rel, r_norm=rn)

    def tuning(self):
        """Launch shape of the tensor-core contractions (defaults or autotuned)."""
        return lrdm_get_tuning(self.handle)

    def set_tuning(self, g1_nb=None, g1_dpt=None, g2_bn=None, g2_kgroup=None):
        """Pins the launch shape (unset fields keep their current value)."""
        t = self.tuning()
        _check("lrdm_set_tuning", lrdm_set_tuning(
            self.handle, t["g1_nb"] if g1_nb is None else g1_nb, t["g1_dpt"] if g1_dpt is None else g1_dpt,
            t["g2_bn"] if g2_bn is None else g2_bn, t["g2_kgroup"] if g2_kgroup is None else g2_kgroup))

    def profile(self, on=True):
        _check("lrdm_profile_enable", lrdm_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self, reset=True):
        return lrdm_profile_read(self.handle, 1 if reset else 0)

    def status(self, synchronize=True):
        return lrdm_status_query(self.handle, 1 if synchronize else 0)


class KpContext:
    """Owns one Brillouin-zone-sampled lrdm_ctx (lrdm_kp_create).

    psi_re / psi_im: per k-point (N_g, N_s) device tensors in the io dtype
    (real and imaginary planes of the lattice-periodic subspace, orthonormal
    under the grid quadrature); eps: per k-point float64 device tensors;
    k_weights: floats summing to 1.  Directions and results are (K, N_g) in
    the io dtype.
    """

    def __init__(self, n, h, psi_re, psi_im, eps, k_weights, n_electrons, kT, g=2.0,
                 rho=None, rho_floor=0.0, prec="fp64", io_dtype=None, k_max=16, degen_tol=1e-5,
                 autotune=False, use_graph=False, stream=None):
        import torch
        self.torch = torch
        self.io_dtype = io_dtype or torch.float64
        o = lrdm_default_options()
        o.prec = PRECISIONS[prec]
        o.io_dtype = DTYPE_F64 if self.io_dtype == torch.float64 else DTYPE_F32
        o.k_max = int(k_max)
        o.degen_tol = float(degen_tol)
        o.autotune = 1 if autotune else 0
        o.use_graph = 1 if use_graph else 0
        nk = len(psi_re)
        assert len(psi_im) == nk and len(eps) == nk and len(k_weights) == nk
        s = lrdm_kpoint_system()
        for i in range(3):
            s.n[i] = int(n[i])
            s.h[i] = float(h[i])
        s.nk = nk
        ns = int(psi_re[0].shape[1])
        s.ns = ns
        s.ld_psi = int(psi_re[0].stride(0))
        for t in list(psi_re) + list(psi_im):
            assert t.is_cuda and t.dtype == self.io_dtype and t.dim() == 2
            assert t.shape[1] == ns and t.stride(1) == 1 and t.stride(0) == s.ld_psi
        for e in eps:
            assert e.is_cuda and e.dtype == torch.float64 and e.is_contiguous() and e.numel() == ns
        pr = (c_void_p * nk)(*[t.data_ptr() for t in psi_re])
        pi = (c_void_p * nk)(*[t.data_ptr() for t in psi_im])
        pe = (c_void_p * nk)(*[e.data_ptr() for e in eps])
        kw = (c_double * nk)(*[float(x) for x in k_weights])
        s.psi_re = ctypes.cast(pr, POINTER(c_void_p))
        s.psi_im = ctypes.cast(pi, POINTER(c_void_p))
        s.eps = ctypes.cast(pe, POINTER(c_void_p))
        s.k_weights = ctypes.cast(kw, POINTER(c_double))
        keep = []
        if rho is not None:
            rho = rho.to(self.io_dtype).contiguous()
            s.rho = rho.data_ptr()
            keep.append(rho)
        s.n_electrons = float(n_electrons)
        s.kT = float(kT)
        s.occ_factor = float(g)
        s.rho_floor = float(rho_floor)
        s.k_max = 0
        self.Ng = int(np.prod(n))
        self.k_max = int(k_max)
        code, hd = lrdm_kp_create(s, o, self._stream(stream))
        _check("lrdm_kp_create", code)
        self.handle = hd
        del keep

    def _stream(self, stream):
        if stream is None:
            return self.torch.cuda.current_stream().cuda_stream
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def close(self):
        if getattr(self, "handle", None):
            lrdm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mu(self):
        return lrdm_get_mu(self.handle, 0)

    def density(self, stream=None):
        out = self.torch.empty(self.Ng, dtype=self.io_dtype, device="cuda")
        _check("lrdm_get_density", lrdm_get_density(self.handle, 0, 0, out.data_ptr(),
                                                    self._stream(stream)))
        return out

    def gateaux(self, V, out=None, dmu=None, stream=None):
        """f_k = drho_k - v_k for V (K, N_g); returns (F, dmu)."""
        torch = self.torch
        assert V.is_contiguous() and V.dtype == self.io_dtype and V.shape[-1] == self.Ng
        K = int(V.shape[0])
        F = out if out is not None else torch.empty_like(V)
        if dmu is None:
            dmu = torch.empty(max(1, K), dtype=torch.float64, device="cuda")
        _check("lrdm_kp_gateaux", lrdm_kp_gateaux(self.handle, V.data_ptr(), K, F.data_ptr(),
                                                  dmu.data_ptr(), self._stream(stream)))
        return F, dmu[:K]

    def apply(self, R, V, F, alpha, rho=None, stream=None):
        """The least-squares step on K derivatives (lrdm_apply, sys 0)."""
        torch = self.torch
        K = int(V.shape[0])
        coeff = torch.empty(K, dtype=torch.float64, device="cuda")
        s_rel = torch.empty(1, dtype=torch.float64, device="cuda")
        _check("lrdm_apply", lrdm_apply(self.handle, 0, R.data_ptr(), V.data_ptr(), F.data_ptr(), K,
                                        float(alpha), rho.data_ptr() if rho is not None else 0,
                                        coeff.data_ptr(), s_rel.data_ptr(), self._stream(stream)))
        return coeff, s_rel

    def profile(self, on=True):
        _check("lrdm_profile_enable", lrdm_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self, reset=True):
        return lrdm_profile_read(self.handle, 1 if reset else 0)

    def tuning(self):
        """Launch shape of the tensor-core contractions (defaults or autotuned)."""
        return lrdm_get_tuning(self.handle)

    def set_tuning(self, g1_nb=None, g1_dpt=None, g2_bn=None, g2_kgroup=None):
        """Pins the launch shape (unset fields keep their current value)."""
        t = self.tuning()
        _check("lrdm_set_tuning", lrdm_set_tuning(
            self.handle, t["g1_nb"] if g1_nb is None else g1_nb, t["g1_dpt"] if g1_dpt is None else g1_dpt,
            t["g2_bn"] if g2_bn is None else g2_bn, t["g2_kgroup"] if g2_kgroup is None else g2_kgroup))

    def split(self, K):
        """Grid-row ranges of the projection for a K-direction call."""
        v = c_int()
        _check("lrdm_kp_get_split", load().lrdm_kp_get_split(self.handle, int(K), ctypes.byref(v)))
        return v.value

    def backward(self, fbar, out=None, stream=None):
        """v_bar = J^T f_bar for the most recent gateaux call (lrdm_backward);
        fbar, v_bar: (K, N_g) in the io dtype."""
        assert fbar.is_contiguous() and fbar.dtype == self.io_dtype
        vbar = out if out is not None else self.torch.empty_like(fbar)
        _check("lrdm_backward", lrdm_backward(self.handle, [fbar.data_ptr()], [vbar.data_ptr()],
                                              None, None, self._stream(stream)))
        return vbar

    def krylov_step(self, R, s_tol=0.3, r_max=8, alpha=-1.0, rho=None, stream=None):
        """The paper's adaptive-rank LRDM step (lrdm_krylov_step) on this
        BZ-sampled system.  R: (N_g,) in the io dtype; rho (same shape) is
        updated in place when given.  Returns dict(U, T, a, rank, s_rel, r_norm)."""
        torch = self.torch
        assert R.is_contiguous() and R.dtype == self.io_dtype and R.numel() == self.Ng
        U = torch.empty((r_max, self.Ng), dtype=self.io_dtype, device="cuda")
        T = torch.empty_like(U)
        a = torch.zeros(r_max, dtype=torch.float64, device="cuda")
        code, rank, s_rel, rn = lrdm_krylov_step(self.handle, 0, R.data_ptr(), s_tol, r_max, alpha,
                                                 rho.data_ptr() if rho is not None else 0,
                                                 U.data_ptr(), T.data_ptr(), a.data_ptr(),
                                                 self._stream(stream))
        _check("lrdm_krylov_step", code)
        return dict(U=U[:rank], T=T[:rank], a=a[:rank], rank=rank, s_rel=s_rel, r_norm=rn)

    def status(self, synchronize=True):
        return lrdm_status_query(self.handle, 1 if synchronize else 0)


class Lrdma:
    """The accumulated LRDM driver (lrdm_lrdma_*): a history of directions and
    Gateaux derivatives kept across SCF steps, for grid functions of
    n = nspin * N_g values in the io dtype with quadrature weight w."""

    def __init__(self, n, io_dtype, w, capacity=16):
        import torch
        self.torch = torch
        code_io = DTYPE_F64 if io_dtype == torch.float64 else DTYPE_F32
        self.n, self.io_dtype, self.w = int(n), io_dtype, float(w)
        h = c_void_p()
        _check("lrdm_lrdma_create", load().lrdm_lrdma_create(ctypes.byref(h), int(n), code_io,
                                                              float(w), int(capacity)))
        self.handle = h

    def step(self, ctx, R, rho=None, sys=0, stream=None, **params):
        """One LRDMA step with context `ctx` (its current subspace); params
        override the paper's settings (s_tol, beta_tol, r_norm_clear, alpha,
        r_max_iter, r_max).  rho is updated in place.  Returns the report."""
        p = lrdm_lrdma_params()
        load().lrdm_lrdma_default_params(ctypes.byref(p))
        for k, v in params.items():
            setattr(p, k, v)
        rep = lrdm_lrdma_report()
        st = ctx._stream(stream)
        _check("lrdm_lrdma_step", load().lrdm_lrdma_step(self.handle, ctx.handle, sys,
                                                          c_void_p(R.data_ptr()),
                                                          c_void_p(rho.data_ptr() if rho is not None else 0),
                                                          ctypes.byref(p), ctypes.byref(rep),
                                                          c_void_p(st)))
        return dict(event=LRDMA_EVENTS[rep.event], rank=rep.rank, rank_new=rep.rank_new,
                    s_rel=rep.s_rel, beta=rep.beta if rep.beta >= 0 else None, r_norm=rep.r_norm,
                    alpha=rep.alpha)

    def clear(self):
        _check("lrdm_lrdma_clear", load().lrdm_lrdma_clear(self.handle))

    def save(self, path):
        """Writes the history (U, T, R_lin, rank and flags) to an .npz file."""
        m, fl = c_int(), c_int()
        _check("lrdm_lrdma_get_state", load().lrdm_lrdma_get_state(self.handle, ctypes.byref(m),
                                                                    ctypes.byref(fl)))
        dt = np.float64 if self.io_dtype == self.torch.float64 else np.float32
        U = np.zeros((max(m.value, 1), self.n), dtype=dt)
        T = np.zeros_like(U)
        R = np.zeros(self.n, dtype=dt)
        _check("lrdm_lrdma_export", load().lrdm_lrdma_export(self.handle, c_void_p(U.ctypes.data),
                                                              c_void_p(T.ctypes.data),
                                                              c_void_p(R.ctypes.data), c_void_p(0)))
        np.savez(path, U=U[:m.value], T=T[:m.value], R_lin=R, m=m.value, flags=fl.value,
                 n=self.n, w=self.w)

    def load(self, path):
        """Restores a history written by save() (same n and io dtype)."""
        d = np.load(path)
        dt = np.float64 if self.io_dtype == self.torch.float64 else np.float32
        if int(d["n"]) != self.n:
            raise ValueError("history of another grid size")
        m = int(d["m"])
        if m:
            U = np.ascontiguousarray(d["U"], dtype=dt)
            T = np.ascontiguousarray(d["T"], dtype=dt)
        else:
            U = T = np.zeros((1, self.n), dtype=dt)
        R = np.ascontiguousarray(d["R_lin"], dtype=dt)
        _check("lrdm_lrdma_import", load().lrdm_lrdma_import(self.handle, m, int(d["flags"]),
                                                              c_void_p(U.ctypes.data), c_void_p(T.ctypes.data),
                                                              c_void_p(R.ctypes.data), c_void_p(0)))

    def close(self):
        if getattr(self, "handle", None):
            load().lrdm_lrdma_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gateaux_function():
    """torch.autograd.Function whose forward is lrdm_gateaux_batch on one system
    (a Context; V (K, nspin, N_g)) or lrdm_kp_gateaux (a KpContext; V (K, N_g))
    and whose backward is lrdm_backward (the hand-written adjoint)."""
    import torch

    class LrdmResponse(torch.autograd.Function):
        @staticmethod
        def forward(fctx, lctx, V):
            fctx.lctx = lctx
            if isinstance(lctx, KpContext):
                F, _ = lctx.gateaux(V.detach().contiguous())
                return F
            (F,), _ = lctx.gateaux([V.detach().contiguous()])
            return F

        @staticmethod
        def backward(fctx, gF):
            if isinstance(fctx.lctx, KpContext):
                return None, fctx.lctx.backward(gF.contiguous())
            vbar, _, _ = fctx.lctx.backward([gF.contiguous()], want_eps=False)
            return None, vbar[0]

    return LrdmResponse
