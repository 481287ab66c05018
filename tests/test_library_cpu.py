"""Host-side checks that need no GPU: the C-ABI library builds, loads, and
exports every function that include/*.h declares; option defaults; the
input generators' recipes."""

import os
import re

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lrdm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2211_07894_gb300 import build, binding
    build.build()
    return binding.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "lrdm_create" in names and "lrdm_gateaux_batch" in names
    assert "lrdm_apply" in names and "lrdm_backward" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options(lib):
    from paper_2211_07894_gb300 import binding
    o = binding.lrdm_default_options()
    assert o.prec == binding.PRECISIONS["bf16x3"] and o.io_dtype == binding.DTYPE_F32
    assert o.k_max == 16 and o.pinv_rcond == 1e-12 and o.degen_tol == 1e-5
    for code in range(10):
        assert binding.lrdm_status_string(code)


def test_create_rejects_bad_arguments_without_gpu(lib):
    """Argument validation runs before any device call."""
    from paper_2211_07894_gb300 import binding
    o = binding.lrdm_default_options()
    code, h = binding.lrdm_create([], o)
    assert code == 1 and not h.value
    s = binding.lrdm_system()
    s.nspin = 3
    code, h = binding.lrdm_create([s], o)
    assert code != 0 and not h.value
    o.k_max = 65
    s.nspin = 1
    code, _ = binding.lrdm_create([s], o)
    assert code != 0


def test_directions_are_unit_norm_and_zero_mean():
    n, h = (8, 6, 10), (0.5, 0.4, 0.3)
    V = workloads.smooth_directions(n, h, 3, 2, workloads.rng_for(0, 0))
    w = float(np.prod(h))
    for k in range(3):
        assert abs(w * np.sum(V[k] ** 2) - 1.0) < 1e-12
        assert np.all(np.abs(V[k].sum(axis=1)) < 1e-10)


def test_random_subspace_is_w_orthonormal():
    n, h = (8, 8, 8), (0.5, 0.5, 0.5)
    psi = workloads.random_subspace(n, h, 30, workloads.rng_for(0, 1))
    w = float(np.prod(h))
    assert np.max(np.abs(w * psi.T @ psi - np.eye(30))) < 1e-13


def test_degenerate_pairs_recipe():
    d = workloads.config4(scale=8)
    eps = d["eps"][0]
    gaps = np.diff(eps)
    for i in d["pairs"]:
        assert abs(gaps[i] - 1e-9) < 1e-15
    assert np.all(gaps > 0)


def test_library_exports_nothing_else(lib):
    """The library is built with hidden visibility: its exported functions are
    exactly those of include/*.h (std:: template instantiations aside)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_2211_07894_gb300 import build
    out = subprocess.run([nm, "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if len(ln.split()) == 3 and ln.split()[1] == "T"}
    assert exported == set(_declared_functions())


def test_no_cpu_fallback_without_a_gpu(lib):
    """Without a CUDA device the library refuses a valid system in every
    precision (no host fallback exists), and a missing library is an error."""
    import torch
    from paper_2211_07894_gb300 import binding
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    psi = np.zeros((64, 8), dtype=np.float32)
    eps = np.linspace(-1.0, 1.0, 8)
    for prec in binding.PRECISIONS.values():
        o = binding.lrdm_default_options()
        o.prec = prec
        s = binding.lrdm_system()
        s.n[0] = s.n[1] = s.n[2] = 4
        s.h[0] = s.h[1] = s.h[2] = 0.5
        s.nspin = 1
        s.ns[0] = s.ld_psi[0] = 8
        s.psi[0] = psi.ctypes.data
        s.eps[0] = eps.ctypes.data
        s.n_electrons, s.kT = 4.0, 0.01
        code, h = binding.lrdm_create([s], o)
        assert code != 0 and not h.value, prec
    with pytest.raises(OSError):
        binding.load(os.path.join(ROOT, "no_such_dir", "liblrdm.so"))


STRUCTS = ["lrdm_system", "lrdm_options", "lrdm_kpoint_system", "lrdm_lrdma_params", "lrdm_lrdma_report",
           "lrdm_rows"]


def test_binding_structs_match_the_header(tmp_path):
    """Every struct of include/lrdm.h as the binding declares it with ctypes:
    same size and the same offset for each field, and the enum values the
    binding hardcodes, checked against a C program compiled from the header
    (a drifted field or code would pass garbage through the boundary without
    any error)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2211_07894_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lrdm.h"', "int main(void) {"]
    for name in STRUCTS:
        st = getattr(binding, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    consts = {"LRDM_FP64": binding.PRECISIONS["fp64"], "LRDM_FP32": binding.PRECISIONS["fp32"],
              "LRDM_TF32": binding.PRECISIONS["tf32"], "LRDM_BF16X3": binding.PRECISIONS["bf16x3"],
              "LRDM_DTYPE_F64": binding.DTYPE_F64, "LRDM_DTYPE_F32": binding.DTYPE_F32,
              "LRDM_DEBUG_STALL_PROJECTION": binding.DEBUG_STALL_PROJECTION}
    events = ["LRDMA_FRESH", "LRDMA_REUSE", "LRDMA_ACCUMULATE", "LRDMA_CLEAR_LINEARITY",
              "LRDMA_CLEAR_RESIDUAL", "LRDMA_CLEAR_TRUNCATED"]
    for c in list(consts) + events:
        lines.append(f'  printf("const {c} %d\\n", (int)({c}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3:
            c_layout[(parts[0], parts[1])] = int(parts[2])
    for name in STRUCTS:
        st = getattr(binding, name)
        assert c_layout[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert c_layout[(name, field)] == getattr(st, field).offset, (name, field)
    for c, v in consts.items():
        assert c_layout[("const", c)] == v, c
    # the binding's event names in the header's order (fresh, reuse, accumulate, CL, CR, CT)
    assert [c_layout[("const", e)] for e in events] == sorted(binding.LRDMA_EVENTS)


def test_binding_argtypes_match_header_prototypes(lib):
    """Each prototype of include/lrdm.h has ctypes argtypes in the binding
    (without them ctypes would pass doubles and 64-bit pointers by guess),
    with the same number of parameters."""
    text = ""
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text += open(os.path.join(inc, fn)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"\b(lrdm_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S)
    assert len(protos) >= 20
    checked = 0
    for name, params in protos:
        params = " ".join(params.split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        argtypes = getattr(getattr(lib, name), "argtypes", None)
        assert argtypes is not None, f"{name} has no argtypes"
        assert len(argtypes) == n, (name, n, len(argtypes))
        checked += 1
    assert checked == len(protos)
