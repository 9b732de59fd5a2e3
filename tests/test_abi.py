"""The C-ABI library loads and exports every symbol include/lsm.h declares; host-side argument checks.

Runs on the CPU: loading liblsm.so makes no CUDA call, and the argument
checks below reject their inputs before any device work starts.
"""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsm.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_12836_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_2301_12836_gb300 import lsm
    return lsm.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("lsm_create", "lsm_create_shared", "lsm_source", "lsm_apply", "lsm_apply_c64", "lsm_adjoint",
                 "lsm_solve", "lsm_solve_batched", "lsm_destroy", "lsm_last_error", "lsm_default_opts"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2301_12836_gb300 import lsm
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(lsm.EXPORTS) == names


def test_default_opts(lib):
    from paper_2301_12836_gb300 import lsm
    o = lsm.lsm_default_opts()
    assert o.precision == lsm.LSM_FP64 and o.green == lsm.LSM_GREEN_EXACT
    assert o.tol == 1e-10 and o.maxit >= 100 and o.inner_tol == 1e-6 and o.max_outer >= 2 and o.taper == 0
    assert o.graph == 1 and o.kernel == lsm.LSM_KERNEL_DIFF
    assert o.residual == lsm.LSM_RESIDUAL_FP64   # the benchmark spec's FP64 refinement residual
    assert o.fused_dots == 1   # alpha's and omega's inner products summed in the FP32 epilogue


def test_opts_binding_matches_the_header():
    """The ctypes lsm_opts lists the header's fields in the header's order with matching C types
    (int / double), so the struct the binding passes has the library's layout."""
    from paper_2301_12836_gb300 import lsm
    with open(HEADER) as f:
        text = f.read()
    body = text[text.index("typedef struct {", text.index("LSM_RESIDUAL_FP64")):text.index("} lsm_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    decl = re.findall(r"\b(int|double)\s+(\w+)\s*;", body)
    ctypes_of = {"int": ct.c_int, "double": ct.c_double}
    assert [(n, ctypes_of[t]) for t, n in decl] == list(lsm.lsm_opts._fields_)


@pytest.mark.parametrize("n,ok", [((2, 2, 2), True), ((1, 4, 4), False), ((7, 4, 4), False),
                                  ((4, 4, 257), False), ((5, 6, 9), True)])
def test_create_rejects_bad_grids_before_any_device_work(lib, n, ok):
    from paper_2301_12836_gb300 import lsm
    out = ct.c_void_p()
    arr = (ct.c_int * 3)(*n)
    o = lsm.lsm_default_opts()
    # a good grid is given null contrast pointers and fails on them; a bad grid gets stand-in
    # pointers that are never dereferenced because the grid check comes first
    ptr = None if ok else ct.c_void_p(16)
    code = lib.lsm_create(ct.byref(out), arr, 10.0, 1e9, 1e9, 2000.0, ptr, ptr, 1.0, ct.byref(o), None)
    assert code == lsm.LSM_ERR_ARG
    assert out.value is None
    msg = lib.lsm_last_error(None).decode()
    if ok:
        assert "null pointer" in msg
    else:
        assert "each n" in msg


@pytest.mark.parametrize("field,val", [("dx", 0.0), ("mu0", -1.0), ("rho0", 0.0), ("omega", 0.0), ("omega", -3.0)])
def test_create_rejects_bad_physics(lib, field, val):
    from paper_2301_12836_gb300 import lsm
    args = dict(dx=10.0, lam=1e9, mu0=1e9, rho0=2000.0, omega=1.0)
    key = {"dx": "dx", "mu0": "mu0", "rho0": "rho0", "omega": "omega"}[field]
    args[key] = val
    out = ct.c_void_p()
    arr = (ct.c_int * 3)(4, 4, 4)
    fake = ct.c_void_p(16)  # never dereferenced: validation fails first
    code = lib.lsm_create(ct.byref(out), arr, args["dx"], args["lam"], args["mu0"], args["rho0"], fake, fake,
                          args["omega"], None, None)
    assert code == lsm.LSM_ERR_ARG


def test_bad_options_rejected(lib):
    from paper_2301_12836_gb300 import lsm
    out = ct.c_void_p()
    arr = (ct.c_int * 3)(4, 4, 4)
    fake = ct.c_void_p(16)
    for kw in (dict(precision=7), dict(green=3), dict(tol=0.0), dict(maxit=0), dict(inner_tol=-1.0), dict(max_outer=0),
               dict(taper=-2), dict(graph=2), dict(kernel=2), dict(kernel=-1), dict(residual=2),
               dict(fused_dots=2), dict(fused_dots=-1)):
        o = lsm.lsm_default_opts(**kw)
        code = lib.lsm_create(ct.byref(out), arr, 10.0, 1e9, 1e9, 2000.0, fake, fake, 1.0, ct.byref(o), None)
        assert code == lsm.LSM_ERR_ARG, kw


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2301_12836_gb300 import lsm
    assert lib.lsm_apply(None, None, None) == lsm.LSM_ERR_ARG
    assert lib.lsm_adjoint(None, None, None) == lsm.LSM_ERR_ARG
    assert lib.lsm_solve(None, None, None, None, None) == lsm.LSM_ERR_ARG
    assert lib.lsm_solve_batched(0, None, None, None, None, None, None) == lsm.LSM_ERR_ARG
    assert lib.lsm_source_moments(None, 1, None, None, None) == lsm.LSM_ERR_ARG
    assert lib.lsm_set_schedule(None, 0, None) == lsm.LSM_ERR_ARG
    assert lib.lsm_autotune(None, 1, 1, None, None) == lsm.LSM_ERR_ARG
    assert lib.lsm_dot_c64(None, 0, None, None, None) == lsm.LSM_ERR_ARG
    lib.lsm_destroy(None)
    assert lib.lsm_launch_count(None) == 0
