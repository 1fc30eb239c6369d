"""The C ABI library loads on a machine without a GPU and exports every entry point that
include/sa.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(sa_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libsa():
    from paper_1104_3830_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sa_scale", "sa_prune", "sa_solve_reduced", "sa_certify", "sa_submit", "sa_poll",
                 "sa_create", "sa_destroy", "sa_assign", "sa_batch_scale"):
        assert must in names


def test_every_declared_symbol_is_exported(libsa):
    missing = [n for n in sorted(declared_functions()) if not hasattr(libsa, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1104_3830_gb300 import _lib
    assert declared_functions() == set(_lib.SIGNATURES)


def test_host_only_entry_points_without_gpu(libsa):
    from paper_1104_3830_gb300 import _lib as L
    L._lib = None
    lib = L.lib()
    assert b"libsa" in lib.sa_version()
    # sa_solve_reduced is host-only: solve a 3x3 CSR exactly
    import numpy as np
    from paper_1104_3830_gb300 import api
    w = np.array([[1, 2, 3], [2, 4, 6], [3, 6, 10]], dtype=np.int32)
    rp = np.array([0, 3, 6, 9], dtype=np.int64)
    col = np.tile(np.arange(3, dtype=np.int32), 3)
    perm, s, al, be = api.sa_solve_reduced(rp, col, w.ravel())
    assert abs(s - max(np.log(w[0, a] * w[1, b] * w[2, c]) for a, b, c in
                       [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)])) < 1e-12
    # invalid arguments are reported as status codes, not crashes
    h = ctypes.c_void_p()
    st = lib.sa_create(ctypes.byref(h), 0, None)
    assert st != 0
    assert lib.sa_set_option(None, L.OPTION["wait_limit_ns"], 1000) == -1


def test_host_solver_argument_errors(libsa):
    """The host solve entry points report bad arguments as SA_E_INVALID (-1) with a message:
    NULL instance, NULL perm, NULL beta0, a column index out of range, n <= 0."""
    import numpy as np
    from paper_1104_3830_gb300 import _lib as L
    lib = L.lib()
    rp = np.array([0, 2, 4], dtype=np.int64)
    col = np.array([0, 1, 0, 1], dtype=np.int32)
    w = np.array([1, 2, 3, 4], dtype=np.int32)
    c = L.sa_csr(2, 4, rp.ctypes.data_as(L._I64P), col.ctypes.data_as(L._I32P), w.ctypes.data_as(L._I32P))
    perm = np.zeros(2, dtype=np.int32)
    b0 = np.zeros(2)
    pp, bp = perm.ctypes.data_as(L._I32P), b0.ctypes.data_as(L._DP)
    assert lib.sa_solve_reduced(None, pp, None, None, None) == -1
    assert lib.sa_solve_reduced(ctypes.byref(c), None, None, None, None) == -1
    for f in (lib.sa_solve_reduced_warm, lib.sa_solve_reduced_near):
        assert f(ctypes.byref(c), None, pp, None, None, None) == -1
        assert f(None, bp, pp, None, None, None) == -1
        assert f(ctypes.byref(c), bp, pp, None, None, None) == 0
        assert sorted(perm) == [0, 1]
    bad = np.array([0, 1, 0, 2], dtype=np.int32)
    cb = L.sa_csr(2, 4, rp.ctypes.data_as(L._I64P), bad.ctypes.data_as(L._I32P), w.ctypes.data_as(L._I32P))
    assert lib.sa_solve_reduced_near(ctypes.byref(cb), bp, pp, None, None, None) == -1
    assert b"out of range" in lib.sa_last_error()
    c0 = L.sa_csr(0, 0, rp.ctypes.data_as(L._I64P), col.ctypes.data_as(L._I32P), w.ctypes.data_as(L._I32P))
    assert lib.sa_solve_reduced_warm(ctypes.byref(c0), bp, pp, None, None, None) == -1
