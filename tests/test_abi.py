"""Host-side checks of the C ABI: the library loads and exports every declared entry point,
and argument validation rejects bad input before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07522_gb300 as rs
    return rs


def declared():
    txt = open(os.path.join(ROOT, "include", "rsrr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rsrr_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(rs):
    names = declared()
    assert len(names) >= 14
    L = ctypes.CDLL(rs.LIB_PATH)
    for nm in names:
        assert hasattr(L, nm), nm
    assert set(rs.EXPORTS) >= set(names)


def test_version_and_error_without_device(rs):
    assert b"sm_103a" in rs.lib().rsrr_version()
    h = ctypes.c_void_p()
    rowptr = np.array([0, 1], dtype=np.int64)
    colind = np.array([0], dtype=np.int32)
    vals = np.array([1.0, 0.0])
    fn = (rs.rsrr_fn * 1)()
    rc = rs.lib().rsrr_create_nep(0, 1, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data, fn, 0,
                                  None, ctypes.byref(h))
    assert rc == -1 and b"n out of range" in rs.lib().rsrr_last_error()
    fn[0].kind = 42
    rc = rs.lib().rsrr_create_nep(1, 1, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data, fn, 0,
                                  None, ctypes.byref(h))
    assert rc == -1 and b"unknown function kind" in rs.lib().rsrr_last_error()
    fn[0].kind = 0
    bad = np.array([np.nan, 0.0])
    rc = rs.lib().rsrr_create_nep(1, 1, rowptr.ctypes.data, colind.ctypes.data, bad.ctypes.data, fn, 0,
                                  None, ctypes.byref(h))
    assert rc == -5
    unsorted = np.array([0, 2], dtype=np.int64)
    cols = np.array([1, 0], dtype=np.int32)
    rc = rs.lib().rsrr_create_nep(2, 1, np.array([0, 2, 2], dtype=np.int64).ctypes.data, cols.ctypes.data,
                                  np.zeros(4).ctypes.data, fn, 0, None, ctypes.byref(h))
    assert rc == -1 and b"strictly increasing" in rs.lib().rsrr_last_error()
    assert unsorted is not None


def test_null_handle_calls_fail_cleanly(rs):
    k = ctypes.c_int32()
    assert rs.lib().rsrr_project(None, 1e-14, ctypes.byref(k)) == -1
    assert rs.lib().rsrr_sample(None, None, 1, 1, None, 0, 1e-10, 1) == -1
    rs.lib().rsrr_destroy(None)


def test_product_path_never_loads_the_oracle():
    # the CUDA package imports nothing from oracle/; the oracle imports nothing from it
    pkg = os.path.join(ROOT, "paper_1510_07522_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle|#include\s+.*oracle", src, flags=re.M), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1510_07522_gb300", src, flags=re.M), f


def test_argument_checks_of_the_later_entry_points(rs):
    """Entry points beyond the core four reject a NULL handle, and rsrr_zgemm rejects a bad path,
    operation or leading dimension, before any device work."""
    L = rs.lib()
    k = ctypes.c_int32()
    assert L.rsrr_project_moments(None, 4, 1e-14, ctypes.byref(k)) == -1
    assert L.rsrr_project_chebyshev(None, 8, -1.0, 1.0, 1e-14, ctypes.byref(k)) == -1
    assert L.rsrr_set_band_preconditioner(None, 3) == -1
    assert L.rsrr_solve(None, 500, 2, 1e10, 10, None, None, None, None) == -1
    assert L.rsrr_sample_points(None, None, 4, None, 1, None, 0, 1e-10, 1) == -1
    info = ctypes.create_string_buffer(4096)
    assert L.rsrr_get_info(None, info) == -1
    buf = np.zeros(64)
    one = np.array([1.0, 0.0])
    zero = np.array([0.0, 0.0])
    p = buf.ctypes.data

    def zg(path, opA, opB, M, N, K, lda, ldb, ldc, batch=1):
        return L.rsrr_zgemm(path, opA, opB, M, N, K, one.ctypes.data, p, lda, 0, p, ldb, 0, zero.ctypes.data,
                            p, ldc, 0, batch, None)

    assert zg(3, 0, 0, 2, 2, 2, 2, 2, 2) == -1 and b"bad argument" in L.rsrr_last_error()
    assert zg(0, 3, 0, 2, 2, 2, 2, 2, 2) == -1
    assert zg(0, 0, 0, -1, 2, 2, 2, 2, 2) == -1
    assert zg(0, 0, 0, 2, 2, 2, 2, 2, 2, batch=0) == -1
    # op(A) = A is M x K: lda must be at least M; op(A) = A^H is K x M stored: lda at least K
    assert zg(0, 0, 0, 4, 2, 3, 3, 3, 4) == -1 and b"leading dimension" in L.rsrr_last_error()
    assert zg(0, 2, 0, 4, 2, 3, 2, 3, 4) == -1 and b"leading dimension" in L.rsrr_last_error()
    assert zg(0, 0, 0, 4, 2, 3, 4, 3, 3) == -1 and b"leading dimension" in L.rsrr_last_error()


def test_selftest_rejects_unknown_kind(rs):
    assert rs.lib().rsrr_selftest_bounded_wait(7, None) == -1
    assert b"kind" in rs.lib().rsrr_last_error()
