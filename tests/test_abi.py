"""The C interface, without a GPU: the library builds, loads, exports every function that
include/igs.h declares, and rejects malformed input before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_07805_gb300 import build
    path = build.build()
    import paper_2205_07805_gb300 as pkg
    return pkg.load_library(path)


def test_exports_every_declared_function(lib):
    hdr = open(os.path.join(ROOT, "include", "igs.h")).read()
    declared = set(re.findall(r"\b(igs_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    import paper_2205_07805_gb300 as pkg
    assert declared == set(pkg.EXPORTED_SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def test_exports_every_declared_batch_function(lib):
    hdr = open(os.path.join(ROOT, "include", "igs_batch.h")).read()
    declared = set(re.findall(r"\b(igs_batch_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    import paper_2205_07805_gb300 as pkg
    assert declared == set(pkg.EXPORTED_BATCH_SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def test_exports_every_declared_serve_function(lib):
    hdr = open(os.path.join(ROOT, "include", "igs_serve.h")).read()
    declared = set(re.findall(r"\b(igs_server_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    import paper_2205_07805_gb300 as pkg
    assert declared == set(pkg.EXPORTED_SERVE_SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def test_server_rejects_bad_options_before_touching_the_device(lib):
    import paper_2205_07805_gb300 as pkg
    h = C.c_void_p()
    for opts in [(0, 0, 1 << 20, 0, 0, 0), (0, 200, 1 << 20, 0, 0, 0), (0, 50, 0, 0, 0, 0),
                 (0, 50, 1 << 20, 257, 0, 0), (0, 50, 1 << 20, 0, 100, 0), (0, 50, 1 << 20, 0, 0, 0, -1)]:
        o = pkg._ServerOpts(*opts)
        assert lib.igs_server_create(C.byref(h), C.byref(o)) == -1 and not h.value
    assert lib.igs_server_create(None, None) == -1
    assert lib.igs_server_gang_selftest(0, 1, 0, None) == -1      # a gang has >= 2 CTAs
    assert lib.igs_server_gang_selftest(0, 4, 2, None) == -1      # stall is 0 or 1
    lib.igs_server_destroy(None)
    assert lib.igs_server_submit(None, None, None) == -1
    assert lib.igs_server_pump(None, None) == -1
    assert lib.igs_server_get_stats(None, None) == -1
    assert lib.igs_server_last_error(None)


def test_status_strings(lib):
    for code in (0, 1, 2, -1, -2, -3, -4, -5, -6):
        assert lib.igs_status_string(code)
    assert lib.igs_status_string(12345) == b"unknown status"


def _create(lib, n, rowptr, colind, vals):
    h = C.c_void_p()
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    va = np.ascontiguousarray(vals, dtype=np.float64)
    rc = lib.igs_create(C.byref(h), n, int(rp[-1]) if rp.size else 0, C.c_void_p(rp.ctypes.data),
                        C.c_void_p(ci.ctypes.data), C.c_void_p(va.ctypes.data), None)
    return rc, h


def test_create_rejects_malformed_csr(lib):
    EINVAL, ENUMERIC = -1, -4
    rc, h = _create(lib, 2, [0, 1, 2], [0, 5], [1.0, 1.0])       # column out of range
    assert rc == EINVAL and not h.value
    rc, _ = _create(lib, 2, [0, 2, 1], [0, 1], [1.0, 1.0])       # decreasing rowptr
    assert rc == EINVAL
    rc, _ = _create(lib, 2, [1, 1, 2], [0, 1], [1.0, 1.0])       # rowptr[0] != 0
    assert rc == EINVAL
    rc, _ = _create(lib, 2, [0, 1, 2], [0, 1], [1.0, np.nan])    # non-finite value
    assert rc == ENUMERIC
    assert b"non-finite" in lib.igs_last_error(None)
    rc, _ = _create(lib, 0, [0], [], [])                         # n < 1
    assert rc == EINVAL


def test_null_arguments(lib):
    assert lib.igs_create(None, 1, 0, None, None, None, None) == -1
    lib.igs_destroy(None)
    assert lib.igs_solve(None, None, None, None, None) == -1
    assert lib.igs_spmv(None, None, None, 0) == -1
    assert lib.igs_launch_count(None) == -1


def test_missing_library_fails_loudly(tmp_path):
    import paper_2205_07805_gb300 as pkg
    with pytest.raises(RuntimeError):
        pkg.load_library(str(tmp_path / "nope.so"))


def _batch_create(lib, sys_ptr, rowptr, colind, vals, m=10, threads=0, bpsm=0):
    import paper_2205_07805_gb300 as pkg
    sp = np.ascontiguousarray(sys_ptr, dtype=np.int64)
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    va = np.ascontiguousarray(vals, dtype=np.float64)
    opts = pkg._BatchOpts(None, 0, m, None, 0, threads, bpsm)
    h = C.c_void_p()
    rc = lib.igs_batch_create(C.byref(h), len(sp) - 1, C.c_void_p(sp.ctypes.data),
                              C.c_void_p(rp.ctypes.data), C.c_void_p(ci.ctypes.data),
                              C.c_void_p(va.ctypes.data), C.byref(opts))
    return rc, h


def test_batch_create_rejects_malformed_input(lib):
    EINVAL, ENUMERIC = -1, -4
    # two 2x2 diagonal blocks; the second block's row 2 reaches into block 0
    rc, h = _batch_create(lib, [0, 2, 4], [0, 1, 2, 4, 5], [0, 1, 0, 2, 3], [1.0] * 5)
    assert rc == EINVAL and not h.value
    rc, _ = _batch_create(lib, [0, 2, 2], [0, 1, 2], [0, 1], [1.0, 1.0])          # empty block
    assert rc == EINVAL
    rc, _ = _batch_create(lib, [1, 2], [0, 1], [0], [1.0])                        # sys_ptr[0] != 0
    assert rc == EINVAL
    rc, _ = _batch_create(lib, [0, 2], [0, 2, 1], [0, 1], [1.0, 1.0])             # decreasing rowptr
    assert rc == EINVAL
    rc, _ = _batch_create(lib, [0, 2], [0, 1, 2], [0, 1], [1.0, np.inf])          # non-finite
    assert rc == ENUMERIC
    rc, _ = _batch_create(lib, [0, 2], [0, 1, 2], [0, 1], [1.0, 1.0], m=0)        # m < 1
    assert rc == EINVAL
    rc, _ = _batch_create(lib, [0, 2], [0, 1, 2], [0, 1], [1.0, 1.0], m=65)       # m too large
    assert rc == EINVAL
    rc, _ = _batch_create(lib, [0, 2], [0, 1, 2], [0, 1], [1.0, 1.0], threads=96)  # bad block size
    assert rc == EINVAL
    big = 16385                                                                   # block too large
    rc, _ = _batch_create(lib, [0, big], np.arange(big + 1), np.arange(big), np.ones(big))
    assert rc == EINVAL


def test_batch_null_arguments(lib):
    assert lib.igs_batch_create(None, 1, None, None, None, None, None) == -1
    lib.igs_batch_destroy(None)
    assert lib.igs_batch_solve(None, None, None, None, None) == -1
    assert lib.igs_batch_set_config(None, 256, 1) == -1
    assert lib.igs_batch_tune(None, 2, 1e-12, 10) == -1
    assert lib.igs_batch_get_info(None, None) == -1
    assert lib.igs_batch_get_norms(None, None) == -1
    assert lib.igs_batch_last_error(None)
