"""CPU oracle for IGS-GMRES (arXiv 2205.07805) -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``igs_oracle.c``: a plain, slow, serial FP64 restatement of the
paper's Alg. 4.1 (IGS-GMRES with one or two Gauss-Seidel iterations) and of MGS-GMRES.
Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library and never imports it.

Layouts: ``V`` is n x (m+1) (returned as a numpy array with ``V[:, j]`` the j-th basis
vector), ``H`` is (m+1) x m, ``L`` is (m+1) x (m+1) strictly lower (row i = v_{i+1}^T V_i).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "igs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libigs_oracle.so")
_OMP_PATH = os.path.join(_OUT_DIR, "libigs_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp = None
_FLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]

MGS, IGS, ONE_REDUCE = 0, 1, 2  # MGS-GMRES, Alg. 4.1, Alg. 4.2
OK, NOT_CONVERGED, BREAKDOWN, EINVAL, ENOMEM, ENUMERIC = 0, 1, 2, -1, -2, -4

_P = np.ctypeslib.ndpointer
_d = C.c_double
_i64 = C.c_int64


def _compile(path: str, extra: list, force: bool) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *_FLAGS, *extra, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (serial, no FMA contraction): the parity build."""
    return _compile(_LIB_PATH, [], force)


def build_openmp(force: bool = False) -> str:
    """Compile the timing build: the same source with -fopenmp.  Its parallel loops write
    disjoint outputs, each formed exactly as in the serial build, so its results are
    bitwise those of ``build()`` (checked by the tests); it exists only to time the oracle
    on all host cores (threads from OMP_NUM_THREADS, default all)."""
    return _compile(_OMP_PATH, ["-fopenmp"], force)


def openmp() -> "Oracle":
    """The OpenMP timing build, for the ``impl=`` argument of the functions below."""
    global _omp
    with _lock:
        if _omp is None:
            _omp = Oracle(build_openmp())
        return _omp


def openmp_threads() -> int:
    """Threads the OpenMP build will use (its omp_get_max_threads())."""
    return int(openmp().lib.ora_threads())


class Oracle:
    """Bindings to one compiled copy of the oracle (the default build, or a variant
    compiled by a test from a modified copy of the source)."""

    def __init__(self, lib_path: str):
        lib = C.CDLL(lib_path)
        f64 = _P(dtype=np.float64, flags="C_CONTIGUOUS")
        f64F = _P(dtype=np.float64, flags="F_CONTIGUOUS")
        i64 = _P(dtype=np.int64, flags="C_CONTIGUOUS")
        i32 = _P(dtype=np.int32, flags="C_CONTIGUOUS")
        lib.ora_spmv.argtypes = [_i64, i64, i32, f64, f64, f64]
        lib.ora_spmv.restype = None
        lib.ora_dot.argtypes = [_i64, f64, f64]
        lib.ora_dot.restype = _d
        lib.ora_arnoldi.argtypes = [_i64, i64, i32, f64, f64, C.c_int, C.c_int, C.c_int, f64F,
                                    f64F, f64, C.POINTER(_d), C.POINTER(C.c_int)]
        lib.ora_arnoldi.restype = C.c_int
        lib.ora_hessenberg_lsq.argtypes = [C.c_int, C.c_int, f64F, _d, f64]
        lib.ora_hessenberg_lsq.restype = _d
        lib.ora_backward_error.argtypes = [_i64, i64, i32, f64, f64, f64, _d]
        lib.ora_backward_error.restype = _d
        lib.ora_gmres.argtypes = [_i64, i64, i32, f64, f64, f64, f64, C.c_int, C.c_int, C.c_int,
                                  _d, C.c_int, _d, _i64, f64, f64, C.POINTER(_i64),
                                  C.POINTER(_d), C.POINTER(C.c_int), C.POINTER(_i64)]
        lib.ora_gmres.restype = C.c_int
        if hasattr(lib, "ora_threads"):
            lib.ora_threads.argtypes = []
            lib.ora_threads.restype = C.c_int
        self.lib = lib
        self.path = lib_path


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a (test-modified) copy of the oracle source to ``out_path``."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", *_FLAGS, "-o", out_path, src, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load(which: "Oracle | None" = None):
    global _lib
    if which is not None:
        return which.lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build()).lib
        return _lib


def _csr(A):
    return (int(A.n), np.ascontiguousarray(A.rowptr, dtype=np.int64),
            np.ascontiguousarray(A.colind, dtype=np.int32),
            np.ascontiguousarray(A.val, dtype=np.float64))


def spmv(A, x, impl: Oracle | None = None) -> np.ndarray:
    """y = A x, row by row in storage order."""
    lib = _load(impl)
    n, rp, ci, va = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n)
    lib.ora_spmv(n, rp, ci, va, x, y)
    return y


def dot(x, y, impl: Oracle | None = None) -> float:
    lib = _load(impl)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib.ora_dot(x.size, x, y))


def arnoldi(A, r0, m: int, method: int = IGS, gs: int = 2, impl: Oracle | None = None) -> dict:
    """One Arnoldi cycle (Alg. 4.1 for ``method=IGS``, MGS otherwise) on start vector r0.

    Returns ``dict(V, H, L, ncols, rho, status)``; only the first ``ncols`` columns of H
    (and ``ncols + 1`` of V) are meaningful."""
    lib = _load(impl)
    n, rp, ci, va = _csr(A)
    r0 = np.ascontiguousarray(r0, dtype=np.float64)
    V = np.zeros((n, m + 1), order="F")
    H = np.zeros((m + 1, m), order="F")
    L = np.zeros((m + 1, m + 1))
    rho = _d(0.0)
    st = C.c_int(0)
    ncols = lib.ora_arnoldi(n, rp, ci, va, r0, m, method, gs, V, H, L, C.byref(rho), C.byref(st))
    return {"V": V, "H": H, "L": L, "ncols": int(ncols), "rho": rho.value, "status": st.value}


def hessenberg_lsq(H, p: int, rho: float, impl: Oracle | None = None):
    """Givens least squares on the first p columns of H; returns (y, residual)."""
    lib = _load(impl)
    H = np.asfortranarray(H, dtype=np.float64)
    m = H.shape[1]
    y = np.zeros(max(p, 1))
    res = lib.ora_hessenberg_lsq(m, p, H, rho, y)
    return y[:p], float(res)


def backward_error(A, b, x, normA: float, impl: Oracle | None = None) -> float:
    lib = _load(impl)
    n, rp, ci, va = _csr(A)
    return float(lib.ora_backward_error(n, rp, ci, va, np.ascontiguousarray(b, dtype=np.float64),
                                        np.ascontiguousarray(x, dtype=np.float64), normA))


def gmres(A, b, x0=None, m: int = 30, method: int = IGS, gs: int = 2, tol: float = 1e-14,
          max_cycles: int = 10, normA: float = 1.0, hist_cap: int | None = None,
          impl: Oracle | None = None) -> dict:
    """Restarted GMRES(m).  Returns ``dict(x, status, beta, cycles, steps, hist_res,
    hist_lfro)``; ``hist_res[j]`` is the Arnoldi residual |g_{j+1}| after column j (each
    cycle restarts the column count) and ``hist_lfro[j]`` = ||L_{j+1}||_F (IGS only)."""
    lib = _load(impl)
    n, rp, ci, va = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x0 = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    x = np.empty(n)
    cap = hist_cap if hist_cap is not None else m * max_cycles
    hres = np.full(max(cap, 1), np.nan)
    hlf = np.full(max(cap, 1), np.nan)
    hlen = _i64(0)
    beta = _d(0.0)
    cycles = C.c_int(0)
    steps = _i64(0)
    st = lib.ora_gmres(n, rp, ci, va, b, x0, x, m, method, gs, tol, max_cycles, normA, cap,
                       hres, hlf, C.byref(hlen), C.byref(beta), C.byref(cycles), C.byref(steps))
    k = int(hlen.value)
    return {"x": x, "status": int(st), "beta": beta.value, "cycles": cycles.value,
            "steps": int(steps.value), "hist_res": hres[:k], "hist_lfro": hlf[:k]}
