"""Python binding of the GB300 IGS-GMRES library (``include/igs.h``, ``_build/libigs.so``).

Argument marshalling only: every step of the solver runs in the library's CUDA kernels.
There is no CPU fallback; if the library cannot be loaded, every entry point raises.

Vectors may be numpy arrays (host memory) or CUDA ``torch.Tensor`` objects (device
memory, float64, contiguous); the library is told which through its ``on_device`` flags.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Any

import numpy as np

__all__ = ["Solver", "BatchSolver", "Server", "block_csr", "IGSError", "load_library", "library_path", "status_string",
           "OK", "NOT_CONVERGED", "BREAKDOWN", "EINVAL", "ENOMEM", "ECUDA", "ENUMERIC",
           "KCLASS_NAMES", "EXPORTED_SYMBOLS", "EXPORTED_BATCH_SYMBOLS",
           "EXPORTED_SERVE_SYMBOLS"]

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, ENOTIMPL = -1, -2, -3, -4, -5, -6
KCLASS_NAMES = ["spmv", "dots", "update", "small", "cycle"]

# Every function declared in include/igs.h.
EXPORTED_SYMBOLS = ["igs_create", "igs_destroy", "igs_solve", "igs_arnoldi", "igs_spmv",
                    "igs_get_info", "igs_profile_enable", "igs_profile_get", "igs_launch_count",
                    "igs_status_string", "igs_last_error", "igs_block_dots_static", "igs_arnoldi_ex",
                    "igs_probe_fma"]
# Every function declared in include/igs_batch.h.
EXPORTED_BATCH_SYMBOLS = ["igs_batch_create", "igs_batch_destroy", "igs_batch_solve",
                          "igs_batch_set_config", "igs_batch_tune", "igs_batch_get_info",
                          "igs_batch_get_norms", "igs_batch_last_error"]
# Every function declared in include/igs_serve.h.
EXPORTED_SERVE_SYMBOLS = ["igs_server_create", "igs_server_destroy", "igs_server_submit",
                          "igs_server_pump", "igs_server_poll", "igs_server_take_result",
                          "igs_server_get_stats", "igs_server_clock", "igs_server_last_error",
                          "igs_server_gang_selftest"]

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libigs.so")


class IGSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class _CreateOpts(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("device", C.c_int), ("max_restart_m", C.c_int),
                ("A_norm2", C.c_double), ("norm2_iters", C.c_int), ("fp32_basis", C.c_int),
                ("stream_alloc", C.c_int)]


class _SolveOpts(C.Structure):
    _fields_ = [("restart_m", C.c_int), ("gs_iters", C.c_int), ("tol_beta", C.c_double),
                ("max_restarts", C.c_int), ("inputs_on_device", C.c_int), ("precision", C.c_int),
                ("inner_tol", C.c_double), ("method", C.c_int)]


PRECISIONS = {"fp64": 0, "fp32_ir": 1, "fp64_df": 2}
# Arnoldi processes: Alg. 4.1 (two-reduce IGS) and Alg. 4.2 (one-reduce hybrid MGS-CGS).
METHODS = {"igs": 1, "one_reduce": 2}


class _Result(C.Structure):
    _fields_ = [("x", C.c_void_p), ("arnoldi_hist", C.c_void_p), ("lfro_hist", C.c_void_p),
                ("hist_cap", C.c_int64), ("hist_len", C.c_int64), ("H", C.c_void_p),
                ("H_ld", C.c_int), ("beta", C.c_double), ("rho0", C.c_double),
                ("steps", C.c_int64), ("cycles", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("max_restart_m", C.c_int),
                ("device", C.c_int), ("A_norm2", C.c_double), ("A_norm2_estimated", C.c_int),
                ("device_bytes", C.c_int64)]


class _Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 5), ("launches", C.c_int64 * 5), ("bytes", C.c_double * 5),
                ("flops", C.c_double * 5)]


class _BatchOpts(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("device", C.c_int), ("restart_m", C.c_int),
                ("A_norm2", C.c_void_p), ("norm2_iters", C.c_int), ("block_threads", C.c_int),
                ("blocks_per_sm", C.c_int)]


class _BatchSolveOpts(C.Structure):
    _fields_ = [("gs_iters", C.c_int), ("tol_beta", C.c_double), ("max_restarts", C.c_int),
                ("inputs_on_device", C.c_int)]


class _BatchResult(C.Structure):
    _fields_ = [("x", C.c_void_p), ("beta", C.c_void_p), ("status", C.c_void_p),
                ("steps", C.c_void_p), ("cycles", C.c_void_p), ("total_steps", C.c_int64),
                ("n_ok", C.c_int), ("n_not_converged", C.c_int), ("n_breakdown", C.c_int),
                ("n_numeric", C.c_int), ("device_ms", C.c_double)]


class _TuneEntry(C.Structure):
    _fields_ = [("block_threads", C.c_int), ("blocks_per_sm", C.c_int), ("ms", C.c_double)]


class _BatchInfo(C.Structure):
    _fields_ = [("count", C.c_int), ("total_rows", C.c_int64), ("nnz", C.c_int64),
                ("max_rows", C.c_int), ("restart_m", C.c_int), ("block_threads", C.c_int),
                ("blocks_per_sm", C.c_int), ("num_sms", C.c_int), ("smem_bytes", C.c_int64),
                ("basis_bytes", C.c_int64), ("n_tune", C.c_int), ("tune", _TuneEntry * 32)]


class _ServerOpts(C.Structure):
    _fields_ = [("device", C.c_int), ("max_restart_m", C.c_int), ("arena_bytes", C.c_int64),
                ("slots", C.c_int), ("rows_per_cta", C.c_int), ("max_queue", C.c_int),
                ("graph_min_n", C.c_int64), ("graph_lanes", C.c_int)]


class _Request(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("vals", C.c_void_p), ("b", C.c_void_p), ("x0", C.c_void_p), ("A_norm2", C.c_double),
                ("restart_m", C.c_int), ("gs_iters", C.c_int), ("tol_beta", C.c_double),
                ("max_restarts", C.c_int), ("precision", C.c_int), ("inner_tol", C.c_double)]


class _Completion(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("beta", C.c_double), ("steps", C.c_int64),
                ("cycles", C.c_int), ("gang_ctas", C.c_int), ("device_bytes", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("path", C.c_int), ("A_norm2", C.c_double)]


class _ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("queued", C.c_int64), ("running", C.c_int64),
                ("completed", C.c_int64), ("arena_bytes", C.c_int64), ("arena_used", C.c_int64),
                ("arena_peak", C.c_int64), ("launches", C.c_int64)]


_lib = None


def load_library(path: str | None = None):
    """Load libigs.so (built by ``paper_2205_07805_gb300.build``).  Raises if missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_2205_07805_gb300.build.build())")
    lib = C.CDLL(p)
    vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
    lib.igs_create.argtypes = [C.POINTER(vp), i64, i64, vp, vp, vp, C.POINTER(_CreateOpts)]
    lib.igs_create.restype = i32
    lib.igs_destroy.argtypes = [vp]
    lib.igs_destroy.restype = None
    lib.igs_solve.argtypes = [vp, vp, vp, C.POINTER(_SolveOpts), C.POINTER(_Result)]
    lib.igs_solve.restype = i32
    lib.igs_arnoldi.argtypes = [vp, vp, i32, i32, i32, vp, i64, vp, vp, C.POINTER(i32), C.POINTER(dbl)]
    lib.igs_arnoldi.restype = i32
    lib.igs_arnoldi_ex.argtypes = [vp, vp, i32, i32, i32, i32, i32, vp, i64, vp, vp, C.POINTER(i32), C.POINTER(dbl)]
    lib.igs_arnoldi_ex.restype = i32
    lib.igs_spmv.argtypes = [vp, vp, vp, i32]
    lib.igs_spmv.restype = i32
    lib.igs_get_info.argtypes = [vp, C.POINTER(_Info)]
    lib.igs_get_info.restype = i32
    lib.igs_profile_enable.argtypes = [vp, i32]
    lib.igs_profile_enable.restype = i32
    lib.igs_profile_get.argtypes = [vp, C.POINTER(_Profile)]
    lib.igs_profile_get.restype = i32
    lib.igs_launch_count.argtypes = [vp]
    lib.igs_launch_count.restype = i64
    lib.igs_status_string.argtypes = [i32]
    lib.igs_status_string.restype = C.c_char_p
    lib.igs_last_error.argtypes = [vp]
    lib.igs_last_error.restype = C.c_char_p
    lib.igs_block_dots_static.argtypes = [vp, i64, i32, i64, vp, vp, vp, vp]
    lib.igs_block_dots_static.restype = i32
    lib.igs_probe_fma.argtypes = [i32, C.POINTER(dbl), C.POINTER(dbl)]
    lib.igs_probe_fma.restype = i32
    lib.igs_batch_create.argtypes = [C.POINTER(vp), i32, vp, vp, vp, vp, C.POINTER(_BatchOpts)]
    lib.igs_batch_create.restype = i32
    lib.igs_batch_destroy.argtypes = [vp]
    lib.igs_batch_destroy.restype = None
    lib.igs_batch_solve.argtypes = [vp, vp, vp, C.POINTER(_BatchSolveOpts), C.POINTER(_BatchResult)]
    lib.igs_batch_solve.restype = i32
    lib.igs_batch_set_config.argtypes = [vp, i32, i32]
    lib.igs_batch_set_config.restype = i32
    lib.igs_batch_tune.argtypes = [vp, i32, dbl, i32]
    lib.igs_batch_tune.restype = i32
    lib.igs_batch_get_info.argtypes = [vp, C.POINTER(_BatchInfo)]
    lib.igs_batch_get_info.restype = i32
    lib.igs_batch_get_norms.argtypes = [vp, vp]
    lib.igs_batch_get_norms.restype = i32
    lib.igs_batch_last_error.argtypes = [vp]
    lib.igs_batch_last_error.restype = C.c_char_p
    lib.igs_server_create.argtypes = [C.POINTER(vp), C.POINTER(_ServerOpts)]
    lib.igs_server_create.restype = i32
    lib.igs_server_destroy.argtypes = [vp]
    lib.igs_server_destroy.restype = None
    lib.igs_server_submit.argtypes = [vp, C.POINTER(_Request), C.POINTER(i64)]
    lib.igs_server_submit.restype = i32
    lib.igs_server_pump.argtypes = [vp, C.POINTER(i32)]
    lib.igs_server_pump.restype = i32
    lib.igs_server_poll.argtypes = [vp, C.POINTER(_Completion), i32, C.POINTER(i32)]
    lib.igs_server_poll.restype = i32
    lib.igs_server_take_result.argtypes = [vp, i64, vp]
    lib.igs_server_take_result.restype = i32
    lib.igs_server_get_stats.argtypes = [vp, C.POINTER(_ServerStats)]
    lib.igs_server_get_stats.restype = i32
    lib.igs_server_clock.argtypes = [vp]
    lib.igs_server_clock.restype = dbl
    lib.igs_server_last_error.argtypes = [vp]
    lib.igs_server_last_error.restype = C.c_char_p
    lib.igs_server_gang_selftest.argtypes = [i32, i32, i32, C.POINTER(i32)]
    lib.igs_server_gang_selftest.restype = i32
    if path is None:
        _lib = lib
    return lib


def status_string(code: int) -> str:
    return load_library().igs_status_string(code).decode()


def _is_tensor(x: Any) -> bool:
    return type(x).__module__.startswith("torch") and hasattr(x, "data_ptr")


def _vec_arg(x, n: int, name: str):
    """(pointer, on_device, keepalive) for a float64 vector of length n."""
    if _is_tensor(x):
        import torch
        if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous() or x.numel() != n:
            raise ValueError(f"{name}: need a contiguous CUDA float64 tensor of length {n}")
        return C.c_void_p(x.data_ptr()), True, x
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.shape != (n,):
        raise ValueError(f"{name}: need shape ({n},), got {a.shape}")
    return C.c_void_p(a.ctypes.data), False, a


def probe_fma(device: int = 0) -> dict:
    """FP64 and FP32 FMA throughput of the GPU (``igs_probe_fma``), in FMAs per second."""
    lib = load_library()
    f64, f32 = C.c_double(0.0), C.c_double(0.0)
    rc = lib.igs_probe_fma(int(device), C.byref(f64), C.byref(f32))
    if rc != OK:
        raise IGSError(rc, "igs_probe_fma")
    return {"fp64_fma_per_s": f64.value, "fp32_fma_per_s": f32.value}


class Solver:
    """IGS-GMRES solver context for one sparse matrix (``igs_create``).

    ``A`` is any object with ``n``, ``rowptr`` (int64, n+1), ``colind`` (int32) and ``val``
    (float64) attributes, or a tuple ``(n, rowptr, colind, val)``."""

    def __init__(self, A, max_restart_m: int = 100, A_norm2: float | None = None,
                 device: int = 0, stream: int | None = None, norm2_iters: int = 100,
                 fp32_basis: bool = False):
        self._lib = load_library()
        if isinstance(A, tuple):
            n, rowptr, colind, val = A
        else:
            n, rowptr, colind, val = A.n, A.rowptr, A.colind, A.val
        self.n = int(n)
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(colind, dtype=np.int32)
        va = np.ascontiguousarray(val, dtype=np.float64)
        opts = _CreateOpts(C.c_void_p(stream) if stream else None, int(device), int(max_restart_m),
                           float(A_norm2) if A_norm2 else 0.0, int(norm2_iters), 1 if fp32_basis else 0)
        h = C.c_void_p()
        rc = self._lib.igs_create(C.byref(h), self.n, int(rp[-1]), C.c_void_p(rp.ctypes.data),
                                  C.c_void_p(ci.ctypes.data), C.c_void_p(va.ctypes.data), C.byref(opts))
        if rc != OK:
            raise IGSError(rc, "igs_create: " + self._lib.igs_last_error(None).decode())
        self._h = h
        self.max_restart_m = int(max_restart_m)

    # ------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.igs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _err(self, rc: int, what: str):
        raise IGSError(rc, f"{what}: {self._lib.igs_status_string(rc).decode()}: "
                           f"{self._lib.igs_last_error(self._h).decode()}")

    @property
    def info(self) -> dict:
        inf = _Info()
        self._lib.igs_get_info(self._h, C.byref(inf))
        return {k: getattr(inf, k) for k, _ in _Info._fields_}

    @property
    def launches(self) -> int:
        return int(self._lib.igs_launch_count(self._h))

    # ------------------------------------------------------------------------------
    def solve(self, b, x0=None, m: int = 30, gs: int = 2, tol: float = 1e-13,
              max_restarts: int = 10, x_out=None, hist_cap: int | None = None,
              want_H: bool = False, precision: str = "fp64", inner_tol: float = 0.0,
              method: str = "igs") -> dict:
        """Restarted IGS-GMRES(m) (``igs_solve``).  Returns ``dict(x, status, beta, rho0,
        steps, cycles, hist_res, hist_lfro[, H])``.  With a CUDA tensor ``b`` the inputs and
        ``x`` stay on the device.  ``precision="fp32_ir"`` runs the cycles on the FP32 basis
        inside FP64 iterative refinement (context created with ``fp32_basis=True``)."""
        bp, dev, kb = _vec_arg(b, self.n, "b")
        if x0 is not None:
            xp, dev0, kx = _vec_arg(x0, self.n, "x0")
            if dev0 != dev:
                raise ValueError("b and x0 must both be host or both be device arrays")
        else:
            xp, kx = None, None
        if x_out is None:
            if dev:
                import torch
                x_out = torch.empty(self.n, dtype=torch.float64, device=b.device)
            else:
                x_out = np.empty(self.n)
        op, devo, ko = _vec_arg(x_out, self.n, "x_out")
        if devo != dev:
            raise ValueError("x_out must live where b lives")
        cap = hist_cap if hist_cap is not None else m * max_restarts
        hres = np.full(max(cap, 1), np.nan)
        hlf = np.full(max(cap, 1), np.nan)
        H = np.zeros((m + 1, m), order="F") if want_H else None
        res = _Result(op, C.c_void_p(hres.ctypes.data), C.c_void_p(hlf.ctypes.data), cap, 0,
                      C.c_void_p(H.ctypes.data) if want_H else None, m + 1, 0.0, 0.0, 0, 0)
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        if method not in METHODS:
            raise ValueError(f"method must be one of {sorted(METHODS)}")
        opts = _SolveOpts(int(m), int(gs), float(tol), int(max_restarts), 1 if dev else 0,
                          PRECISIONS[precision], float(inner_tol), METHODS[method])
        rc = self._lib.igs_solve(self._h, bp, xp, C.byref(opts), C.byref(res))
        if rc < 0:
            self._err(rc, "igs_solve")
        k = int(res.hist_len)
        out = {"x": x_out, "status": rc, "beta": res.beta, "rho0": res.rho0, "steps": int(res.steps),
               "cycles": int(res.cycles), "hist_res": hres[:k].copy(), "hist_lfro": hlf[:k].copy()}
        if want_H:
            out["H"] = H
        return out

    def arnoldi(self, r0, m: int, gs: int = 2, V=None, H=None, L=None, method: str = "igs",
                precision: str = "fp64") -> dict:
        """One Arnoldi cycle (``igs_arnoldi``).  Host input gives numpy outputs
        (V: n x (m+1), H: (m+1) x m, L: (m+1) x (m+1) row-major); a CUDA tensor input gives
        CUDA tensor outputs unless output tensors are passed."""
        rp, dev, kr = _vec_arg(r0, self.n, "r0")
        if dev:
            import torch
            if V is None:
                V = torch.zeros((m + 1, self.n), dtype=torch.float64, device=r0.device)  # column j = row j
            if H is None:
                H = torch.zeros((m, m + 1), dtype=torch.float64, device=r0.device)
            if L is None:
                L = torch.zeros((m + 1, m + 1), dtype=torch.float64, device=r0.device)
            vptr, hptr, lptr = V.data_ptr(), H.data_ptr(), L.data_ptr()
        else:
            V = np.zeros((self.n, m + 1), order="F")
            H = np.zeros((m + 1, m), order="F")
            L = np.zeros((m + 1, m + 1))
            vptr, hptr, lptr = V.ctypes.data, H.ctypes.data, L.ctypes.data
        ncols = C.c_int(0)
        rho = C.c_double(0.0)
        if method not in METHODS:
            raise ValueError(f"method must be one of {sorted(METHODS)}")
        if precision not in ("fp64", "fp64_df"):
            raise ValueError("arnoldi runs precision 'fp64' or 'fp64_df'")
        rc = self._lib.igs_arnoldi_ex(self._h, rp, int(m), METHODS[method], int(gs), PRECISIONS[precision],
                                      1 if dev else 0,
                                      C.c_void_p(vptr), self.n, C.c_void_p(hptr), C.c_void_p(lptr),
                                      C.byref(ncols), C.byref(rho))
        if rc < 0:
            self._err(rc, "igs_arnoldi")
        if dev:  # tensors were laid out column-major via transposed shapes
            V, H = V.T, H.T
        return {"V": V, "H": H, "L": L, "ncols": ncols.value, "rho": rho.value, "status": rc}

    def spmv(self, x, y=None):
        """y = A x (``igs_spmv``)."""
        xp, dev, kx = _vec_arg(x, self.n, "x")
        if y is None:
            if dev:
                import torch
                y = torch.empty(self.n, dtype=torch.float64, device=x.device)
            else:
                y = np.empty(self.n)
        yp, devy, ky = _vec_arg(y, self.n, "y")
        rc = self._lib.igs_spmv(self._h, xp, yp, 1 if dev else 0)
        if rc != OK:
            self._err(rc, "igs_spmv")
        return y

    # ------------------------------------------------------------------------------
    def profile_enable(self, on: bool = True):
        self._lib.igs_profile_enable(self._h, 1 if on else 0)

    def profile(self) -> dict:
        p = _Profile()
        self._lib.igs_profile_get(self._h, C.byref(p))
        return {name: {"ms": p.ms[i], "launches": int(p.launches[i]), "bytes": p.bytes[i],
                       "flops": p.flops[i]} for i, name in enumerate(KCLASS_NAMES)}


# ----------------------------------------------------------------------------------------
# Batched solver (include/igs_batch.h)
# ----------------------------------------------------------------------------------------
def block_csr(systems):
    """Concatenate square CSR systems (objects with n, rowptr, colind, val) into the
    block-diagonal CSR that ``igs_batch_create`` takes: ``(sys_ptr, rowptr, colind, val)``
    with global column indices."""
    ns = np.array([int(A.n) for A in systems], dtype=np.int64)
    sys_ptr = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(ns, out=sys_ptr[1:])
    nnzs = np.array([int(A.rowptr[-1]) for A in systems], dtype=np.int64)
    nz_off = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(nnzs, out=nz_off[1:])
    rowptr = np.empty(int(sys_ptr[-1]) + 1, dtype=np.int64)
    rowptr[-1] = nz_off[-1]
    colind = np.empty(int(nz_off[-1]), dtype=np.int32)
    val = np.empty(int(nz_off[-1]), dtype=np.float64)
    for s, A in enumerate(systems):
        r0, r1 = int(sys_ptr[s]), int(sys_ptr[s + 1])
        rowptr[r0:r1] = np.asarray(A.rowptr[:-1], dtype=np.int64) + nz_off[s]
        colind[nz_off[s]:nz_off[s + 1]] = np.asarray(A.colind, dtype=np.int64) + r0
        val[nz_off[s]:nz_off[s + 1]] = A.val
    return sys_ptr, rowptr, colind, val


class BatchSolver:
    """Many independent systems solved by one persistent launch (``igs_batch_create``).

    ``systems`` is a list of CSR objects (n, rowptr, colind, val) or a tuple
    ``(sys_ptr, rowptr, colind, val)`` in block-diagonal form.  ``A_norm2``: per-system
    ||A_s||_2 (sequence) or None to estimate them on the GPU.  ``block_threads`` and
    ``blocks_per_sm`` both 0: tune the launch configuration at creation."""

    def __init__(self, systems, m: int = 50, A_norm2=None, device: int = 0,
                 stream: int | None = None, block_threads: int = 0, blocks_per_sm: int = 0,
                 norm2_iters: int = 100):
        self._lib = load_library()
        if isinstance(systems, tuple):
            sys_ptr, rowptr, colind, val = systems
        else:
            sys_ptr, rowptr, colind, val = block_csr(systems)
        self.sys_ptr = np.ascontiguousarray(sys_ptr, dtype=np.int64)
        self.count = len(self.sys_ptr) - 1
        self.N = int(self.sys_ptr[-1])
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(colind, dtype=np.int32)
        va = np.ascontiguousarray(val, dtype=np.float64)
        nrm = None
        if A_norm2 is not None:
            nrm = np.ascontiguousarray(A_norm2, dtype=np.float64)
            if nrm.shape != (self.count,):
                raise ValueError(f"A_norm2: need {self.count} values")
        opts = _BatchOpts(C.c_void_p(stream) if stream else None, int(device), int(m),
                          C.c_void_p(nrm.ctypes.data) if nrm is not None else None,
                          int(norm2_iters), int(block_threads), int(blocks_per_sm))
        h = C.c_void_p()
        rc = self._lib.igs_batch_create(C.byref(h), self.count, C.c_void_p(self.sys_ptr.ctypes.data),
                                        C.c_void_p(rp.ctypes.data), C.c_void_p(ci.ctypes.data),
                                        C.c_void_p(va.ctypes.data), C.byref(opts))
        if rc != OK:
            raise IGSError(rc, "igs_batch_create")
        self._h = h
        self.m = int(m)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.igs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _err(self, rc: int, what: str):
        raise IGSError(rc, f"{what}: {self._lib.igs_status_string(rc).decode()}: "
                           f"{self._lib.igs_batch_last_error(self._h).decode()}")

    @property
    def info(self) -> dict:
        inf = _BatchInfo()
        self._lib.igs_batch_get_info(self._h, C.byref(inf))
        out = {k: getattr(inf, k) for k, _ in _BatchInfo._fields_ if k != "tune"}
        out["tune"] = [(inf.tune[i].block_threads, inf.tune[i].blocks_per_sm, inf.tune[i].ms)
                       for i in range(inf.n_tune)]
        return out

    def norms(self) -> np.ndarray:
        out = np.empty(self.count)
        self._lib.igs_batch_get_norms(self._h, C.c_void_p(out.ctypes.data))
        return out

    def set_config(self, block_threads: int, blocks_per_sm: int):
        rc = self._lib.igs_batch_set_config(self._h, int(block_threads), int(blocks_per_sm))
        if rc != OK:
            self._err(rc, "igs_batch_set_config")

    def tune(self, gs: int = 2, tol: float = 1e-12, max_restarts: int = 20):
        rc = self._lib.igs_batch_tune(self._h, int(gs), float(tol), int(max_restarts))
        if rc != OK:
            self._err(rc, "igs_batch_tune")

    def solve(self, b, x0=None, gs: int = 2, tol: float = 1e-12, max_restarts: int = 20,
              x_out=None, out=None) -> dict:
        """Solve every system (``igs_batch_solve``).  Host numpy ``b`` gives numpy results;
        a CUDA tensor ``b`` keeps everything on the device (``out`` may pass preallocated
        device tensors x, beta, status, steps, cycles).  Returns ``dict(x, beta, status,
        steps, cycles, rc, total_steps, n_ok, n_not_converged, n_breakdown, n_numeric,
        device_ms)``."""
        bp, dev, kb = _vec_arg(b, self.N, "b")
        if x0 is not None:
            xp, dev0, kx = _vec_arg(x0, self.N, "x0")
            if dev0 != dev:
                raise ValueError("b and x0 must both be host or both be device arrays")
        else:
            xp, kx = None, None
        if dev:
            import torch
            o = dict(out or {})
            dv = b.device
            if x_out is not None:
                o["x"] = x_out
            o.setdefault("x", torch.empty(self.N, dtype=torch.float64, device=dv))
            o.setdefault("beta", torch.empty(self.count, dtype=torch.float64, device=dv))
            o.setdefault("status", torch.empty(self.count, dtype=torch.int32, device=dv))
            o.setdefault("steps", torch.empty(self.count, dtype=torch.int64, device=dv))
            o.setdefault("cycles", torch.empty(self.count, dtype=torch.int32, device=dv))
            ptr = {k: C.c_void_p(v.data_ptr()) for k, v in o.items()}
        else:
            o = {"x": np.empty(self.N) if x_out is None else x_out,
                 "beta": np.empty(self.count), "status": np.empty(self.count, dtype=np.int32),
                 "steps": np.empty(self.count, dtype=np.int64),
                 "cycles": np.empty(self.count, dtype=np.int32)}
            ptr = {k: C.c_void_p(v.ctypes.data) for k, v in o.items()}
        res = _BatchResult(ptr["x"], ptr["beta"], ptr["status"], ptr["steps"], ptr["cycles"],
                           0, 0, 0, 0, 0, 0.0)
        opts = _BatchSolveOpts(int(gs), float(tol), int(max_restarts), 1 if dev else 0)
        rc = self._lib.igs_batch_solve(self._h, bp, xp, C.byref(opts), C.byref(res))
        if rc < 0 and rc != ENUMERIC:
            self._err(rc, "igs_batch_solve")
        o.update(rc=rc, total_steps=int(res.total_steps), n_ok=res.n_ok,
                 n_not_converged=res.n_not_converged, n_breakdown=res.n_breakdown,
                 n_numeric=res.n_numeric, device_ms=res.device_ms)
        return o


# ----------------------------------------------------------------------------------------
# Request server (include/igs_serve.h)
# ----------------------------------------------------------------------------------------
class Server:
    """Continuous-batching request server (``igs_server_create``).  ``submit`` queues a
    request (host arrays), ``pump`` admits what fits and collects finished requests,
    ``poll`` returns completion records, ``take`` the solution of a completed request.
    Requests with n >= ``graph_min_n`` (when > 0) take a graph lane (``path`` 1 in their
    completion record); ``graph_lanes`` of them run at once."""

    def __init__(self, max_restart_m: int = 100, arena_bytes: int = 1 << 30, slots: int = 8,
                 rows_per_cta: int = 4096, max_queue: int = 0, device: int = 0, graph_min_n: int = 0,
                 graph_lanes: int = 1):
        self._lib = load_library()
        opts = _ServerOpts(int(device), int(max_restart_m), int(arena_bytes), int(slots),
                           int(rows_per_cta), int(max_queue), int(graph_min_n), int(graph_lanes))
        h = C.c_void_p()
        rc = self._lib.igs_server_create(C.byref(h), C.byref(opts))
        if rc != OK:
            raise IGSError(rc, "igs_server_create")
        self._h = h
        self._n = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.igs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _err(self, rc: int, what: str):
        raise IGSError(rc, f"{what}: {self._lib.igs_status_string(rc).decode()}: "
                           f"{self._lib.igs_server_last_error(self._h).decode()}")

    def submit(self, A, b, x0=None, A_norm2: float = 0.0, m: int = 100, gs: int = 2,
               tol: float = 1e-12, max_restarts: int = 100, precision: str = "fp64",
               inner_tol: float = 0.0):
        """Queue one request; returns its id, or None when the queue is full."""
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.colind, dtype=np.int32)
        va = np.ascontiguousarray(A.val, dtype=np.float64)
        bb = np.ascontiguousarray(b, dtype=np.float64)
        xx = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        req = _Request(int(A.n), int(rp[-1]), C.c_void_p(rp.ctypes.data), C.c_void_p(ci.ctypes.data),
                       C.c_void_p(va.ctypes.data), C.c_void_p(bb.ctypes.data),
                       C.c_void_p(xx.ctypes.data) if xx is not None else None, float(A_norm2),
                       int(m), int(gs), float(tol), int(max_restarts), PRECISIONS[precision],
                       float(inner_tol))
        rid = C.c_int64(0)
        rc = self._lib.igs_server_submit(self._h, C.byref(req), C.byref(rid))
        if rc == ENOMEM:
            return None
        if rc != OK:
            self._err(rc, "igs_server_submit")
        self._n[rid.value] = int(A.n)
        return rid.value

    def pump(self) -> int:
        running = C.c_int(0)
        rc = self._lib.igs_server_pump(self._h, C.byref(running))
        if rc != OK:
            self._err(rc, "igs_server_pump")
        return running.value

    def poll(self, max_out: int = 256) -> list:
        buf = (_Completion * max_out)()
        k = C.c_int(0)
        self._lib.igs_server_poll(self._h, buf, int(max_out), C.byref(k))
        return [{f: getattr(buf[i], f) for f, _ in _Completion._fields_} for i in range(k.value)]

    def take(self, rid: int) -> np.ndarray:
        x = np.empty(self._n[rid])
        rc = self._lib.igs_server_take_result(self._h, int(rid), C.c_void_p(x.ctypes.data))
        if rc != OK:
            self._err(rc, "igs_server_take_result")
        del self._n[rid]
        return x

    def stats(self) -> dict:
        st = _ServerStats()
        self._lib.igs_server_get_stats(self._h, C.byref(st))
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def clock(self) -> float:
        return float(self._lib.igs_server_clock(self._h))

    def run_all(self, sleep_s: float = 0.0005) -> list:
        """Pump until nothing is queued or running; returns all completion records."""
        import time
        out = []
        while True:
            running = self.pump()
            out += self.poll()
            st = self.stats()
            if running == 0 and st["queued"] == 0:
                out += self.poll()
                return out
            time.sleep(sleep_s)
