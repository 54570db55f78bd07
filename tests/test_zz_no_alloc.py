"""The allocation-free block multi-dot (igs_block_dots_static), called through the C
interface, against the existing entry point's output.

Some callers may not call cudaMalloc (a host application that owns all device memory, code
running during another thread's global-mode graph capture, loops that cannot take the
implicit synchronisation).  igs_block_dots_static serves them: its scratch is a fixed device
array.  This checks it against igs_arnoldi: the library's L satisfies L[k][c] = v_{k+1}^T v_c
to 1e-14 (the tolerance of the L tests), so V_k^T v_{k+1} from the new entry point must
match row k of L to the same tolerance -- on two calls in a row, since the calls share the
scratch array.  This file sorts last so that a run stopping at the first failure has run
every other test first.
"""
import ctypes as C

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def test_block_dots_static_matches_arnoldi():
    import torch

    import paper_2205_07805_gb300 as pkg
    from paper_2205_07805_gb300 import build
    build.build()
    lib = pkg.load_library()
    A, b, _, _ = gen.cd2d(64, 50.0, seed=2)  # n = 4096, a multiple of 4
    n, m = A.n, 30
    with pkg.Solver(A, max_restart_m=m, A_norm2=8.0) as s:
        arn = s.arnoldi(torch.from_numpy(b).cuda(), m, gs=2)
    V = arn["V"]                      # (n, m+1) view of a column-major device buffer
    Vbuf = V.T.contiguous()           # row j = basis vector j, i.e. column-major n x (m+1)
    L = arn["L"].cpu().numpy()
    stream = torch.cuda.current_stream()
    for k in (17, 29):                # two calls in a row share the scratch array
        out = torch.full((2 * k,), np.nan, dtype=torch.float64, device="cuda")
        x0 = Vbuf[k]
        x1 = Vbuf[k - 1]
        rc = lib.igs_block_dots_static(C.c_void_p(Vbuf.data_ptr()), n, k, n, C.c_void_p(x0.data_ptr()),
                                       C.c_void_p(x1.data_ptr()), C.c_void_p(out.data_ptr()),
                                       C.c_void_p(stream.cuda_stream))
        assert rc == pkg.OK
        got = out.cpu().numpy()
        # V_k^T v_{k+1} against row k of the library's L
        assert np.abs(got[:k] - L[k, :k]).max() <= 1e-14
        # V_k^T v_k: the last entry is ||v_k||^2 = 1 and the rest is row k-1 of L
        assert np.abs(got[k:2 * k - 1] - L[k - 1, :k - 1]).max() <= 1e-14
        assert abs(got[2 * k - 1] - 1.0) <= 1e-14
    # one vector (x1 = NULL): V_k^T v_k alone, against row k-1 of L and ||v_k||^2 = 1
    k = 23
    out = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
    rc = lib.igs_block_dots_static(C.c_void_p(Vbuf.data_ptr()), n, k, n, C.c_void_p(Vbuf[k - 1].data_ptr()),
                                   None, C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == pkg.OK
    got = out.cpu().numpy()
    assert np.abs(got[:k - 1] - L[k - 1, :k - 1]).max() <= 1e-14
    assert abs(got[k - 1] - 1.0) <= 1e-14
    # and both against a direct product in NumPy on the same basis (independent of the library's L)
    Vh = Vbuf.cpu().numpy()
    assert np.abs(got - Vh[:k] @ Vh[k - 1]).max() <= 1e-14


def test_block_dots_static_rejects_bad_sizes():
    import torch

    import paper_2205_07805_gb300 as pkg
    lib = pkg.load_library()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(4096, dtype=torch.float64, device="cuda")
    ptr = C.c_void_p(x.data_ptr())
    assert lib.igs_block_dots_static(ptr, 64, 1, 62, ptr, None, C.c_void_p(out.data_ptr()), None) == pkg.EINVAL
    # 2 x 20000 partial sums exceed the fixed 16384-entry scratch array
    big = torch.zeros(8 * 20000, dtype=torch.float64, device="cuda")
    assert lib.igs_block_dots_static(C.c_void_p(big.data_ptr()), 8, 20000, 8, ptr, ptr,
                                     C.c_void_p(out.data_ptr()), None) == pkg.EINVAL
    # just above the widest launch the kernel can compute (8 columns per block, 3 blocks per
    # SM): rejected with and without x1, before anything is launched
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pmax = min(24 * sms, 8192)
    wide = torch.zeros(8 * (pmax + 1), dtype=torch.float64, device="cuda")
    for x1 in (ptr, None):
        assert lib.igs_block_dots_static(C.c_void_p(wide.data_ptr()), 8, pmax + 1, 8, ptr, x1,
                                         C.c_void_p(out.data_ptr()), None) == pkg.EINVAL
    # the widest accepted launch on this GPU runs and is right (8 rows, pmax columns)
    Vw = torch.randn(pmax, 8, dtype=torch.float64, device="cuda")
    xw = torch.randn(8, dtype=torch.float64, device="cuda")
    yw = torch.randn(8, dtype=torch.float64, device="cuda")
    outw = torch.full((2 * pmax,), np.nan, dtype=torch.float64, device="cuda")
    assert lib.igs_block_dots_static(C.c_void_p(Vw.data_ptr()), 8, pmax, 8, C.c_void_p(xw.data_ptr()),
                                     C.c_void_p(yw.data_ptr()), C.c_void_p(outw.data_ptr()), None) == pkg.OK
    Vn = Vw.cpu().numpy()
    ref = np.concatenate([Vn @ xw.cpu().numpy(), Vn @ yw.cpu().numpy()])
    assert np.abs(outw.cpu().numpy() - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
