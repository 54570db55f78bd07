"""The IGS_PREC_FP64_DF form (block reductions in double-float arithmetic on the FP32 pipes)
against the FP64 oracle (needs a GB300; -m gpu).

The form keeps every vector, the SpMV, the basis updates and the small steps in FP64 and
evaluates the reductions of Alg. 4.1 steps 5 and 14 (Alg. 4.2 step 4) as double-float dot
products, from n = 16384 rows on.  It must meet the same bars as the FP64 form: H columns
within 1e-10 while kappa(B_k) < 1e6 (two iterations; one iteration: the FP64 noise floor
2 eps kappa(B_k) where larger), the Arnoldi relation and two-iteration orthogonality within
1e-13, the library's L equal to strict_lower(V^T V) to 1e-14, and solves with the oracle's
status, beta <= tol and step counts within +-2.  Below 16384 rows the form runs the FP64
reductions, so its results are bitwise the FP64 form's.
"""
import numpy as np
import pytest

import _parity as P
import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2205_07805_gb300 as pkg
    from paper_2205_07805_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


CASES = {
    "cd2d_130": gen.cd2d(130, 50.0, seed=3),    # n = 16900: just above the threshold, ragged tail
    "cd2d_256": gen.cd2d(256, 50.0, seed=1),    # n = 65536
    "cd3d_32": gen.cd3d(32, 20.0, seed=2),      # n = 32768, 7-point
}


def _norm(A):
    return gen.norm2_power(A, iters=100)


@pytest.mark.parametrize("name,m,gs,method", [("cd2d_130", 60, 2, "igs"), ("cd2d_256", 80, 2, "igs"),
                                              ("cd2d_256", 60, 1, "igs"), ("cd3d_32", 50, 2, "igs"),
                                              ("cd2d_256", 60, 2, "one_reduce")])
def test_df_arnoldi_parity(pkg, name, m, gs, method):
    A, b, _, _ = CASES[name]
    normA = _norm(A)
    with pkg.Solver(A, max_restart_m=m, A_norm2=normA) as s:
        g = s.arnoldi(b, m, gs=gs, method=method, precision="fp64_df")
    o = oracle.arnoldi(A, b, m, oracle.ONE_REDUCE if method == "one_reduce" else oracle.IGS, gs,
                       impl=oracle.openmp())
    assert g["ncols"] == o["ncols"] == m and g["status"] == o["status"]
    kap = P.kappa_prefix(A, b, o["V"], m)
    herr = P.h_column_errors(g["H"], o["H"], m)
    well = kap < 1e6
    assert well[0]
    tol = np.full(m, 1e-10) if gs == 2 else np.maximum(1e-10, 2 * P.EPS * kap)
    assert np.all(herr[well] <= tol[well]), f"max H column error ratio {(herr / tol)[well].max():.3g}"
    Vg = g["V"]
    assert P.arnoldi_relation(A, Vg, g["H"], m, normA) <= 1e-13
    if gs == 2:
        assert P.orth_loss(Vg, m + 1) <= 1e-13
    if method == "igs":
        Lref = np.tril(Vg[:, :m + 1].T @ Vg[:, :m + 1], -1)
        assert np.abs(g["L"][:m + 1, :m + 1] - Lref).max() <= 1e-14


@pytest.mark.parametrize("name,m,gs,tol,method", [("cd2d_130", 40, 2, 1e-12, "igs"), ("cd2d_256", 60, 1, 1e-10, "igs"),
                                                  ("cd2d_130", 40, 2, 1e-12, "one_reduce")])
def test_df_solve_parity(pkg, name, m, gs, tol, method):
    A, b, _, _ = CASES[name]
    normA = _norm(A)
    omp = oracle.openmp()
    meth = oracle.ONE_REDUCE if method == "one_reduce" else oracle.IGS
    o = oracle.gmres(A, b, m=m, method=meth, gs=gs, tol=tol, max_cycles=300, normA=normA, impl=omp)
    with pkg.Solver(A, max_restart_m=m, A_norm2=normA) as s:
        g = s.solve(b, m=m, gs=gs, tol=tol, max_restarts=300, method=method, precision="fp64_df")
    assert g["status"] == o["status"] == oracle.OK, (g["status"], o["status"])
    assert g["beta"] <= tol
    assert abs(g["steps"] - o["steps"]) <= 2, (g["steps"], o["steps"])
    assert oracle.backward_error(A, b, g["x"], normA) <= tol


def test_df_full_size_cycle(pkg):
    """The benchmark workload (cd2d 512 x 512, m = 100, two iterations) in the double-float
    form: H against the oracle's FP64 cycle, relation and orthogonality at full size."""
    A, b, _, _ = gen.cd2d(512, 50.0, seed=0)
    m = 100
    normA = gen.norm2_power(A, iters=50)
    with pkg.Solver(A, max_restart_m=m, A_norm2=normA) as s:
        g = s.arnoldi(b, m, gs=2, precision="fp64_df")
    o = oracle.arnoldi(A, b, m, oracle.IGS, 2, impl=oracle.openmp())
    kap = P.kappa_prefix(A, b, o["V"], m)
    herr = P.h_column_errors(g["H"], o["H"], m)
    assert herr[kap < 1e6].max() <= 1e-10
    assert P.orth_loss(g["V"], m + 1) <= 1e-13
    assert P.arnoldi_relation(A, g["V"], g["H"], m, normA) <= 1e-13


def test_df_small_systems_use_fp64_reductions(pkg):
    """Below 16384 rows the form runs the FP64 reductions: bitwise the FP64 form."""
    A, b, _, _ = gen.cd2d(100, 30.0, seed=5)  # n = 10000
    normA = _norm(A)
    with pkg.Solver(A, max_restart_m=30, A_norm2=normA) as s:
        a = s.arnoldi(b, 30, gs=2, precision="fp64")
        d = s.arnoldi(b, 30, gs=2, precision="fp64_df")
        xa = s.solve(b, m=30, gs=2, tol=0.0, max_restarts=2)
        xd = s.solve(b, m=30, gs=2, tol=0.0, max_restarts=2, precision="fp64_df")
    assert np.array_equal(a["H"], d["H"]) and np.array_equal(a["V"], d["V"])
    assert np.array_equal(xa["x"], xd["x"])


def test_df_out_of_range_is_enumeric(pkg):
    """The reductions see the normalised basis and A v: with ||A|| beyond the double-float
    range (entries of A v >= 2^127) they become non-finite and the solve stops with
    IGS_ENUMERIC instead of returning a wrong x; the FP64 form solves the same system."""
    A, b, _, _ = CASES["cd2d_130"]
    big = gen.CSR(A.n, A.rowptr.copy(), A.colind.copy(), A.val * 1e39)
    normA = _norm(A) * 1e39
    with pkg.Solver(big, max_restart_m=20, A_norm2=normA) as s:
        with pytest.raises(pkg.IGSError) as ei:
            s.solve(b, m=20, gs=2, tol=1e-12, max_restarts=2, precision="fp64_df")
        assert ei.value.code == pkg.ENUMERIC
        ok = s.solve(b, m=20, gs=2, tol=0.0, max_restarts=1)
    assert np.all(np.isfinite(ok["x"])) and ok["steps"] == 20


@pytest.mark.parametrize("method", ["igs", "one_reduce"])
def test_df_largest_restart_length(pkg, method):
    """The double-float form at the largest restart length (m = 232: multi-dots over up to
    233 columns in 59 column groups, the updates' coefficient splits at their largest) on a
    system above its 16384-row threshold: H against the oracle while kappa(B_k) < 1e6, the
    Arnoldi relation, and (two iterations) orthogonality."""
    A, b, _, _ = CASES["cd2d_130"]
    normA = _norm(A)
    m = 232
    with pkg.Solver(A, max_restart_m=m, A_norm2=normA) as s:
        g = s.arnoldi(b, m, gs=2, method=method, precision="fp64_df")
    o = oracle.arnoldi(A, b, m, oracle.ONE_REDUCE if method == "one_reduce" else oracle.IGS, 2,
                       impl=oracle.openmp())
    assert g["ncols"] == o["ncols"] == m and g["status"] == o["status"]
    kap = P.kappa_prefix(A, b, o["V"], m)
    herr = P.h_column_errors(g["H"], o["H"], m)
    well = kap < 1e6
    assert well.sum() > 10 and herr[well].max() <= 1e-10
    assert P.arnoldi_relation(A, g["V"], g["H"], m, normA) <= 1e-13
    assert P.orth_loss(g["V"], m + 1) <= 1e-13
