"""Edge cases of the single-system library against the oracle (needs a GB300; -m gpu):
the largest restart length the context allows (m = 232: every single-block step at its
shared-memory limit, the (I+L) solves at p up to 232), a 1 x 1 system, and a matrix with
empty CSR rows.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import _parity as P
import gen
import oracle

pytestmark = pytest.mark.gpu

M_MAX = 232


@pytest.fixture(scope="module")
def pkg():
    import paper_2205_07805_gb300 as pkg
    from paper_2205_07805_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


@pytest.fixture(scope="module")
def big_m_case():
    A, b, _, _ = gen.cd2d(30, 20.0, seed=11)                 # n = 900 > m + 1
    return A, b, gen.norm2_power(A, iters=100)


@pytest.mark.parametrize("gs", [2, 1])
def test_largest_restart_length(pkg, big_m_case, gs):
    A, b, normA = big_m_case
    with pkg.Solver(A, max_restart_m=M_MAX, A_norm2=normA) as s:
        g = s.arnoldi(b, M_MAX, gs=gs)
    o = oracle.arnoldi(A, b, M_MAX, oracle.IGS, gs)
    assert g["ncols"] == o["ncols"]
    k = g["ncols"]
    kap = P.kappa_prefix(A, b, o["V"], k)
    herr = P.h_column_errors(g["H"], o["H"], k)
    well = kap < 1e6
    assert well.sum() > 10
    bound = 1e-10 if gs == 2 else np.maximum(1e-10, 2 * P.EPS * kap)
    assert np.all(herr[well] <= (bound[well] if gs == 1 else bound)), herr[well].max()
    assert P.arnoldi_relation(A, g["V"], g["H"], k, normA) <= 1e-13
    if gs == 2:
        assert P.orth_loss(g["V"], k + 1) <= 1e-13


def test_largest_restart_length_one_reduce_and_fp32(pkg, big_m_case):
    """Alg. 4.2 and the FP32-basis form at m = 232: the same number of columns as the
    oracle's Alg. 4.2 cycle, the Arnoldi relation, and an FP32-IR solve to beta <= 1e-14."""
    A, b, normA = big_m_case
    with pkg.Solver(A, max_restart_m=M_MAX, A_norm2=normA, fp32_basis=True) as s:
        g = s.arnoldi(b, M_MAX, gs=2, method="one_reduce")
        r = s.solve(b, m=M_MAX, gs=2, tol=1e-14, max_restarts=30, precision="fp32_ir")
    o = oracle.arnoldi(A, b, M_MAX, oracle.ONE_REDUCE, 2)
    assert g["ncols"] == o["ncols"]
    assert P.arnoldi_relation(A, g["V"], g["H"], g["ncols"], normA) <= 1e-13
    assert r["status"] == 0 and r["beta"] <= 1e-14


def test_one_by_one_system(pkg):
    A = gen.csr_from_dense(np.array([[2.0]]))
    b = np.array([4.0])
    o = oracle.gmres(A, b, m=1, gs=2, tol=1e-15, max_cycles=2, normA=2.0)
    with pkg.Solver(A, max_restart_m=1, A_norm2=2.0) as s:
        g = s.solve(b, m=1, gs=2, tol=1e-15, max_restarts=2)
    assert g["status"] == o["status"]
    assert g["x"][0] == pytest.approx(2.0, rel=1e-15) and g["beta"] <= 1e-15


def test_empty_rows(pkg):
    """Rows with no stored entry (b zero there): the SpMV gives 0 for them and the solve
    matches the oracle's."""
    rng = np.random.default_rng(12)
    n = 300
    D = np.diag(rng.uniform(1.0, 3.0, n)) + np.diag(rng.uniform(-0.5, 0.5, n - 1), 1)
    empty = np.arange(7, n, 37)
    D[empty, :] = 0.0
    A = gen.csr_from_dense(D, drop_zeros=True)
    assert np.all(np.diff(A.rowptr)[empty] == 0)
    b = D @ np.ones(n)
    with pkg.Solver(A, max_restart_m=40, A_norm2=4.0) as s:
        y = s.spmv(np.ones(n))
        g = s.solve(b, m=40, gs=2, tol=1e-13, max_restarts=20)
    assert np.all(y[empty] == 0.0)
    o = oracle.gmres(A, b, m=40, gs=2, tol=1e-13, max_cycles=20, normA=4.0)
    assert g["status"] == o["status"] and abs(g["steps"] - o["steps"]) <= 2
    assert np.linalg.norm(g["x"] - o["x"]) <= 1e-8 * np.linalg.norm(o["x"])
