"""The CPU oracle against what the paper and the mathematics fix (no GPU needed)."""
import numpy as np
import pytest

import _pins
import gen
import oracle


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    ok, detail = pin()
    assert ok, detail


def test_generators_match_paper_constants():
    """The closed-form examples reproduce the norms and condition numbers the paper
    prints (Sec. 5), and Walker's departure from normality is alpha exactly."""
    g = _pins.GOLDEN
    A, _, _, _ = gen.walker(10, g["walker"]["alpha"])
    D = gen.csr_to_dense(A)
    s = np.linalg.svd(D, compute_uv=False)
    assert abs(s[0] / g["walker"]["normA"] - 1) < 0.01
    assert abs((s[0] / s[-1]) / g["walker"]["cond"] - 1) < 0.01
    dep = np.sqrt(np.linalg.norm(D, "fro") ** 2 - np.sum(np.abs(np.linalg.eigvals(D)) ** 2))
    assert abs(dep - g["walker"]["dep"]) < 1e-6
    A, _, _, _ = gen.embree(100, g["embree"]["delta"])
    s = np.linalg.svd(gen.csr_to_dense(A), compute_uv=False)
    assert abs(s[0] - g["embree"]["normA"]) < 0.01 and abs(s[0] / s[-1] - g["embree"]["cond"]) < 0.05
    A, _, _, _ = gen.simoncini(0)
    s = np.linalg.svd(gen.csr_to_dense(A), compute_uv=False)
    assert s[0] == g["simoncini"]["normA"] and abs(s[0] / s[-1] - g["simoncini"]["cond"]) < 1e-6


def test_cd_generators_structure():
    """Stencil sizes: nnz = 5N^2 - 4N (2-D) and 7N^3 - 6N^2 (3-D); interior rows sum to 0."""
    for N in (3, 8, 17):
        A, b, _, _ = gen.cd2d(N, 50.0, seed=1)
        assert A.n == N * N and A.nnz == 5 * N * N - 4 * N
        assert np.all(np.diff(A.rowptr) >= 3)
        D = gen.csr_to_dense(A)
        interior = [x + N * y for y in range(1, N - 1) for x in range(1, N - 1)]
        assert np.abs(D[interior].sum(axis=1)).max() < 1e-12
        A3, _, _, _ = gen.cd3d(N, 20.0, seed=1)
        assert A3.n == N ** 3 and A3.nnz == 7 * N ** 3 - 6 * N ** 2
    A, _, _, _ = gen.cd2d(512, 50.0)
    assert A.n == 262144 and A.nnz == 1308672


def test_dense_usv_spectrum():
    A, b, x0, info = gen.dense_usv(50, 3, 1e-6)
    s = np.linalg.svd(gen.csr_to_dense(A), compute_uv=False)
    assert abs(s[0] - 1) < 1e-12 and abs(s[-1] / 1e-6 - 1) < 1e-6
    assert info["normA"] == 1.0 and np.all(x0 == 0)


def test_restart_resumes():
    """Restarted GMRES: a second cycle starts from x_m and lowers beta further."""
    A, b, _, _ = gen.cd2d(16, 10.0, seed=2)
    normA = gen.norm2_power(A)
    one = oracle.gmres(A, b, m=10, tol=0.0, max_cycles=1, normA=normA)
    two = oracle.gmres(A, b, m=10, tol=0.0, max_cycles=2, normA=normA)
    assert two["cycles"] == 2 and two["steps"] == 20 and two["beta"] < one["beta"]
    cont = oracle.gmres(A, b, x0=one["x"], m=10, tol=0.0, max_cycles=1, normA=normA)
    assert np.allclose(cont["x"], two["x"], rtol=0, atol=1e-13 * np.abs(two["x"]).max())


def test_in_cycle_stop_and_breakdown():
    """In-cycle stop: the estimate ends the cycle early and the true beta is met; an
    invariant subspace (diagonal matrix with 3 distinct eigenvalues) breaks down after 3
    columns with the exact solution."""
    A, b, _, _ = gen.cd2d(12, 5.0, seed=3)
    normA = gen.norm2_power(A)
    out = oracle.gmres(A, b, m=144, tol=1e-12, max_cycles=2, normA=normA)
    assert out["status"] == oracle.OK and out["beta"] <= 1e-12 and out["steps"] < 144
    D = np.diag([1.0, 2.0, 3.0, 1.0, 2.0, 3.0])
    Ad = gen.csr_from_dense(D, drop_zeros=True)
    bd = np.arange(1.0, 7.0)
    o = oracle.arnoldi(Ad, bd, 6, oracle.IGS, 2)
    assert o["status"] == oracle.BREAKDOWN and o["ncols"] == 3
    g = oracle.gmres(Ad, bd, m=6, tol=1e-15, max_cycles=1, normA=3.0)
    assert g["status"] == oracle.OK and g["steps"] == 3
    assert np.allclose(g["x"], bd / np.diag(D), rtol=1e-14)
