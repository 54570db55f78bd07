"""The oracle's OpenMP timing build gives bitwise the parity build's results (CPU only).

The benchmark times the oracle on all host cores with a build of the same source compiled
with -fopenmp.  Its parallel loops write disjoint outputs (rows, vector entries, one inner
product per basis column), each formed by the same serial operations in the same order, so
every result must be identical to the serial build's, bit for bit.
"""
import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module")
def omp():
    return oracle.openmp()


CASES = {
    "cd2d_40": gen.cd2d(40, 30.0, seed=4),
    "random_500": (gen.random_sparse(500, 9, seed=3, diag_shift=6.0), None, None, {}),
}


def _rhs(A, b):
    return b if b is not None else np.random.default_rng(17).standard_normal(A.n)


def test_openmp_build_uses_threads(omp):
    assert oracle.openmp_threads() >= 1
    assert int(oracle.Oracle(oracle.build()).lib.ora_threads()) == 1


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("method,gs", [(oracle.IGS, 1), (oracle.IGS, 2), (oracle.ONE_REDUCE, 2),
                                       (oracle.MGS, 1)])
def test_openmp_arnoldi_bitwise(omp, name, method, gs):
    A, b, _, _ = CASES[name]
    r0 = _rhs(A, b)
    a = oracle.arnoldi(A, r0, 30, method, gs)
    o = oracle.arnoldi(A, r0, 30, method, gs, impl=omp)
    assert a["ncols"] == o["ncols"] and a["status"] == o["status"]
    for key in ("V", "H", "L"):
        assert np.array_equal(a[key], o[key]), key


@pytest.mark.parametrize("name", sorted(CASES))
def test_openmp_gmres_bitwise(omp, name):
    A, b, _, _ = CASES[name]
    b = _rhs(A, b)
    normA = gen.norm2_power(A)
    a = oracle.gmres(A, b, m=20, gs=2, tol=1e-13, max_cycles=8, normA=normA)
    o = oracle.gmres(A, b, m=20, gs=2, tol=1e-13, max_cycles=8, normA=normA, impl=omp)
    assert a["steps"] == o["steps"] and a["status"] == o["status"]
    assert np.array_equal(a["x"], o["x"]) and a["beta"] == o["beta"]
    assert np.array_equal(a["hist_res"], o["hist_res"])
    y = oracle.spmv(A, b)
    assert np.array_equal(y, oracle.spmv(A, b, impl=omp))
