"""The seeded input recipes (no GPU): the sizes, structures and value rules the workloads are
stated with, checked against independent constructions, so that a generator change cannot
silently change what the parity tests and the benchmark run on."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen


def _dense(A):
    return sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n)).toarray()


@pytest.mark.parametrize("N,Pe", [(7, 50.0), (12, 1.0)])
def test_cd2d_stencil_by_definition(N, Pe):
    """5-point upwind convection-diffusion on the unit square, h = 1/(N+1), rows scaled by
    h^2, c = (1,1)/sqrt 2: diagonal 4 + Pe h sqrt 2, west/south -1 - Pe h / sqrt 2, east/north
    -1, Dirichlet nodes eliminated; nnz = 5 N^2 - 4 N; b = A 1 + 1e-3 N(0,1)."""
    A, b, x0, _ = gen.cd2d(N, Pe, seed=3)
    h, c = 1.0 / (N + 1), 1.0 / np.sqrt(2.0)
    D = np.zeros((N * N, N * N))
    for y in range(N):
        for x in range(N):
            i = y * N + x
            D[i, i] = 4.0 + Pe * h * c * 2
            if x > 0:
                D[i, i - 1] = -1.0 - Pe * h * c
            if y > 0:
                D[i, i - N] = -1.0 - Pe * h * c
            if x < N - 1:
                D[i, i + 1] = -1.0
            if y < N - 1:
                D[i, i + N] = -1.0
    assert A.n == N * N and A.rowptr[-1] == 5 * N * N - 4 * N
    assert np.array_equal(_dense(A), D)
    for i in range(A.n):   # column indices increase within each row
        assert np.all(np.diff(A.colind[A.rowptr[i]:A.rowptr[i + 1]]) > 0)
    assert np.all(x0 == 0.0)
    r = b - D @ np.ones(A.n)
    assert 0.0 < np.std(r) < 2e-3 and abs(np.mean(r)) < 1e-3


def test_cd3d_sizes_and_rows():
    N = 6
    A, _, _, _ = gen.cd3d(N, 20.0)
    assert A.n == N ** 3 and A.rowptr[-1] == 7 * N ** 3 - 6 * N ** 2
    D = _dense(A)
    h, c = 1.0 / (N + 1), 1.0 / np.sqrt(3.0)
    assert np.allclose(np.diag(D), 6.0 + 20.0 * h * c * 3, rtol=0, atol=1e-15)
    i = N * N + N + 1          # an interior node: all six neighbours
    assert D[i, i - 1] == D[i, i - N] == D[i, i - N * N] == -1.0 - 20.0 * h * c
    assert D[i, i + 1] == D[i, i + N] == D[i, i + N * N] == -1.0


def test_banded_batch_recipe():
    """7 diagonals clipped at the edges, diagonal = 1.1 x the row's off-diagonal absolute
    sum (strict dominance), n in [nmin, nmax], the same systems for the same seed."""
    sysA = gen.banded_batch(count=5, nmin=10, nmax=40, seed=4)
    again = gen.banded_batch(count=5, nmin=10, nmax=40, seed=4)
    for (A, b, x0, _), (A2, b2, _, _) in zip(sysA, again):
        assert 10 <= A.n <= 40
        assert np.array_equal(A.val, A2.val) and np.array_equal(b, b2)
        D = _dense(A)
        i, j = np.nonzero(D)
        assert np.all(np.abs(i - j) <= 3)
        off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
        assert np.allclose(np.diag(D), 1.1 * off, rtol=1e-15, atol=0)
        assert A.rowptr[-1] == sum(min(A.n, k + 4) - max(0, k - 3) for k in range(A.n))
        assert np.all(x0 == 0.0)


def test_dense_usv_spectrum():
    """Config 1: A = U diag(s) W^T with Haar U, W and s = logspace(0, -10, n)."""
    A, _, _, _ = gen.dense_usv(60, 0)
    s = np.linalg.svd(_dense(A), compute_uv=False)
    assert np.allclose(s, np.logspace(0, -10, 60), rtol=1e-6, atol=0)


def test_closed_form_examples():
    A, b, _, info = gen.simoncini(0)
    assert np.allclose(np.diag(_dense(A)), np.r_[1e-4, np.arange(2.0, 101.0)])
    assert abs(np.linalg.norm(b) - 1.0) < 1e-15 and info["normA"] == 100.0
    W, _, _, _ = gen.walker(10, 2000.0)
    Wd = _dense(W)
    assert Wd[0, 9] == 2000.0 and np.count_nonzero(Wd) == 11
    H, _, _, _ = gen.helmert(18)
    Hd = _dense(H)
    assert np.allclose(Hd @ Hd.T, np.eye(18), atol=1e-14)
