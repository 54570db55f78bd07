"""Seeded synthetic inputs for IGS-GMRES (arXiv 2205.07805).

This module builds matrices and right-hand sides only; it holds none of the solver's
arithmetic.  Both the CPU oracle (``oracle/``) and the CUDA library's tests and benchmark
draw their inputs from here, so the two sides see identical data.

Every generator is deterministic in its arguments (``numpy.random.default_rng(seed)``).
Matrices are returned as :class:`CSR` (int64 row pointers, int32 column indices, float64
values, column indices sorted within each row).

Workloads
---------
* :func:`dense_usv` -- dense ``A = U diag(s) W^T`` with Haar-orthogonal U, W and
  log-spaced singular values (non-normal, ill-conditioned; stands in for the paper's
  external ill-conditioned test matrices of Sec. 5).
* :func:`cd2d`, :func:`cd3d` -- upwind convection-diffusion on the unit square / cube
  (non-symmetric, non-normal sparse systems).
* :func:`simoncini`, :func:`walker`, :func:`embree`, :func:`helmert` -- the closed-form
  examples of Sec. 5 (Simoncini-Szyld diagonal, Walker's matrix eq. "walker", Embree's
  delta-bidiagonal, the Helmert matrix).
* :func:`banded_batch` -- many small non-symmetric banded systems of uneven size.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "csr_from_dense", "csr_to_dense", "dense_usv", "cd2d", "cd3d", "simoncini",
    "walker", "embree", "helmert", "banded_batch", "random_sparse", "norm2_power",
]


@dataclass(frozen=True)
class CSR:
    """Compressed sparse rows: ``n`` x ``n`` matrix, row ``i`` owns entries
    ``rowptr[i]:rowptr[i+1]`` of ``colind`` / ``val``."""

    n: int
    rowptr: np.ndarray  # int64, n+1
    colind: np.ndarray  # int32, nnz
    val: np.ndarray     # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_sums(self) -> np.ndarray:
        """Sum of each row's stored values (``A @ ones``), in storage order."""
        out = np.zeros(self.n)
        lens = np.diff(self.rowptr)
        nz = lens > 0
        out[nz] = np.add.reduceat(self.val, self.rowptr[:-1][nz])
        return out


def csr_from_dense(A: np.ndarray, drop_zeros: bool = False) -> CSR:
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    assert A.shape == (n, n)
    if drop_zeros:
        mask = A != 0.0
    else:
        mask = np.ones_like(A, dtype=bool)
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    rows, cols = np.nonzero(mask)
    return CSR(n, rowptr, cols.astype(np.int32), A[rows, cols].astype(np.float64))


def csr_to_dense(A: CSR) -> np.ndarray:
    D = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    np.add.at(D, (rows, A.colind), A.val)
    return D


def _haar(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian with the signs of R's diagonal
    moved into Q."""
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def dense_usv(n: int = 200, seed: int = 0, smin: float = 1e-10):
    """Dense ``A = U diag(s) W^T``; ``s`` log-spaced from 1 down to ``smin``.

    Returns ``(A, b, x0, info)`` with ``b ~ N(0, 1)``, ``x0 = 0`` and
    ``info = {"normA": 1.0, "cond": 1/smin}`` (exact by construction)."""
    rng = np.random.default_rng(seed)
    U = _haar(n, rng)
    W = _haar(n, rng)
    s = np.logspace(0.0, np.log10(smin), n)
    A = (U * s[None, :]) @ W.T
    b = rng.standard_normal(n)
    return csr_from_dense(A), b, np.zeros(n), {"normA": float(s[0]), "cond": float(s[0] / s[-1])}


def _cd_stencil(N: int, Pe: float, dim: int):
    """Upwind convection-diffusion  -lap u + Pe (c . grad u)  on the unit square (dim=2)
    or cube (dim=3), N interior points per side, h = 1/(N+1), Dirichlet nodes eliminated,
    rows scaled by h^2, velocity c = (1,..,1)/sqrt(dim).  First-order upwind differences:
    the upwind (lower-index) neighbour in direction d gets -1 - Pe h c_d, the downwind one
    -1, the diagonal 2 dim + Pe h sum(c).  Rows are ordered with x fastest."""
    h = 1.0 / (N + 1)
    c = 1.0 / np.sqrt(dim)
    n = N ** dim
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // (N ** d)) % N for d in range(dim)]
    diag = 2.0 * dim + Pe * h * c * dim
    up = -1.0 - Pe * h * c
    down = -1.0
    # Offsets sorted ascending so column indices in every row are increasing.
    entries = []  # (column offset, value, valid mask)
    for d in reversed(range(dim)):
        entries.append((-(N ** d), up, coords[d] > 0))
    entries.append((0, diag, np.ones(n, dtype=bool)))
    for d in range(dim):
        entries.append((N ** d, down, coords[d] < N - 1))
    valid = np.stack([e[2] for e in entries], axis=1)          # n x (2 dim + 1)
    cols = idx[:, None] + np.array([e[0] for e in entries])[None, :]
    vals = np.broadcast_to(np.array([e[1] for e in entries]), valid.shape)
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr, cols[valid].astype(np.int32), np.ascontiguousarray(vals[valid]))


def cd2d(N: int = 512, Pe: float = 50.0, seed: int = 0, noise: float = 1e-3):
    """2-D 5-point upwind convection-diffusion, n = N^2, nnz = 5 N^2 - 4 N.
    ``b = A 1 + noise * N(0,1)``, ``x0 = 0``.  Returns ``(A, b, x0, info)``."""
    A = _cd_stencil(N, Pe, 2)
    rng = np.random.default_rng(seed)
    b = A.row_sums() + noise * rng.standard_normal(A.n)
    return A, b, np.zeros(A.n), {"N": N, "Pe": Pe}


def cd3d(N: int = 160, Pe: float = 20.0, seed: int = 0, noise: float = 1e-3):
    """3-D 7-point upwind convection-diffusion, n = N^3, nnz = 7 N^3 - 6 N^2."""
    A = _cd_stencil(N, Pe, 3)
    rng = np.random.default_rng(seed)
    b = A.row_sums() + noise * rng.standard_normal(A.n)
    return A, b, np.zeros(A.n), {"N": N, "Pe": Pe}


def simoncini(seed: int = 0):
    """Simoncini-Szyld example (Sec. 5, "Ill-Conditioned Diagonal Matrix"):
    ``A = diag(1e-4, 2, 3, ..., 100)``, ``b = randn(100)`` scaled to unit norm."""
    d = np.arange(1.0, 101.0)
    d[0] = 1e-4
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(100)
    b = b / np.linalg.norm(b)
    return csr_from_dense(np.diag(d), drop_zeros=True), b, np.zeros(100), {"normA": 100.0}


def walker(n: int = 10, alpha: float = 2000.0):
    """Walker's matrix (eq. "walker"): ``diag(1, ..., n)`` with ``A[0, n-1] = alpha``,
    ``b = ones``."""
    A = np.diag(np.arange(1.0, n + 1.0))
    A[0, n - 1] = alpha
    return csr_from_dense(A, drop_zeros=True), np.ones(n), np.zeros(n), {}


def embree(n: int = 100, delta: float = 0.1):
    """Embree's delta-bidiagonal matrix (Sec. 5, "Highly Non-Normal Matrices"): unit
    diagonal, ``delta`` on the superdiagonal (completely defective); ``b = ones``."""
    A = np.eye(n) + delta * np.eye(n, k=1)
    return csr_from_dense(A, drop_zeros=True), np.ones(n), np.zeros(n), {}


def helmert(n: int = 18):
    """Textbook Helmert matrix (orthogonal): first row ``ones/sqrt(n)``; row ``i >= 1``
    has ``i`` entries ``1/sqrt(i(i+1))`` followed by ``-i/sqrt(i(i+1))``.  ``b = ones``."""
    A = np.zeros((n, n))
    A[0, :] = 1.0 / np.sqrt(n)
    for i in range(1, n):
        s = 1.0 / np.sqrt(i * (i + 1.0))
        A[i, :i] = s
        A[i, i] = -i * s
    return csr_from_dense(A, drop_zeros=True), np.ones(n), np.zeros(n), {"normA": 1.0}


def random_sparse(n: int, per_row: int, seed: int = 0, diag_shift: float = 0.0) -> CSR:
    """Random sparse matrix with up to ``per_row`` N(0,1) entries per row at random
    columns (duplicates merged), plus ``diag_shift`` on the diagonal.  Used for parity
    tests with irregular rows."""
    rng = np.random.default_rng(seed)
    rowptr = [0]
    cols_all, vals_all = [], []
    for i in range(n):
        k = int(rng.integers(0, per_row + 1))
        cols = np.unique(np.concatenate([rng.integers(0, n, size=k), [i]]))
        vals = rng.standard_normal(cols.size)
        vals[cols == i] += diag_shift
        cols_all.append(cols)
        vals_all.append(vals)
        rowptr.append(rowptr[-1] + cols.size)
    return CSR(n, np.asarray(rowptr, dtype=np.int64), np.concatenate(cols_all).astype(np.int32),
               np.concatenate(vals_all).astype(np.float64))


def banded_batch(count: int = 4096, nmin: int = 64, nmax: int = 2048, half_bw: int = 3,
                 dom: float = 1.1, seed: int = 0):
    """``count`` independent non-symmetric banded systems: n_i ~ U{nmin..nmax}, offsets
    ``-half_bw..half_bw`` (7 diagonals for half_bw = 3, clipped at the edges), off-diagonal
    entries N(0,1), diagonal set to ``dom`` times the row's off-diagonal absolute sum,
    ``b ~ N(0,1)``, ``x0 = 0``.  Returns a list of ``(A, b, x0, info)``."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        offs = np.arange(-half_bw, half_bw + 1)
        i = np.arange(n)[:, None]
        cols = i + offs[None, :]
        valid = (cols >= 0) & (cols < n)
        vals = rng.standard_normal(valid.shape)
        vals[:, half_bw] = 0.0
        vals = np.where(valid, vals, 0.0)
        vals[:, half_bw] = dom * np.abs(vals).sum(axis=1)
        counts = valid.sum(axis=1)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
        A = CSR(n, rowptr, cols[valid].astype(np.int32), np.ascontiguousarray(vals[valid]))
        out.append((A, rng.standard_normal(n), np.zeros(n), {}))
    return out


def norm2_power(A: CSR, iters: int = 100, seed: int = 0) -> float:
    """Estimate of ||A||_2 by power iteration on A^T A from a seeded start vector (the
    constant in the backward error; both implementations receive the same number)."""
    import scipy.sparse as sp

    M = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.n)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = M.T @ (M @ x)
        lam = float(np.linalg.norm(y))
        if lam == 0.0:
            return 0.0
        x = y / lam
    return float(np.sqrt(lam))
