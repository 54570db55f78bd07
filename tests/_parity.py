"""Helpers shared by the GPU parity tests: metrics computed with numpy/scipy from the
factors either implementation returns."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

EPS = np.finfo(np.float64).eps


def sparse(A):
    return sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))


def kappa_prefix(A, r0, V, kmax):
    """kappa(B_k), B_k = [r0, A V_k], for k = 1..kmax, from one QR of B_kmax: the R factor
    of the leading k+1 columns is the leading block of R."""
    M = sparse(A)
    B = np.column_stack([r0, M @ V[:, :kmax]])
    R = np.linalg.qr(B, mode="r")
    out = []
    for k in range(1, kmax + 1):
        if k + 1 > A.n:  # more columns than rows: B_k is rank deficient
            out.append(np.inf)
            continue
        s = np.linalg.svd(R[:k + 1, :k + 1], compute_uv=False)
        out.append(s[0] / s[-1] if s[-1] > 0 else np.inf)
    return np.array(out)


def arnoldi_relation(A, V, H, k, normA):
    M = sparse(A)
    num = np.linalg.norm(M @ V[:, :k] - V[:, :k + 1] @ H[:k + 1, :k])
    return float(num / (normA * np.linalg.norm(V[:, :k])))


def orth_loss(V, k):
    Vk = V[:, :k]
    return float(np.linalg.norm(np.eye(k) - Vk.T @ Vk))


def h_column_errors(Hg, Ho, k):
    """||H_gpu(:,j) - H_oracle(:,j)|| / ||H_oracle(:,j)|| for j < k."""
    e = np.empty(k)
    for j in range(k):
        e[j] = np.linalg.norm(Hg[:j + 2, j] - Ho[:j + 2, j]) / np.linalg.norm(Ho[:j + 2, j])
    return e
