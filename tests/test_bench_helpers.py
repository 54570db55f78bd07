"""Host-side helpers of bench.py (no GPU): the served arrival stream (seeded, within the
stated ranges, at the stated rate), the norm bound the server and the one-at-a-time
comparison share, and the FMA model of the batched roofline against a direct count."""
import numpy as np
import scipy.sparse as sp

import bench
import gen


def test_serve_stream_is_seeded_and_in_range():
    a = bench.serve_stream(7, 2.0)
    assert a == bench.serve_stream(7, 2.0)
    t = np.array([x[0] for x in a])
    assert np.all(np.diff(t) > 0) and t[0] >= 0.0 and t[-1] < 2.0
    lam = bench.SERVE_LAMBDA
    assert abs(len(a) - 2.0 * lam) <= 5 * np.sqrt(2.0 * lam)      # Poisson count
    for _, side, pe, tol, prec, seed in a:
        assert bench.SERVE_SIDES[0] <= side <= bench.SERVE_SIDES[1]
        assert bench.SERVE_PE[0] <= pe <= bench.SERVE_PE[1]
        assert tol in bench.SERVE_TOLS and prec in ("fp64", "fp32_ir")
    assert 0.4 < np.mean([x[4] == "fp32_ir" for x in a]) < 0.6


def test_norm_bound():
    A, _, _, _ = gen.cd2d(9, 40.0)
    D = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n)).toarray()
    nb = bench.norm_bound(A)
    assert np.isclose(nb, np.sqrt(np.abs(D).sum(0).max() * np.abs(D).sum(1).max()), rtol=1e-15)
    assert nb >= np.linalg.norm(D, 2)


def test_batch_fma_model_one_cycle():
    """One cycle of m columns on one system: the model's count equals the operations of
    Alg. 4.1 tallied step by step (start residual, prime, loop columns k = 3..m+1, flush,
    x update, the residual of beta)."""
    n, nnz, m = 100, 480, 10
    total = bench.batch_fma([n], [nnz], [m], [1], m, 2)
    expect = nnz + 2 * n            # r = b - A x0, ||r||, ||x||
    expect += nnz + 2 * n           # prime: A v1 and its two-vector reduction
    expect += m * n                 # x = x0 + V_m y
    for p in range(2, m + 1):       # step k = p + 1 works on p basis columns
        expect += nnz + 5 * n * p   # SpMV, [V,w]^T[w,z] (2pn), two updates (2pn), V^T u (pn)
    expect += n                     # flush norm
    expect += nnz + 2 * n           # r = b - A x_m and the norms of beta at the cycle end
    assert abs(total - expect) <= 1e-9 * expect, (total, expect)
