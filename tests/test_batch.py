"""Batched IGS-GMRES (include/igs_batch.h) against the CPU oracle, system by system.

Tolerances (FP64 on both sides, different summation orders):
  * converged solves: the same status, both beta <= tol, step counts within +-2, and
    ||x_gpu - x_oracle|| <= 1e-8 ||x_oracle|| (both are within beta <= 1e-12 of the
    solution of a diagonally dominant system, kappa below 1e2);
  * one fixed cycle (tol = 0, one restart): the same number of steps and
    ||x_gpu - x_oracle|| <= 1e-10 ||x_oracle||: x = V y depends on every H entry of the cycle;
    beta within 1e-13 + the relative x difference in absolute terms (beta near 1e-12 sits at
    the rounding level of the residual it is computed from);
  * determinism: a system's x, beta, status, steps and cycles are bitwise equal alone and in
    a batch, and under every launch configuration.
"""
import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module")
def pkg():
    import paper_2205_07805_gb300 as pkg
    from paper_2205_07805_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def _systems(count, seed, nmin=64, nmax=2048):
    out = gen.banded_batch(count=count, nmin=nmin, nmax=nmax, seed=seed)
    As = [s[0] for s in out]
    b = np.concatenate([s[1] for s in out])
    norms = np.array([gen.norm2_power(A, iters=60) for A in As])
    return As, b, norms


def _split(v, As):
    off = np.cumsum([0] + [A.n for A in As])
    return [v[off[i]:off[i + 1]] for i in range(len(As))]


# ----------------------------------------------------------------------------------------
# Host logic (no GPU)
# ----------------------------------------------------------------------------------------
def test_block_csr_marshalling():
    import paper_2205_07805_gb300 as pkg
    As = [s[0] for s in gen.banded_batch(count=5, nmin=3, nmax=40, seed=9)]
    sys_ptr, rp, ci, va = pkg.block_csr(As)
    assert sys_ptr[0] == 0 and sys_ptr[-1] == sum(A.n for A in As)
    for s, A in enumerate(As):
        r0, r1 = sys_ptr[s], sys_ptr[s + 1]
        blk = gen.CSR(A.n, rp[r0:r1 + 1] - rp[r0], (ci[rp[r0]:rp[r1]] - r0).astype(np.int32),
                      va[rp[r0]:rp[r1]])
        assert np.array_equal(gen.csr_to_dense(blk), gen.csr_to_dense(A))


# ----------------------------------------------------------------------------------------
# GPU parity
# ----------------------------------------------------------------------------------------
@pytest.mark.gpu
@pytest.mark.parametrize("gs", [2, 1])
def test_batch_converged_solves_match_oracle(pkg, gs):
    As, b, norms = _systems(40, seed=1)
    with pkg.BatchSolver(As, m=50, A_norm2=norms, block_threads=256, blocks_per_sm=1) as bs:
        r = bs.solve(b, gs=gs, tol=1e-12, max_restarts=20)
    assert r["n_ok"] == len(As), r["status"]
    xs = _split(r["x"], As)
    worst = 0.0
    for i, A in enumerate(As):
        o = oracle.gmres(A, _split(b, As)[i], m=50, gs=gs, tol=1e-12, max_cycles=20, normA=norms[i])
        assert r["status"][i] == o["status"] == 0
        assert r["beta"][i] <= 1e-12 and o["beta"] <= 1e-12
        assert abs(int(r["steps"][i]) - o["steps"]) <= 2, (i, r["steps"][i], o["steps"])
        err = np.linalg.norm(xs[i] - o["x"]) / np.linalg.norm(o["x"])
        worst = max(worst, err)
        assert err <= 1e-8, (i, err)
    print(f"gs={gs}: worst relative x difference {worst:.2e}")


@pytest.mark.gpu
@pytest.mark.parametrize("gs", [2, 1])
def test_batch_one_cycle_matches_oracle(pkg, gs):
    # odd and even sizes, one slice and several (slices are 64-row multiples)
    As, b, norms = _systems(24, seed=2, nmin=65, nmax=1500)
    with pkg.BatchSolver(As, m=50, A_norm2=norms, block_threads=128, blocks_per_sm=2) as bs:
        r = bs.solve(b, gs=gs, tol=0.0, max_restarts=1)
    xs = _split(r["x"], As)
    worst = 0.0
    for i, A in enumerate(As):
        o = oracle.gmres(A, _split(b, As)[i], m=50, gs=gs, tol=0.0, max_cycles=1, normA=norms[i])
        assert r["status"][i] == o["status"]
        assert int(r["steps"][i]) == o["steps"] == 50
        assert r["cycles"][i] == o["cycles"] == 1
        err = np.linalg.norm(xs[i] - o["x"]) / np.linalg.norm(o["x"])
        worst = max(worst, err)
        assert err <= 1e-10, (i, err)
        # beta is normalised by ||b|| + ||A|| ||x||: the residual's own rounding gives an
        # absolute spread of a few (row nnz) eps, the x difference adds err
        assert abs(r["beta"][i] - o["beta"]) <= 1e-6 * o["beta"] + 1e-13 + err
    print(f"gs={gs}: one cycle, worst relative x difference {worst:.2e}")


@pytest.mark.gpu
def test_batch_bitwise_across_configurations_and_alone(pkg):
    As, b, norms = _systems(20, seed=3, nmin=64, nmax=1200)
    with pkg.BatchSolver(As, m=30, A_norm2=norms, block_threads=128, blocks_per_sm=1) as bs:
        ref = bs.solve(b, gs=2, tol=1e-12, max_restarts=5)
        for t, k in [(128, 3), (256, 1), (256, 2), (512, 1)]:
            bs.set_config(t, k)
            r = bs.solve(b, gs=2, tol=1e-12, max_restarts=5)
            for key in ("x", "beta", "status", "steps", "cycles"):
                assert np.array_equal(r[key], ref[key]), (t, k, key)
    bs_parts = _split(b, As)
    xs = _split(ref["x"], As)
    for i in (0, 7, 19):
        with pkg.BatchSolver([As[i]], m=30, A_norm2=norms[i:i + 1], block_threads=256,
                             blocks_per_sm=1) as one:
            r1 = one.solve(bs_parts[i], gs=2, tol=1e-12, max_restarts=5)
        assert np.array_equal(r1["x"], xs[i])
        assert r1["beta"][0] == ref["beta"][i] and r1["steps"][0] == ref["steps"][i]


@pytest.mark.gpu
def test_batch_edge_cases(pkg):
    rng = np.random.default_rng(4)
    tiny = [s[0] for s in gen.banded_batch(count=6, nmin=1, nmax=7, seed=5)]
    diag2 = gen.CSR(40, np.arange(41, dtype=np.int64), np.arange(40, dtype=np.int32),
                    np.where(np.arange(40) % 2 == 0, 2.0, 3.0))       # two eigenvalues: breakdown
    ban = [s[0] for s in gen.banded_batch(count=3, nmin=100, nmax=300, seed=6)]
    As = tiny + [diag2] + ban
    norms = np.array([gen.norm2_power(A, iters=60) for A in As])
    bparts = [rng.standard_normal(A.n) for A in As]
    bparts[-1][:] = 0.0                                                  # b = 0: x = 0
    b = np.concatenate(bparts)
    with pkg.BatchSolver(As, m=10, A_norm2=norms, block_threads=128, blocks_per_sm=1) as bs:
        r = bs.solve(b, gs=2, tol=1e-12, max_restarts=30)
        xs = _split(r["x"], As)
        for i, A in enumerate(As):
            o = oracle.gmres(A, bparts[i], m=10, gs=2, tol=1e-12, max_cycles=30, normA=norms[i])
            assert r["status"][i] == o["status"], (i, A.n, r["status"][i], o["status"])
            assert abs(int(r["steps"][i]) - o["steps"]) <= 2, (i, r["steps"][i], o["steps"])
            if o["status"] == 0:
                assert r["beta"][i] <= 1e-12
            den = max(np.linalg.norm(o["x"]), 1e-300)
            assert np.linalg.norm(xs[i] - o["x"]) <= 1e-8 * den
        assert np.all(xs[-1] == 0.0) and r["beta"][-1] == 0.0 and r["steps"][-1] == 0
        # too few restarts (one cycle of 10 steps): NOT_CONVERGED for the banded systems on
        # both sides, the same outcome for the rest (tol well above the rounding level)
        r2 = bs.solve(b, gs=2, tol=1e-12, max_restarts=1)
        for i, A in enumerate(As):
            o = oracle.gmres(A, bparts[i], m=10, gs=2, tol=1e-12, max_cycles=1, normA=norms[i])
            assert r2["status"][i] == o["status"], (i, r2["status"][i], o["status"])
            assert r2["steps"][i] == o["steps"]
        assert np.all(r2["status"][-3:-1] == pkg.NOT_CONVERGED)
        # a converged x as x0: no step
        r3 = bs.solve(b, x0=r["x"], gs=2, tol=1e-12, max_restarts=3)
        ok = r["status"] == 0
        assert np.all(r3["steps"][ok] == 0) and np.all(r3["status"][ok] == 0)
        # a NaN in one system's b: that system reports IGS_ENUMERIC, the others are unchanged
        bn = b.copy()
        bn[len(bparts[0])] = np.nan
        r4 = bs.solve(bn, gs=2, tol=1e-12, max_restarts=30)
        assert r4["status"][1] == pkg.ENUMERIC and r4["rc"] == pkg.ENUMERIC
        for key in ("beta", "status", "steps"):
            assert np.array_equal(np.delete(r4[key], 1), np.delete(r[key], 1))
    # m = 1
    with pkg.BatchSolver(ban, m=1, A_norm2=norms[-3:], block_threads=128, blocks_per_sm=1) as bs:
        rb = np.concatenate(bparts[-3:-1] + [rng.standard_normal(ban[-1].n)])
        r5 = bs.solve(rb, gs=2, tol=1e-10, max_restarts=400)
        parts = _split(rb, ban)
        for i, A in enumerate(ban):
            o = oracle.gmres(A, parts[i], m=1, gs=2, tol=1e-10, max_cycles=400, normA=norms[-3 + i])
            assert r5["status"][i] == o["status"]
            assert abs(int(r5["steps"][i]) - o["steps"]) <= 2


@pytest.mark.gpu
def test_batch_device_io_and_norm_estimate(pkg):
    torch = pytest.importorskip("torch")
    As, b, norms = _systems(12, seed=7, nmin=64, nmax=900)
    with pkg.BatchSolver(As, m=50, A_norm2=norms, block_threads=256, blocks_per_sm=1) as bs:
        rh = bs.solve(b, gs=2, tol=1e-12)
        bd = torch.from_numpy(b).cuda()
        rd = bs.solve(bd, gs=2, tol=1e-12)
        torch.cuda.synchronize()
        assert np.array_equal(rd["x"].cpu().numpy(), rh["x"])
        assert np.array_equal(rd["steps"].cpu().numpy(), rh["steps"])
    with pkg.BatchSolver(As, m=50, block_threads=256, blocks_per_sm=1) as bs:  # estimated norms
        est = bs.norms()
    exact = np.array([np.linalg.norm(gen.csr_to_dense(A), 2) for A in As])
    # power iteration approaches ||A||_2 from below
    assert np.all(est <= exact * (1 + 1e-12)) and np.all(est >= 0.99 * exact), est / exact


@pytest.mark.gpu
def test_batch_full_size_with_tuner(pkg):
    """4096 banded systems, n in [64, 2048], m = 50, beta <= 1e-12, tuned launch; a sample of
    systems (smallest, largest, spread between) checked against the oracle."""
    out = gen.banded_batch(count=4096, seed=0)
    As = [s[0] for s in out]
    b = np.concatenate([s[1] for s in out])
    with pkg.BatchSolver(As, m=50) as bs:
        info = bs.info
        assert info["n_tune"] >= 2
        r = bs.solve(b, gs=2, tol=1e-12, max_restarts=20)
        norms = bs.norms()
    assert r["n_ok"] == 4096 and np.all(r["beta"] <= 1e-12)
    ns = np.array([A.n for A in As])
    pick = sorted(set([int(np.argmin(ns)), int(np.argmax(ns))] + list(range(0, 4096, 512))))
    xs = _split(r["x"], As)
    for i in pick:
        o = oracle.gmres(As[i], out[i][1], m=50, gs=2, tol=1e-12, max_cycles=20, normA=norms[i])
        assert o["status"] == 0
        assert abs(int(r["steps"][i]) - o["steps"]) <= 2
        assert np.linalg.norm(xs[i] - o["x"]) <= 1e-8 * np.linalg.norm(o["x"])
