"""Precision form (igs_solve with precision = IGS_PREC_FP32_IR): FP32 SpMV and Krylov basis
inside FP64 iterative refinement, checked against the FP64 oracle (needs a GB300; -m gpu).

Stated errors (FP32 unit roundoff u32 = 6e-8; the FP64 parts as in the FP64 form):
  * converged solves: beta <= tol = 1e-14 like the oracle, and
    ||x - x_oracle|| <= 1e-10 ||x_oracle|| (both solutions are within beta 1e-14 of the
    exact one; kappa(A) is below 1e3 for these grids);
  * one FP32 cycle against the oracle's FP64 cycle: every Hessenberg column within
    1e-4 relative (measured about 1e-6: the basis and products carry u32, the Gram sums are
    FP64 over FP32 chunks of 32 rows), the same number of columns, and the cycle's x within
    1e-4 relative;
  * the FP32 Arnoldi relation of a cycle is not returned; its effect is what the x and H
    bounds above measure.
"""
import numpy as np
import pytest

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
    "cd3d_24": lambda: gen.cd3d(24, 20.0, seed=0),   # n = 13824, config-3 shape at small N
    "cd2d_63": lambda: gen.cd2d(63, 50.0, seed=1),   # n = 3969, ragged tail
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("gs", [2, 1])
def test_fp32_ir_reaches_fp64_accuracy(pkg, name, gs):
    A, b, _, _ = CASES[name]()
    nA = gen.norm2_power(A, iters=100)
    o = oracle.gmres(A, b, m=100, gs=gs, tol=1e-14, max_cycles=50, normA=nA)
    assert o["status"] == 0 and o["beta"] <= 1e-14
    with pkg.Solver(A, max_restart_m=100, A_norm2=nA, fp32_basis=True) as s:
        r = s.solve(b, m=100, gs=gs, tol=1e-14, max_restarts=50, precision="fp32_ir")
        r64 = s.solve(b, m=100, gs=gs, tol=1e-14, max_restarts=50)
    assert r["status"] == 0 and r["beta"] <= 1e-14, (r["status"], r["beta"], r["cycles"])
    err = np.linalg.norm(r["x"] - o["x"]) / np.linalg.norm(o["x"])
    err64 = np.linalg.norm(r64["x"] - o["x"]) / np.linalg.norm(o["x"])
    print(f"{name} gs={gs}: FP32-IR {r['steps']} steps / {r['cycles']} cycles, beta {r['beta']:.1e}, "
          f"x error {err:.1e}; FP64 {r64['steps']} steps, x error {err64:.1e}; oracle {o['steps']} steps")
    assert err <= 1e-10


@pytest.mark.parametrize("gs", [2, 1])
def test_fp32_cycle_against_fp64_oracle(pkg, gs):
    A, b, _, _ = gen.cd3d(24, 20.0, seed=0)
    nA = gen.norm2_power(A, iters=100)
    m = 40
    o = oracle.arnoldi(A, b, m, oracle.IGS, gs)
    oy = oracle.gmres(A, b, m=m, gs=gs, tol=0.0, max_cycles=1, normA=nA)
    with pkg.Solver(A, max_restart_m=m, A_norm2=nA, fp32_basis=True) as s:
        r = s.solve(b, m=m, gs=gs, tol=0.0, max_restarts=1, precision="fp32_ir", want_H=True)
    assert r["steps"] == o["ncols"] == m
    H, Ho = r["H"], o["H"]
    worst = 0.0
    for j in range(m):
        e = np.linalg.norm(H[: j + 2, j] - Ho[: j + 2, j]) / np.linalg.norm(Ho[: j + 2, j])
        worst = max(worst, e)
    ex = np.linalg.norm(r["x"] - oy["x"]) / np.linalg.norm(oy["x"])
    print(f"gs={gs}: FP32 cycle vs FP64 oracle: worst H column {worst:.2e}, x {ex:.2e}")
    assert worst <= 1e-4
    assert ex <= 1e-4


def test_fp32_ir_needs_fp32_context_and_valid_precision(pkg):
    A, b, _, _ = gen.cd2d(16, 10.0, seed=0)
    with pkg.Solver(A, max_restart_m=10, A_norm2=8.0) as s:
        with pytest.raises(pkg.IGSError):
            s.solve(b, m=10, precision="fp32_ir")
        with pytest.raises(ValueError):
            s.solve(b, m=10, precision="fp16")


def test_fp32_ir_inner_tolerance(pkg):
    """A looser inner tolerance stops each FP32 cycle earlier: more refinement steps, the
    same final accuracy."""
    A, b, _, _ = gen.cd2d(63, 50.0, seed=1)
    nA = gen.norm2_power(A, iters=100)
    with pkg.Solver(A, max_restart_m=100, A_norm2=nA, fp32_basis=True) as s:
        tight = s.solve(b, m=100, tol=1e-14, max_restarts=60, precision="fp32_ir", inner_tol=1e-6)
        loose = s.solve(b, m=100, tol=1e-14, max_restarts=60, precision="fp32_ir", inner_tol=1e-2)
    assert tight["status"] == 0 and loose["status"] == 0
    assert loose["cycles"] > tight["cycles"]
    assert np.linalg.norm(loose["x"] - tight["x"]) <= 1e-10 * np.linalg.norm(tight["x"])


def test_fp32_ir_full_size_backward_error(pkg):
    """The 3-D system the benchmark times (160^3, n = 4,096,000, 28.5 M non-zeros, m = 200,
    the launch configuration of bench.py): FP32-IR to beta <= 1e-14, with beta recomputed by
    the oracle (its own SpMV and norms) from the returned x at full size, and ||A||_2 from
    the context's own estimate passed to both."""
    A, b, _, _ = gen.cd3d(160, 20.0, seed=0)
    with pkg.Solver(A, max_restart_m=200, fp32_basis=True) as s:
        normA = s.info["A_norm2"]
        r = s.solve(b, m=200, gs=2, tol=1e-14, max_restarts=100, precision="fp32_ir")
    assert r["status"] == 0 and r["beta"] <= 1e-14, (r["status"], r["beta"])
    beta_o = oracle.backward_error(A, b, r["x"], normA)
    print(f"160^3 FP32-IR: {r['steps']} steps / {r['cycles']} refinement steps, beta {r['beta']:.2e}, "
          f"oracle beta {beta_o:.2e}")
    assert beta_o <= 1e-14 * (1 + 1e-6) + 1e-16
