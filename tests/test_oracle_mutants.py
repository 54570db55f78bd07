"""The pins are strong enough: each plausible mistake, planted in a copy of the oracle
source (compiled on the CPU into a temporary library), fails at least one pin.  The
unmodified source passes all of them.

Two edits are deliberately absent because they change no result beyond rounding:
flipping the sign of r^(3) in the Hessenberg column (step 17) and dropping the (I+L) solve
on r^(2) (step 15).  r^(3) is the second Gauss-Seidel correction; its size is the first
pass's loss of orthogonality times ||u_k||, which is O(eps) ||H_{:,k-1}|| (Sec. 3), and
with two iterations L itself is O(eps), so both edits move H by O(eps) only (measured:
the Arnoldi-relation residual goes from ~1e-16 to ~5e-16).  For the same reason three
edits of Alg. 4.2 are absent: the lagged norm without ||r^(2)||^2 (step 6), step 14 without
r^(3), and L transposed in step 5's solve; r^(2) = V^T u is the first projection's loss of
orthogonality, so each of these moves results by second-order terms only."""
import os

import pytest

import _pins
import oracle

# (name, original text, planted mistake) -- each original occurs exactly once.
MUTANTS = [
    ("drop step 9 (second division of the last r0 entry)",
     "r0c[p - 1] = r0c[p - 1] / gamma;", "r0c[p - 1] = r0c[p - 1];"),
    ("drop step 10 scaling of the L row",
     "L[(int64_t)(p - 1) * ldl + c] = lrow[c] / gamma;", "L[(int64_t)(p - 1) * ldl + c] = lrow[c];"),
    ("drop step 11 (v_k not divided by gamma)",
     "for (int64_t i = 0; i < n; ++i) z[i] = z[i] / gamma;", "for (int64_t i = 0; i < n; ++i) z[i] = z[i];"),
    ("step 16 subtracts V r^(1) again instead of V r^(3)",
     "project_out(n, p, V, r3, u, wk);", "project_out(n, p, V, r1, u, wk);"),
    ("transposed L in the triangular solve",
     "s -= L[(int64_t)i * ldl + c] * out[c];", "s -= L[(int64_t)c * ldl + i] * out[c];"),
    ("step 14 projects v_k instead of u_k",
     "for (int c = 0; c < p; ++c) r2[c] = ora_dot(n, V + (int64_t)c * n, u);",
     "for (int c = 0; c < p; ++c) r2[c] = ora_dot(n, V + (int64_t)c * n, z);"),
    ("step 5 omits w^T v_k from r^(0)",
     "for (int c = 0; c < p; ++c) r0c[c] = ora_dot(n, V + (int64_t)c * n, z);",
     "for (int c = 0; c < p - 1; ++c) r0c[c] = ora_dot(n, V + (int64_t)c * n, z); r0c[p - 1] = 0.0;"),
    ("subdiagonal set to gamma^2",
     "H[(int64_t)(k - 3) * ldh + (k - 2)] = gamma;", "H[(int64_t)(k - 3) * ldh + (k - 2)] = gamma * gamma;"),
    ("Givens rotation sign error",
     "h[i + 1] = -G->sn[i] * h[i] + G->cs[i] * h[i + 1];", "h[i + 1] = G->sn[i] * h[i] + G->cs[i] * h[i + 1];"),
    ("update adds instead of subtracting the projection",
     "out[i] = a[i] - s;", "out[i] = a[i] + s;"),
    ("SpMV reads the row index instead of the column index",
     "s += val[p] * x[colind[p]];", "s += val[p] * x[i];"),
    ("priming step skips the projection of w_2",
     "for (int64_t i = 0; i < n; ++i) w2[i] -= h11 * V[i];", ""),
    ("backward error omits ||A|| ||x||",
     "rn / (ora_nrm2(n, b) + normA * ora_nrm2(n, x));", "rn / ora_nrm2(n, b);"),
    # Alg. 4.2 (one-reduce)
    ("Alg. 4.2 drops Stephen's trick (step 12)", "r1[nb] = t - lr;", "r1[nb] = t;"),
    ("Alg. 4.2 step 8 divides u^T A u by gamma once", "t = t / gamma / gamma;", "t = t / gamma;"),
    ("Alg. 4.2 without the Jacobi re-orthogonalisation (step 10)",
     "project_out(n, nb, V, r2, u, vnew);", "for (int64_t i = 0; i < n; ++i) vnew[i] = u[i];"),
    ("Alg. 4.2 step 15 adds H r^(3) / gamma", "q[i] = r1[i] - hs;", "q[i] = r1[i] + hs;"),
    ("Alg. 4.2 step 13 without 1/gamma", "zs[i] = z[i] / gamma;", "zs[i] = z[i];"),
    ("Alg. 4.2 L row not scaled (step 9)",
     "L[(int64_t)nb * ldl + c] = r2[c] / gamma;", "L[(int64_t)nb * ldl + c] = r2[c];"),
    ("Alg. 4.2 r^(0) not scaled (step 7)", "s0[c] = s0[c] / gamma;", "s0[c] = s0[c];"),
    ("Alg. 4.2 step 15 with r^(2) and no 1/gamma",
     "hs += H[(int64_t)c * ldh + i] * (r3[c] / gamma);", "hs += H[(int64_t)c * ldh + i] * r2[c];"),
]


def _battery(impl):
    failed = []
    for pin in _pins.ALL_PINS:
        try:
            ok, detail = pin(impl=impl)
        except Exception as exc:  # a crash counts as detection
            ok, detail = False, repr(exc)
        if not ok:
            failed.append(f"{pin.__name__}: {detail}")
    return failed


@pytest.mark.parametrize("mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(mut, tmp_path):
    name, old, new = mut
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor not unique/missing: {old!r}"
    path = oracle.compile_variant(src.replace(old, new), os.path.join(str(tmp_path), "libmut.so"))
    failed = _battery(oracle.Oracle(path))
    assert failed, f"mutant '{name}' passed every pin"


def test_unmodified_passes_all(tmp_path):
    path = oracle.compile_variant(oracle.source_text(), os.path.join(str(tmp_path), "libclean.so"))
    assert _battery(oracle.Oracle(path)) == []
