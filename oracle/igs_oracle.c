/*
 * Reference oracle for IGS-GMRES (Thomas, Carson, Rozloznik, Carr, Swirydowicz,
 * "Iterated Gauss-Seidel GMRES", arXiv 2205.07805).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, serial FP64 restatement of
 * the paper's algorithms, used to check the CUDA library.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header or constant with the CUDA path.
 *
 * Conventions
 *  - IEEE binary64, round to nearest; built with -ffp-contract=off so that no
 *    multiply-add is fused (identical results on x86-64 and AArch64).
 *  - Every sum is taken left to right in index order; no blocking or reordering.
 *  - The parity build is serial (no -fopenmp: the "omp" pragmas are ignored).  A second
 *    build with -fopenmp exists only to time the oracle on all host cores; its pragmas
 *    sit on loops whose iterations write different outputs (matrix rows, vector entries,
 *    one inner product per basis column), and every output is still formed by the same
 *    serial operations in the same order, so both builds give bitwise the same results.
 *  - Matrices: A in CSR (int64 row pointers, int32 column indices).  V is n x (m+1)
 *    column-major (ld = n).  H is (m+1) x m column-major (ld = m+1).  L is
 *    (m+1) x (m+1) row-major; row i holds the strictly-lower row v_{i+1}^T V_i.
 *  - Paper indices are 1-based; C indices are 0-based.  Comments give both.
 *
 * Pins (see tests/test_oracle_pins.py): Arnoldi relation, orthogonality classes for one
 * and two Gauss-Seidel iterations, L = strict_lower(V^T V), H against the Krylov-matrix
 * QR, Givens least squares against LAPACK lstsq, k = n exactness, the paper's worked
 * examples (Simoncini-Szyld, Walker, Embree).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORA_MGS = 0, ORA_IGS = 1, ORA_ONE_REDUCE = 2 };
enum { ORA_OK = 0, ORA_NOT_CONVERGED = 1, ORA_BREAKDOWN = 2, ORA_EINVAL = -1, ORA_ENOMEM = -2,
       ORA_ENUMERIC = -4 };

/* Threads the loops below run on: 1 in the serial parity build. */
int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------
 * Basic kernels (plain loops).
 * ------------------------------------------------------------------------------------- */

/* y = A x (Sec. 1: the matrix-vector product of the Arnoldi process).  Each row is summed
 * in the order its entries are stored. */
void ora_spmv(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
              const double *x, double *y)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[colind[p]];
        y[i] = s;
    }
}

/* x^T y, summed left to right. */
double ora_dot(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* ||x||_2 = sqrt(x^T x). */
double ora_nrm2(int64_t n, const double *x) { return sqrt(ora_dot(n, x, x)); }

/* Forward substitution with the unit lower-triangular M = I + L_p (Alg. 4.1 steps 12 and
 * 15; Sec. 2, eq. "correct": T^(1) = (I + L)^{-1} = M^{-1}).  L is row-major with leading
 * dimension ldl; only rows 0..p-1 and their strictly-lower parts are read. */
static void unit_lower_solve(int p, const double *L, int ldl, const double *rhs, double *out)
{
    for (int i = 0; i < p; ++i) {
        double s = rhs[i];
        for (int c = 0; c < i; ++c) s -= L[(int64_t)i * ldl + c] * out[c];
        out[i] = s;
    }
}

/* out = a - V[:, 0:p] coef   (the Gram-Schmidt projection a - V r of Sec. 2).  The
 * product V coef is formed row by row, then subtracted. */
static void project_out(int64_t n, int p, const double *V, const double *coef, const double *a,
                        double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int c = 0; c < p; ++c) s += V[(int64_t)c * n + i] * coef[c];
        out[i] = a[i] - s;
    }
}

/* ---------------------------------------------------------------------------------------
 * Givens least squares for min || rho e1 - H y || (eq. "llse").  The paper does not name
 * a method; this is the textbook incremental Givens QR of the Hessenberg matrix.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int m;
    double *R;  /* (m+1) x m col-major copy of H, rotated in place */
    double *cs, *sn;
    double *g;  /* rotated right-hand side, length m+1 */
} givens_ls;

static int givens_init(givens_ls *G, int m, double rho)
{
    G->m = m;
    G->R = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
    G->cs = (double *)calloc((size_t)m, sizeof(double));
    G->sn = (double *)calloc((size_t)m, sizeof(double));
    G->g = (double *)calloc((size_t)m + 1, sizeof(double));
    if (!G->R || !G->cs || !G->sn || !G->g) return ORA_ENOMEM;
    G->g[0] = rho;
    return ORA_OK;
}

static void givens_free(givens_ls *G)
{
    free(G->R); free(G->cs); free(G->sn); free(G->g);
}

/* Bring column j (entries 0..j+1 of H[:, j]) into the factorization; returns |g_{j+1}|,
 * the Arnoldi residual norm || rho e1 - H_{j+2,j+1} y ||. */
static double givens_add_column(givens_ls *G, const double *H, int j)
{
    const int ld = G->m + 1;
    double *h = G->R + (int64_t)j * ld;
    for (int i = 0; i <= j + 1; ++i) h[i] = H[(int64_t)j * ld + i];
    for (int i = 0; i < j; ++i) {
        double t = G->cs[i] * h[i] + G->sn[i] * h[i + 1];
        h[i + 1] = -G->sn[i] * h[i] + G->cs[i] * h[i + 1];
        h[i] = t;
    }
    double r = hypot(h[j], h[j + 1]);
    double c = 1.0, s = 0.0;
    if (r != 0.0) { c = h[j] / r; s = h[j + 1] / r; }
    G->cs[j] = c; G->sn[j] = s;
    h[j] = r; h[j + 1] = 0.0;
    G->g[j + 1] = -s * G->g[j];
    G->g[j] = c * G->g[j];
    return fabs(G->g[j + 1]);
}

/* Back substitution R y = g for the first p columns. */
static void givens_solve(const givens_ls *G, int p, double *y)
{
    const int ld = G->m + 1;
    for (int i = p - 1; i >= 0; --i) {
        double s = G->g[i];
        for (int c = i + 1; c < p; ++c) s -= G->R[(int64_t)c * ld + i] * y[c];
        y[i] = s / G->R[(int64_t)i * ld + i];
    }
}

/* ---------------------------------------------------------------------------------------
 * One Arnoldi cycle.
 * ------------------------------------------------------------------------------------- */

/* Cycle control: optional in-cycle stop when the estimated backward error
 *   res_j / (||b|| + ||A||_2 ||x0||)  <=  tol
 * (the paper states no in-cycle rule; this denominator never exceeds the true one when
 * x0 = 0).  hist_* receive one entry per completed column. */
typedef struct {
    double stop_den;   /* ||b|| + ||A||_2 ||x0||; <= 0 disables the in-cycle stop */
    double tol;
    double *hist_res;  /* |g_{j+1}| per completed column (nullable) */
    double *hist_lfro; /* ||L_{j+1}||_F per completed column (nullable) */
    int64_t hist_room;
    double res_last;
} cycle_ctl;

static void record(cycle_ctl *ctl, int j, double res, double lfro)
{
    if (!ctl) return;
    if (j < ctl->hist_room) {
        if (ctl->hist_res) ctl->hist_res[j] = res;
        if (ctl->hist_lfro) ctl->hist_lfro[j] = lfro;
    }
    ctl->res_last = res;
}

static int converged(const cycle_ctl *ctl, double res)
{
    return ctl && ctl->stop_den > 0.0 && res / ctl->stop_den <= ctl->tol;
}

/* Breakdown (invariant Krylov subspace; the paper leaves it unspecified): the new
 * subdiagonal entry is at the rounding level of the column it completes,
 *   gamma <= 64 eps ||H_{1:j,j}||_2   (or gamma = 0). */
#define ORA_BREAKDOWN_FACTOR (64.0 * 2.220446049250313e-16)
static int is_breakdown(const double *H, int ldh, int j, double gamma)
{
    double s = 0.0;
    for (int i = 0; i <= j; ++i) s += H[(int64_t)j * ldh + i] * H[(int64_t)j * ldh + i];
    return gamma == 0.0 || gamma <= ORA_BREAKDOWN_FACTOR * sqrt(s);
}

/* ||L_p||_F over rows 0..p-1. */
static double lower_fro(const double *L, int ldl, int p)
{
    double s = 0.0;
    for (int i = 0; i < p; ++i)
        for (int c = 0; c < i; ++c) s += L[(int64_t)i * ldl + c] * L[(int64_t)i * ldl + c];
    return sqrt(s);
}

/* MGS-GMRES Arnoldi (Saad and Schultz; Sec. 1): for j = 1..m, w = A v_j, then one inner
 * product and one update per previous basis vector, h_{j+1,j} = ||w||, v_{j+1} = w / h.
 * Returns the number of completed columns; *status = ORA_BREAKDOWN per is_breakdown. */
static int mgs_cycle(int64_t n, const int64_t *rp, const int32_t *ci, const double *va,
                     const double *r0, int m, double *V, double *H, double rho,
                     givens_ls *G, cycle_ctl *ctl, int *status)
{
    const int ldh = m + 1;
    double *w = (double *)malloc((size_t)n * sizeof(double));
    if (!w) { *status = ORA_ENOMEM; return 0; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) V[i] = r0[i] / rho;
    int done = 0;
    for (int j = 0; j < m; ++j) {
        ora_spmv(n, rp, ci, va, V + (int64_t)j * n, w);
        for (int i = 0; i <= j; ++i) {
            const double *vi = V + (int64_t)i * n;
            double h = ora_dot(n, vi, w);
            H[(int64_t)j * ldh + i] = h;
            #pragma omp parallel for schedule(static)
            for (int64_t r = 0; r < n; ++r) w[r] -= h * vi[r];
        }
        double h = ora_nrm2(n, w);
        H[(int64_t)j * ldh + j + 1] = h;
        if (!isfinite(h)) { *status = ORA_ENUMERIC; break; }
        double res = givens_add_column(G, H, j);
        record(ctl, j, res, NAN);
        done = j + 1;
        if (is_breakdown(H, ldh, j, h)) { *status = ORA_BREAKDOWN; break; }
        #pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < n; ++r) V[(int64_t)(j + 1) * n + r] = w[r] / h;
        if (converged(ctl, res)) break;
    }
    free(w);
    return done;
}

/* IGS-GMRES Arnoldi, Alg. 4.1 ("Low-Synchronization Two-Reduce Iterated Gauss-Seidel
 * GMRES"), with gs = 1 (steps 14-16 skipped, r^(3) = 0, w_k = u_k: the inverse compact WY
 * MGS of Sec. 1-2) or gs = 2.
 *
 * Readings where the paper leaves a choice:
 *  - The loop runs k = 3..m+1 and a final "flush" sets H_{m+1,m} = ||w_{m+1}|| and the last
 *    row of L, so that a cycle yields m full Hessenberg columns from m products with A.
 *  - Step 2 projects once, as printed, for both gs = 1 and gs = 2.
 *  - Steps 8 and 9 both divide the last entry of r^(0): that entry is w^T A w and carries
 *    gamma twice.
 *  - H_{k-1,k-2} = gamma_{k-1} is set at step 6 of iteration k (the subdiagonal of the
 *    column completed one iteration earlier); the Givens rotation for that column is
 *    applied right there, so the in-cycle stop test can end the cycle before step 12.
 *  - gamma_{k-1} at the rounding level of its column (is_breakdown) is a breakdown
 *    (invariant Krylov subspace): the cycle ends with the completed columns.
 */
static int igs_cycle(int64_t n, const int64_t *rp, const int32_t *ci, const double *va,
                     const double *r0, int m, int gs, double *V, double *H, double *L,
                     double rho, givens_ls *G, cycle_ctl *ctl, int *status)
{
    const int ldh = m + 1, ldl = m + 1;
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *u = (double *)malloc((size_t)n * sizeof(double));
    double *r0c = (double *)calloc((size_t)m + 1, sizeof(double));
    double *r1 = (double *)calloc((size_t)m + 1, sizeof(double));
    double *r2 = (double *)calloc((size_t)m + 1, sizeof(double));
    double *r3 = (double *)calloc((size_t)m + 1, sizeof(double));
    double *lrow = (double *)calloc((size_t)m + 1, sizeof(double));
    int done = 0, stopped = 0;
    if (!z || !u || !r0c || !r1 || !r2 || !r3 || !lrow) { *status = ORA_ENOMEM; goto out; }

    /* Step 1: v_1 = r_0 / rho (rho = ||r_0|| is computed by the caller). */
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) V[i] = r0[i] / rho;

    /* Step 2: w_2 = A v_1, H_{1,1} = v_1^T w_2, w_2 = w_2 - H_{1,1} v_1, V_2 = [v_1, w_2]. */
    {
        double *w2 = V + n;
        ora_spmv(n, rp, ci, va, V, w2);
        double h11 = ora_dot(n, V, w2);
        H[0] = h11;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) w2[i] -= h11 * V[i];
    }

    for (int k = 3; k <= m + 1; ++k) {
        const int p = k - 1;              /* columns of V_{k-1}; w_{k-1} is V[:, p-1] */
        double *w = V + (int64_t)(p - 1) * n;

        /* Step 4: v_k = A w_{k-1}  (held in z; w_{k-1} is not yet normalized). */
        ora_spmv(n, rp, ci, va, w, z);

        /* Step 5, the one global reduction: L^T_{1:k-2,k-1} = V_{k-2}^T w_{k-1} and
         * r^(0)_{1:k-1,k} = V_{k-1}^T v_k, with ||w_{k-1}||^2 folded in (step 6). */
        #pragma omp parallel for schedule(static)
        for (int c = 0; c < p - 1; ++c) lrow[c] = ora_dot(n, V + (int64_t)c * n, w);
        #pragma omp parallel for schedule(static)
        for (int c = 0; c < p; ++c) r0c[c] = ora_dot(n, V + (int64_t)c * n, z);
        double ww = ora_dot(n, w, w);

        /* Step 6: gamma_{k-1} = ||w_{k-1}||, the subdiagonal H_{k-1,k-2}. */
        double gamma = sqrt(ww);
        H[(int64_t)(k - 3) * ldh + (k - 2)] = gamma;
        if (!isfinite(gamma)) { *status = ORA_ENUMERIC; break; }
        {   /* column k-2 (1-based) is now complete: Givens + history + stop test */
            double res = givens_add_column(G, H, k - 3);
            record(ctl, k - 3, res, lower_fro(L, ldl, k - 2));
            done = k - 2;
            if (is_breakdown(H, ldh, k - 3, gamma)) { *status = ORA_BREAKDOWN; break; }
            if (converged(ctl, res)) { stopped = 1; break; }
        }

        /* Step 7: v_{k-1} = w_{k-1} / gamma_{k-1} (lagged normalization, in place). */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) w[i] = w[i] / gamma;
        /* Step 8: r^(0)_{1:k-1,k} /= gamma;  Step 9: r^(0)_{k-1,k} /= gamma once more. */
        for (int c = 0; c < p; ++c) r0c[c] = r0c[c] / gamma;
        r0c[p - 1] = r0c[p - 1] / gamma;
        /* Step 10: L_{k-1,1:k-2} = L_{k-1,1:k-2} / gamma (new row p-1 of L). */
        for (int c = 0; c < p - 1; ++c) L[(int64_t)(p - 1) * ldl + c] = lrow[c] / gamma;
        /* Step 11: v_k = v_k / gamma. */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) z[i] = z[i] / gamma;

        /* Step 12: r^(1) = (I + L_{k-1})^{-1} r^(0).  Step 13: u_k = v_k - V_{k-1} r^(1). */
        unit_lower_solve(p, L, ldl, r0c, r1);
        project_out(n, p, V, r1, z, u);

        double *wk = V + (int64_t)p * n;
        if (gs == 2) {
            /* Step 14: r^(2) = V_{k-1}^T u_k (second reduction). */
            #pragma omp parallel for schedule(static)
            for (int c = 0; c < p; ++c) r2[c] = ora_dot(n, V + (int64_t)c * n, u);
            /* Step 15: r^(3) = (I + L_{k-1})^{-1} r^(2).  Step 16: w_k = u_k - V_{k-1} r^(3). */
            unit_lower_solve(p, L, ldl, r2, r3);
            project_out(n, p, V, r3, u, wk);
        } else {
            for (int c = 0; c < p; ++c) r3[c] = 0.0;
            memcpy(wk, u, (size_t)n * sizeof(double));
        }
        /* Step 17: H_{1:k-1,k-1} = r^(1) + r^(3).  Step 18: V_k = [V_{k-1}, w_k]. */
        for (int c = 0; c < p; ++c) H[(int64_t)(k - 2) * ldh + c] = r1[c] + r3[c];
    }

    /* Flush (end of cycle, all m columns built): gamma_{m+1} = ||w_{m+1}||,
     * H_{m+1,m} = gamma_{m+1}, v_{m+1} = w_{m+1} / gamma_{m+1}, last row of L. */
    if (*status == ORA_OK && !stopped && done == m - 1) {
        double *w = V + (int64_t)m * n;
        #pragma omp parallel for schedule(static)
        for (int c = 0; c < m; ++c) lrow[c] = ora_dot(n, V + (int64_t)c * n, w);
        double gamma = sqrt(ora_dot(n, w, w));
        H[(int64_t)(m - 1) * ldh + m] = gamma;
        if (!isfinite(gamma)) { *status = ORA_ENUMERIC; goto out; }
        double res = givens_add_column(G, H, m - 1);
        record(ctl, m - 1, res, lower_fro(L, ldl, m));
        done = m;
        if (is_breakdown(H, ldh, m - 1, gamma)) { *status = ORA_BREAKDOWN; goto out; }
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) w[i] = w[i] / gamma;
        for (int c = 0; c < m; ++c) L[(int64_t)m * ldl + c] = lrow[c] / gamma;
    }
out:
    free(z); free(u); free(r0c); free(r1); free(r2); free(r3); free(lrow);
    return done;
}

/* Alg. 4.2 ("Low-Synch One-Reduce hybrid MGS-CGS GMRES"), one cycle, one global reduction
 * per column.  The vector entering iteration k is u_{k-1}, the output of the previous
 * iteration's single projection (step 13), not yet re-orthogonalised; the reduction of step 4
 * gives r^(2) = V_{k-2}^T u_{k-1}, ||u_{k-1}||^2, r^(0) = V_{k-2}^T A u_{k-1} and
 * u_{k-1}^T A u_{k-1}.
 *
 * Readings where the printed algorithm is garbled or silent:
 *  - Step 2: u_2 = w_2 - v_1 H_{1,1} (the printed division by H_{1,1} is taken as a typo).
 *  - Hessenberg columns are completed one iteration late: column k-2 (1-based) gets
 *    H_{1:k-2,k-2} = q + r^(3) (step 14) and H_{k-1,k-2} = gamma_{k-1}, where q is the
 *    first-projection coefficient vector of the previous iteration (step 15).
 *  - Step 15 is q = r^(1) - H_{1:k-1,1:k-2} r^(3) / gamma_{k-1}: the derivation (eq. "Aw":
 *    A w_{k-1} = A u_{k-1} - V_{k-1} H r^(2), and step 13 subtracting V r^(1)) fixes r^(1)
 *    and the 1/gamma that the printed step 15 (r^(0), r^(3)) leaves out; r^(3) replaces r^(2)
 *    there as it does in step 14.
 *  - Step 10 uses r^(2) (Jacobi) and step 14 uses r^(3) = (I + L)^{-1} r^(2), as printed.
 *  - L's new row (step 9) is r^(2) / gamma = u_{k-1}^T V_{k-2} / gamma, as printed (not
 *    v^T V as in Alg. 4.1).
 *  - gamma (step 6, the lagged norm) = sqrt(||u||^2 - ||r^(2)||^2); a non-positive argument
 *    is a breakdown (gamma = 0).
 *  - The cycle builds m columns from m products with A (step 2 and k = 3..m+1) and a flush
 *    re-orthogonalises u_{m+1} (one more reduction, no product) to set column m.
 */
static int one_reduce_cycle(int64_t n, const int64_t *rp, const int32_t *ci, const double *va,
                            const double *r0, int m, double *V, double *H, double *L, double rho,
                            givens_ls *G, cycle_ctl *ctl, int *status)
{
    const int ldh = m + 1, ldl = m + 1;
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *u = (double *)malloc((size_t)n * sizeof(double));
    double *zs = (double *)malloc((size_t)n * sizeof(double));
    double *r1 = (double *)calloc((size_t)m + 2, sizeof(double));
    double *r2 = (double *)calloc((size_t)m + 2, sizeof(double));
    double *r3 = (double *)calloc((size_t)m + 2, sizeof(double));
    double *s0 = (double *)calloc((size_t)m + 2, sizeof(double));
    double *q = (double *)calloc((size_t)m + 2, sizeof(double));
    int done = 0, stopped = 0;
    if (!z || !u || !zs || !r1 || !r2 || !r3 || !s0 || !q) { *status = ORA_ENOMEM; goto out; }

    /* Step 1: v_1 = r_0 / rho. */
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) V[i] = r0[i] / rho;
    /* Step 2: w_2 = A v_1, H_11 = v_1^T w_2, u_2 = w_2 - v_1 H_11; H_11 is the first entry of
     * column 1's first-projection coefficients q. */
    {
        ora_spmv(n, rp, ci, va, V, z);
        const double h11 = ora_dot(n, V, z);
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) u[i] = z[i] - V[i] * h11;
        q[0] = h11;
    }
    for (int k = 3; k <= m + 2; ++k) {
        const int nb = k - 2;            /* normalised columns v_1..v_{k-2} */
        const int flush = k == m + 2;    /* last: re-orthogonalise u_{m+1} only */
        /* Step 4, the one global reduction. */
        if (!flush) ora_spmv(n, rp, ci, va, u, z);
        #pragma omp parallel for schedule(static)
        for (int c = 0; c < nb; ++c) r2[c] = ora_dot(n, V + (int64_t)c * n, u);
        const double uu = ora_dot(n, u, u);
        double t = 0.0;
        if (!flush) {
            #pragma omp parallel for schedule(static)
            for (int c = 0; c < nb; ++c) s0[c] = ora_dot(n, V + (int64_t)c * n, z);
            t = ora_dot(n, u, z);
        }
        /* Step 5: r^(3) = (I + L_{k-2})^{-1} r^(2) (normal equations). */
        unit_lower_solve(nb, L, ldl, r2, r3);
        /* Step 6: the lagged norm. */
        double rr = 0.0;
        for (int c = 0; c < nb; ++c) rr += r2[c] * r2[c];
        const double g2 = uu - rr;
        const double gamma = g2 > 0.0 ? sqrt(g2) : (g2 == g2 ? 0.0 : g2);
        /* Step 14: column k-2 (1-based) complete. */
        for (int c = 0; c < nb; ++c) H[(int64_t)(nb - 1) * ldh + c] = q[c] + r3[c];
        H[(int64_t)(nb - 1) * ldh + nb] = gamma;
        if (!isfinite(gamma)) { *status = ORA_ENUMERIC; break; }
        {
            double res = givens_add_column(G, H, nb - 1);
            record(ctl, nb - 1, res, lower_fro(L, ldl, nb));
            done = nb;
            if (is_breakdown(H, ldh, nb - 1, gamma)) { *status = ORA_BREAKDOWN; break; }
            if (converged(ctl, res)) { stopped = 1; break; }
        }
        /* Steps 9-11 (also at the flush, so that a cycle returns m+1 basis vectors and
         * m+1 rows of L): L row = r^(2) / gamma, v_{k-1} = (u_{k-1} - V_{k-2} r^(2)) / gamma. */
        for (int c = 0; c < nb; ++c) L[(int64_t)nb * ldl + c] = r2[c] / gamma;
        {
            double *vnew = V + (int64_t)nb * n;
            project_out(n, nb, V, r2, u, vnew);
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) vnew[i] = vnew[i] / gamma;
        }
        if (flush) break;
        /* Steps 7-8: r^(0) / gamma, its last entry once more. */
        for (int c = 0; c < nb; ++c) s0[c] = s0[c] / gamma;
        t = t / gamma / gamma;
        /* (Steps 10-11, w_{k-1} = u_{k-1} - V_{k-2} r^(2) (Jacobi) and v_{k-1} = w_{k-1} / gamma,
         * are above.)  Step 12: r^(1) = [I 0; -L_{k-1,1:k-2} 1] r^(0) (the last entry by
         * "Stephen's trick"). */
        for (int c = 0; c < nb; ++c) r1[c] = s0[c];
        {
            double lr = 0.0;
            for (int c = 0; c < nb; ++c) lr += L[(int64_t)nb * ldl + c] * s0[c];
            r1[nb] = t - lr;
        }
        /* Step 13: u_k = A u_{k-1} / gamma - V_{k-1} r^(1). */
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) zs[i] = z[i] / gamma;
        project_out(n, nb + 1, V, r1, zs, u);
        /* Step 15: first-projection coefficients of column k-1: q = r^(1) - H r^(3) / gamma. */
        for (int i = 0; i <= nb; ++i) {
            double hs = 0.0;
            for (int c = 0; c < nb; ++c) hs += H[(int64_t)c * ldh + i] * (r3[c] / gamma);
            q[i] = r1[i] - hs;
        }
    }
    (void)stopped;
out:
    free(z); free(u); free(zs); free(r1); free(r2); free(r3); free(s0); free(q);
    return done;
}

/* Public: one Arnoldi cycle on r0 (no in-cycle stop).  V, H, L as described at the top
 * (caller-allocated, zero-filled by this routine).  Returns the number of completed
 * columns; *rho_out = ||r0||; *status_out per the ORA_* codes. */
int ora_arnoldi(int64_t n, const int64_t *rp, const int32_t *ci, const double *va,
                const double *r0, int m, int method, int gs, double *V, double *H, double *L,
                double *rho_out, int *status_out)
{
    int status = ORA_OK;
    if (n <= 0 || m < 1 || (method != ORA_MGS && method != ORA_IGS && method != ORA_ONE_REDUCE) || gs < 1 ||
        gs > 2) {
        *status_out = ORA_EINVAL;
        return 0;
    }
    memset(V, 0, (size_t)n * (m + 1) * sizeof(double));
    memset(H, 0, (size_t)(m + 1) * m * sizeof(double));
    memset(L, 0, (size_t)(m + 1) * (m + 1) * sizeof(double));
    double rho = ora_nrm2(n, r0);
    *rho_out = rho;
    if (rho == 0.0 || !isfinite(rho)) {
        *status_out = rho == 0.0 ? ORA_BREAKDOWN : ORA_ENUMERIC;
        return 0;
    }
    givens_ls G;
    if (givens_init(&G, m, rho) != ORA_OK) { givens_free(&G); *status_out = ORA_ENOMEM; return 0; }
    int done = method == ORA_MGS
                   ? mgs_cycle(n, rp, ci, va, r0, m, V, H, rho, &G, NULL, &status)
                   : method == ORA_IGS
                         ? igs_cycle(n, rp, ci, va, r0, m, gs, V, H, L, rho, &G, NULL, &status)
                         : one_reduce_cycle(n, rp, ci, va, r0, m, V, H, L, rho, &G, NULL, &status);
    givens_free(&G);
    *status_out = status;
    return done;
}

/* Least squares y = argmin || rho e1 - H_{p+1,p} y || by Givens (eq. "llse"); returns the
 * residual norm.  H is (m+1) x m col-major; only its first p columns are read. */
double ora_hessenberg_lsq(int m, int p, const double *H, double rho, double *y)
{
    givens_ls G;
    if (givens_init(&G, m, rho) != ORA_OK) { givens_free(&G); return NAN; }
    double res = rho;
    for (int j = 0; j < p; ++j) res = givens_add_column(&G, H, j);
    givens_solve(&G, p, y);
    givens_free(&G);
    return res;
}

/* Backward error beta(x) = ||b - A x|| / (||b|| + ||A||_2 ||x||)  (eq. "nrbe"). */
double ora_backward_error(int64_t n, const int64_t *rp, const int32_t *ci, const double *va,
                          const double *b, const double *x, double normA)
{
    double *r = (double *)malloc((size_t)n * sizeof(double));
    if (!r) return NAN;
    ora_spmv(n, rp, ci, va, x, r);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    /* A zero residual is an exact solution: beta = 0 (also for b = 0, x = 0). */
    double rn = ora_nrm2(n, r);
    double beta = rn == 0.0 ? 0.0 : rn / (ora_nrm2(n, b) + normA * ora_nrm2(n, x));
    free(r);
    return beta;
}

/* Restarted GMRES(m): cycles of the chosen Arnoldi method, x_m = x_0 + V_m y_m at the end
 * of each cycle (the last line of Alg. 4.1), true backward error after each cycle, restart
 * from x_m until beta <= tol or max_cycles cycles ran.  hist_res/hist_lfro (nullable, room
 * hist_cap) get one entry per completed column over all cycles.  Returns an ORA_* code. */
int ora_gmres(int64_t n, const int64_t *rp, const int32_t *ci, const double *va,
              const double *b, const double *x0, double *x, int m, int method, int gs,
              double tol, int max_cycles, double normA, int64_t hist_cap, double *hist_res,
              double *hist_lfro, int64_t *hist_len, double *beta_out, int *cycles_out,
              int64_t *steps_out)
{
    if (n <= 0 || m < 1 || (method != ORA_MGS && method != ORA_IGS && method != ORA_ONE_REDUCE) || gs < 1 ||
        gs > 2 || max_cycles < 1)
        return ORA_EINVAL;
    double *V = (double *)malloc((size_t)n * (m + 1) * sizeof(double));
    double *H = (double *)malloc((size_t)(m + 1) * m * sizeof(double));
    double *L = (double *)malloc((size_t)(m + 1) * (m + 1) * sizeof(double));
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)malloc((size_t)m * sizeof(double));
    if (!V || !H || !L || !r || !y) {
        free(V); free(H); free(L); free(r); free(y);
        return ORA_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = x0 ? x0[i] : 0.0;
    const double nb = ora_nrm2(n, b);
    int64_t hlen = 0, steps = 0;
    int cycles = 0, status = ORA_NOT_CONVERGED;
    double beta = NAN;
    for (;;) {
        /* r_0 = b - A x_0, rho = ||r_0|| (step 1). */
        ora_spmv(n, rp, ci, va, x, r);
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        beta = ora_backward_error(n, rp, ci, va, b, x, normA);
        if (!isfinite(beta)) { status = ORA_ENUMERIC; break; }
        if (beta <= tol) { status = ORA_OK; break; }
        if (cycles >= max_cycles) { status = ORA_NOT_CONVERGED; break; }
        double rho = ora_nrm2(n, r);
        if (rho == 0.0) { status = ORA_OK; break; }

        memset(V, 0, (size_t)n * (m + 1) * sizeof(double));
        memset(H, 0, (size_t)(m + 1) * m * sizeof(double));
        memset(L, 0, (size_t)(m + 1) * (m + 1) * sizeof(double));
        givens_ls G;
        if (givens_init(&G, m, rho) != ORA_OK) { givens_free(&G); status = ORA_ENOMEM; break; }
        cycle_ctl ctl;
        ctl.stop_den = nb + normA * ora_nrm2(n, x);
        ctl.tol = tol;
        ctl.hist_res = hist_res ? hist_res + hlen : NULL;
        ctl.hist_lfro = hist_lfro ? hist_lfro + hlen : NULL;
        ctl.hist_room = hist_cap - hlen;
        ctl.res_last = rho;
        int cst = ORA_OK;
        int done = method == ORA_MGS
                       ? mgs_cycle(n, rp, ci, va, r, m, V, H, rho, &G, &ctl, &cst)
                       : method == ORA_IGS
                             ? igs_cycle(n, rp, ci, va, r, m, gs, V, H, L, rho, &G, &ctl, &cst)
                             : one_reduce_cycle(n, rp, ci, va, r, m, V, H, L, rho, &G, &ctl, &cst);
        int64_t room = hist_cap - hlen;
        hlen += done < room ? done : (room > 0 ? room : 0);
        steps += done;
        cycles += 1;
        if (cst == ORA_ENUMERIC || cst == ORA_ENOMEM) { givens_free(&G); status = cst; break; }
        /* x_m = x_0 + V_m y_m. */
        if (done > 0) {
            givens_solve(&G, done, y);
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                double s = 0.0;
                for (int c = 0; c < done; ++c) s += V[(int64_t)c * n + i] * y[c];
                x[i] = x[i] + s;
            }
        }
        givens_free(&G);
        if (cst == ORA_BREAKDOWN) {
            beta = ora_backward_error(n, rp, ci, va, b, x, normA);
            status = (isfinite(beta) && beta <= tol) ? ORA_OK : ORA_BREAKDOWN;
            break;
        }
    }
    if (hist_len) *hist_len = hlen;
    if (beta_out) *beta_out = beta;
    if (cycles_out) *cycles_out = cycles;
    if (steps_out) *steps_out = steps;
    free(V); free(H); free(L); free(r); free(y);
    return status;
}
