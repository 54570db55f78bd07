/*
 * igs_batch.h -- batched IGS-GMRES: many independent sparse FP64 systems A_s x_s = b_s solved
 * by one persistent GPU launch (sm_103a).
 *
 * Each system is solved by the restarted IGS-GMRES(m) of Alg. 4.1 (arXiv 2205.07805), with
 * the same readings as the single-system solver of igs.h: the prime step projects once, the
 * loop runs k = 3..m+1 plus a flush that sets H_{m+1,m}, the Givens least squares (eq.
 * "llse") is updated every step, the in-cycle stop test is |g_{j+1}| <= tol (||b|| +
 * ||A||_2 ||x0||), a cycle ends early on breakdown (gamma <= 64 eps ||H(1:j, j)||), and
 * after each cycle the true backward error beta(x) = ||b - A x|| / (||b|| + ||A||_2 ||x||)
 * of eq. "nrbe" decides convergence.  All arithmetic is IEEE binary64.
 *
 * Determinism: a system's results (x, beta, steps, cycles, status) depend only on that
 * system and the solve options.  They are bitwise identical whether the system is solved
 * alone or inside any batch, and under every launch configuration (block threads, blocks per
 * SM) that igs_batch_set_config or the tuner can choose.
 *
 * Conventions are those of igs.h: status codes are IGS_*, the caller owns every pointer, the
 * calls return after their GPU work completes, calls on one batch must be serialised.
 */
#ifndef IGS_BATCH_H
#define IGS_BATCH_H

#include <stdint.h>

#include "igs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct igs_batch igs_batch;

/* Largest restart length and largest system of a batch. */
enum { IGS_BATCH_MAX_M = 64, IGS_BATCH_MAX_N = 16384, IGS_BATCH_MAX_TUNE = 32 };

typedef struct {
    void *stream;           /* cudaStream_t for all GPU work; NULL: a private stream          */
    int device;             /* CUDA device ordinal                                           */
    int restart_m;          /* m, 1..IGS_BATCH_MAX_M                                          */
    const double *A_norm2;  /* host array[count] of ||A_s||_2 (>= 0) for beta; NULL: estimate  */
                            /* each by power iteration on A_s^T A_s on the GPU                */
    int norm2_iters;        /* power iterations (<= 0: 100)                                   */
    int block_threads;      /* 128, 256 or 512; 0 (with blocks_per_sm = 0): autotune at create */
    int blocks_per_sm;      /* resident CTAs per SM, 1..8; 0: autotune                         */
} igs_batch_opts;

typedef struct {
    int gs_iters;           /* Gauss-Seidel iterations per step: 1 or 2                        */
    double tol_beta;        /* stop when beta(x_s) <= tol_beta (>= 0)                          */
    int max_restarts;       /* cycles per system, >= 1                                         */
    int inputs_on_device;   /* nonzero: b, x0 and every pointer in igs_batch_result are device */
                            /* pointers; zero: host pointers                                   */
} igs_batch_solve_opts;

typedef struct {
    double *x;              /* [total_rows], caller-allocated (required)                       */
    double *beta;           /* [count] backward error per system (nullable)                    */
    int *status;            /* [count] IGS_OK / IGS_NOT_CONVERGED / IGS_BREAKDOWN / IGS_ENUMERIC */
    int64_t *steps;         /* [count] Arnoldi steps (completed Hessenberg columns) (nullable) */
    int *cycles;            /* [count] cycles run (nullable)                                   */
    int64_t total_steps;    /* out: sum of steps over the batch                                */
    int n_ok, n_not_converged, n_breakdown, n_numeric;  /* out: systems per status            */
    double device_ms;       /* out: device time of the launch (CUDA events)                    */
} igs_batch_result;

typedef struct {
    int block_threads;
    int blocks_per_sm;
    double ms;              /* device time of the tuning sample under this configuration      */
} igs_batch_tune_entry;

typedef struct {
    int count;
    int64_t total_rows, nnz;
    int max_rows, restart_m;
    int block_threads, blocks_per_sm, num_sms;  /* launch configuration in use              */
    int64_t smem_bytes;     /* dynamic shared memory per CTA                                   */
    int64_t basis_bytes;    /* device memory of the per-CTA Krylov bases                       */
    int n_tune;             /* entries of tune[] filled by the last tuning run                 */
    igs_batch_tune_entry tune[IGS_BATCH_MAX_TUNE];
} igs_batch_info;

/* Copy `count` systems to the device.  The systems are the diagonal blocks of one
 * block-diagonal CSR matrix: rows sys_ptr[s] .. sys_ptr[s+1]-1 (sys_ptr[0] = 0, count+1
 * entries, each block 1..IGS_BATCH_MAX_N rows) belong to system s, and every entry of those
 * rows must have its column in the same range.  rowptr has sys_ptr[count]+1 entries (int64,
 * nondecreasing, rowptr[0] = 0), colind/vals rowptr[total] entries (< 2^31).  Vectors of the
 * batch (b, x0, x) are the systems' vectors concatenated in the same order.
 * With opts->block_threads = opts->blocks_per_sm = 0 the launch configuration is tuned here:
 * every configuration the GPU can hold is timed on every 4th system (largest first) with
 * b = A * ones, two Gauss-Seidel iterations and tol_beta = 1e-12; the fastest is kept.
 * Errors: IGS_EINVAL (null pointer, bad sizes, an entry outside its block, restart_m out of
 * range, a block too large for shared memory), IGS_ENUMERIC (non-finite entry), IGS_ENOMEM,
 * IGS_ECUDA.  *out is NULL on error. */
int igs_batch_create(igs_batch **out, int count, const int64_t *sys_ptr, const int64_t *rowptr,
                     const int32_t *colind, const double *vals, const igs_batch_opts *opts);

/* Release everything (NULL-safe). */
void igs_batch_destroy(igs_batch *bt);

/* Solve every system: one graph-captured persistent launch.  x0 may be NULL (zero start).
 * Returns IGS_OK when every system converged, else the worst per-system outcome in the
 * order IGS_ENUMERIC, IGS_NOT_CONVERGED, IGS_BREAKDOWN (res filled in every case), or
 * IGS_EINVAL / IGS_ECUDA. */
int igs_batch_solve(igs_batch *bt, const double *b, const double *x0,
                    const igs_batch_solve_opts *opts, igs_batch_result *res);

/* Use a given launch configuration (block_threads 128/256/512, blocks_per_sm within the
 * GPU's occupancy and the basis slots allocated at create).  Results do not change. */
int igs_batch_set_config(igs_batch *bt, int block_threads, int blocks_per_sm);

/* Re-run the tuner (see igs_batch_create) with the given solve options. */
int igs_batch_tune(igs_batch *bt, int gs_iters, double tol_beta, int max_restarts);

/* Sizes, launch configuration and the last tuning table. */
int igs_batch_get_info(const igs_batch *bt, igs_batch_info *info);

/* The ||A_s||_2 in use (given or estimated): out[count], host. */
int igs_batch_get_norms(const igs_batch *bt, double *out);

/* Text of the last error met by bt (never NULL). */
const char *igs_batch_last_error(const igs_batch *bt);

#ifdef __cplusplus
}
#endif
#endif /* IGS_BATCH_H */
