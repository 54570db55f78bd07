/*
 * igs.h -- C interface of the GB300 (sm_103a) IGS-GMRES library.
 *
 * IGS-GMRES is GMRES (Saad and Schultz) whose Arnoldi process orthogonalises each new
 * Krylov vector with one or two iterations of Gauss-Seidel on the normal equations of the
 * Gram-Schmidt projector (Thomas, Carson, Rozloznik, Carr, Swirydowicz, "Iterated
 * Gauss-Seidel GMRES", arXiv 2205.07805: Sec. 1 states the problem, Alg. 4.1 the method).
 * All arithmetic is IEEE binary64 on the GPU.
 *
 * Conventions shared by every call
 *  - Return value: one of the IGS_* status codes below; no call throws or aborts.
 *  - Ownership: the caller owns every pointer it passes; the library never frees or keeps
 *    one after the call returns (igs_create copies A).
 *  - Host/device: a flag names whether vector arguments are host or device (CUDA) memory.
 *    Device pointers must live on the context's device.
 *  - Layouts: vectors are dense float64 arrays of length n.  Matrices returned to the caller
 *    are column-major with the stated leading dimension.
 *  - Streams: all GPU work of a context is ordered on one CUDA stream (given at create, or
 *    a private one).  Every call below returns only after its results are complete.
 *  - Thread safety: calls on different contexts may run concurrently; calls on one context
 *    must be serialised by the caller.
 */
#ifndef IGS_H
#define IGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------------------- */
/* Status codes                                                                         */
/* ----------------------------------------------------------------------------------- */
enum {
    IGS_OK = 0,             /* converged: beta(x) <= tol_beta                              */
    IGS_NOT_CONVERGED = 1,  /* max_restarts cycles ran; x is the last iterate                */
    IGS_BREAKDOWN = 2,      /* invariant Krylov subspace reached with beta(x) > tol; x valid  */
    IGS_EINVAL = -1,        /* invalid argument (null pointer, bad size, malformed CSR)       */
    IGS_ENOMEM = -2,        /* device or host allocation failed                               */
    IGS_ECUDA = -3,         /* a CUDA runtime call failed (igs_last_error has the text)       */
    IGS_ENUMERIC = -4,      /* NaN or Inf met (e.g. in b, A or a normalisation)              */
    IGS_ETIMEOUT = -5,      /* a bounded device-side wait gave up                             */
    IGS_ENOTIMPL = -6       /* option not supported by this build                             */
};

/* Orthogonalisation method of an Arnoldi cycle. */
/* Arnoldi process of a solve (igs_solve_opts.method, igs_arnoldi_ex). */
enum {
    IGS_METHOD_IGS = 1,        /* Alg. 4.1, two-reduce IGS with 1 or 2 Gauss-Seidel iterations  */
    IGS_METHOD_ONE_REDUCE = 2  /* Alg. 4.2, one-reduce hybrid MGS-CGS: one global reduction per
                                  column (lagged norm, Jacobi re-orthogonalisation of the lagged
                                  vector, "Stephen's trick"); gs_iters is ignored.  The paper
                                  leaves its stability analysis open (Sec. 4).                 */
};

typedef struct igs_ctx igs_ctx;

/* Options of igs_create (a null pointer means all defaults). */
typedef struct {
    void *stream;       /* cudaStream_t to run on; NULL: the library creates a private
                           non-blocking stream                                            */
    int device;         /* CUDA device ordinal; < 0: the device current on the calling thread */
    int max_restart_m;  /* largest restart length m of any later solve, 1..232; sizes the
                           Krylov basis (n x (m+1) float64).  <= 0: 100                     */
    double A_norm2;     /* ||A||_2 used by the backward error beta (eq. "nrbe", Sec. 1); <= 0:
                           estimated on the GPU by power iteration on A^T A                 */
    int norm2_iters;    /* power iterations for that estimate; <= 0: 100                     */
    int fp32_basis;     /* nonzero: also allocate an FP32 Krylov basis and FP32 copy of A's
                           values (4 (n+32)(m+2) + 4 nnz bytes more), which solves with
                           precision = IGS_PREC_FP32_IR require                             */
    int stream_alloc;   /* nonzero: the context's device memory comes from the device's
                           stream-ordered pool (cudaMallocAsync on the context's stream) and
                           igs_destroy returns it with cudaFreeAsync, so that neither call
                           waits for work on other streams (cudaFree would); the norm
                           estimate's scratch comes from the same pool                      */
} igs_create_opts;

/* Arithmetic of igs_solve's Arnoldi cycles. */
enum {
    IGS_PREC_FP64 = 0,     /* everything in FP64 (Alg. 4.1 as stated)                          */
    IGS_PREC_FP32_IR = 1,  /* FP32 SpMV, basis and basis updates; FP64 Gram accumulation (FP32
                              sums over 32 rows promoted to FP64), (I+L) solves, Givens least
                              squares, x and r = b - A x.  Each restart is one step of FP64
                              iterative refinement: r = b - A x, an FP32 cycle on A d = r
                              stopped when its residual estimate falls by inner_tol (or meets
                              tol_beta), x = x + d.  The paper names mixed precision only as
                              future work (Sec. 6); this form is this library's extension.   */
    IGS_PREC_FP64_DF = 2   /* FP64 data, SpMV, small steps and x = x0 + V y; the block
                              reductions (Alg. 4.1 steps 5 and 14, Alg. 4.2 step 4) and Alg.
                              4.1's basis updates (steps 13 and 16, out = a src - V c, error
                              <= ~2^-45 sum |V c| per row) are evaluated with double-float
                              arithmetic on the FP32 pipes: each
                              FP64 operand split into two FP32 parts (exact to 2^-47 for
                              2^-100 <= |a| < 2^127), exact products of the high parts, cross
                              terms in FP32 (<= ~2^-45 relative per product), TwoSum
                              accumulation folded into FP64 every 32 terms, FP64 lane sums.
                              For vectors spread over n >= 16384 rows the added error is
                              below the FP64 summation error; smaller systems run the FP64
                              reductions.  GB300's FP64 pipe (1.26 TFLOP/s) bounds the FP64
                              reductions at ~1/3 of HBM bandwidth; these run near HBM speed.
                              An operand >= 2^127 makes the solve stop with IGS_ENUMERIC.
                              The paper's precision is FP64 (Sec. 3); this is a library
                              extension, checked against the FP64 oracle.                   */
};

/* Options of igs_solve. */
typedef struct {
    int restart_m;        /* m, Arnoldi columns per cycle: 1 <= m <= max_restart_m         */
    int gs_iters;         /* Gauss-Seidel iterations per column: 1 or 2 (Alg. 4.1; with 1,
                             steps 14-16 are skipped)                                       */
    double tol_beta;      /* stop when beta(x) <= tol_beta; 0 runs max_restarts full cycles  */
    int max_restarts;     /* at most this many cycles (>= 1)                                 */
    int inputs_on_device; /* 1: b, x0 and res->x are device pointers; 0: host pointers        */
    int precision;        /* IGS_PREC_FP64 (0, default), IGS_PREC_FP32_IR (needs a context
                             created with fp32_basis) or IGS_PREC_FP64_DF; anything else:
                             IGS_EINVAL                                                     */
    double inner_tol;     /* IGS_PREC_FP32_IR: relative residual reduction per FP32 cycle;
                             <= 0: 1e-6.  Ignored for FP64                                   */
    int method;           /* 0 or IGS_METHOD_IGS: Alg. 4.1; IGS_METHOD_ONE_REDUCE: Alg. 4.2
                             (FP64 or FP64_DF)                                               */
} igs_solve_opts;

/* Results of igs_solve.  Input fields are marked "in". */
typedef struct {
    double *x;            /* in: caller-allocated, n entries (host or device per
                             inputs_on_device); out: the approximate solution x_m           */
    double *arnoldi_hist; /* in, nullable host array: out |g_{j+1}| = ||rho e1 - H y||, the
                             Arnoldi residual norm after each completed column, all cycles   */
    double *lfro_hist;    /* in, nullable host array: out ||L_{j+1}||_F per completed column
                             (Henrici departure of I+L, eq. "LOO", Sec. 4)                  */
    int64_t hist_cap;     /* in: capacity of the two history arrays                          */
    int64_t hist_len;     /* out: history entries written                                    */
    double *H;            /* in, nullable host array: out the Hessenberg matrix of the last
                             cycle, (m+1) x m column-major, leading dimension H_ld           */
    int H_ld;             /* in: >= m+1 when H is given                                      */
    double beta;          /* out: beta(x) = ||b - A x|| / (||b|| + ||A||_2 ||x||)            */
    double rho0;          /* out: ||b - A x0||                                               */
    int64_t steps;        /* out: Arnoldi columns built over all cycles                      */
    int cycles;           /* out: cycles run                                                 */
} igs_result;

/* Context information (igs_get_info). */
typedef struct {
    int64_t n, nnz;
    int max_restart_m;
    int device;
    double A_norm2;        /* the value beta uses (given or estimated)                      */
    int A_norm2_estimated; /* 1 when estimated on the GPU                                   */
    int64_t device_bytes;  /* device memory held by the context                             */
} igs_info;

/* ----------------------------------------------------------------------------------- */
/* Calls                                                                                */
/* ----------------------------------------------------------------------------------- */

/* Create a solver context for the n x n matrix A given in CSR form (Sec. 1: "A x = b with
 * A an n x n real matrix").  rowptr (n+1 entries, rowptr[0] = 0, non-decreasing,
 * rowptr[n] = nnz), colind (nnz entries in [0, n)) and vals (nnz) are HOST arrays; they are
 * validated, copied to the device and may be freed on return.  The context allocates the
 * Krylov basis and all workspace here; igs_solve allocates nothing on the device.
 * Errors: IGS_EINVAL (null pointers, n < 1, nnz < 0, nnz >= 2^31, malformed CSR),
 * IGS_ENOMEM, IGS_ECUDA, IGS_ENUMERIC (non-finite value).  *out is NULL on error. */
int igs_create(igs_ctx **out, int64_t n, int64_t nnz, const int64_t *rowptr,
               const int32_t *colind, const double *vals, const igs_create_opts *opts);

/* Release a context and its device memory.  NULL is accepted. */
void igs_destroy(igs_ctx *ctx);

/* Solve A x = b by restarted IGS-GMRES(m) (Alg. 4.1, then y_m = argmin ||rho e1 - H y||,
 * x_m = x_0 + V_m y_m; restart from x_m).  b (n entries) and x0 (n entries, NULL = zero)
 * follow opts->inputs_on_device.  Within a cycle the run stops early once the estimate
 * |g_{j+1}| / (||b|| + ||A||_2 ||x0||) <= tol_beta; after each cycle the true beta(x) is
 * computed on the GPU and decides convergence.
 * Returns IGS_OK, IGS_NOT_CONVERGED or IGS_BREAKDOWN with res filled (x is always
 * written), or an error code (res->x unspecified). */
int igs_solve(igs_ctx *ctx, const double *b, const double *x0, const igs_solve_opts *opts,
              igs_result *res);

/* Run exactly one Arnoldi cycle (Alg. 4.1 steps 1-18 for k = 3..m+1 plus the final
 * normalisation of w_{m+1}) on the start vector r0 (n entries) and copy out its factors:
 *   V: n x (m+1) column-major, leading dimension ldv >= n (nullable),
 *   H: (m+1) x m column-major, leading dimension m+1 (nullable),
 *   L: (m+1) x (m+1) row-major; row i holds v_{i+1}^T V_i in columns 0..i-1 (nullable).
 * on_device selects host or device memory for r0, V, H and L.  *ncols receives the number
 * of completed Hessenberg columns (< m after a breakdown), *rho = ||r0||.
 * Returns IGS_OK, IGS_BREAKDOWN or an error code. */
int igs_arnoldi(igs_ctx *ctx, const double *r0, int m, int gs_iters, int on_device,
                double *V, int64_t ldv, double *H, double *L, int *ncols, double *rho);

/* y = A x with the context's matrix (n entries each; host or device per on_device). */
int igs_spmv(igs_ctx *ctx, const double *x, double *y, int on_device);

/* igs_arnoldi with the Arnoldi process chosen: method IGS_METHOD_IGS (Alg. 4.1, gs_iters 1
 * or 2) or IGS_METHOD_ONE_REDUCE (Alg. 4.2; L then holds the rows u_{k-1}^T V_{k-2} / gamma of
 * the lagged vectors, as the algorithm defines them), and the arithmetic: precision
 * IGS_PREC_FP64 or IGS_PREC_FP64_DF (anything else: IGS_EINVAL).  Same arguments and results
 * otherwise. */
int igs_arnoldi_ex(igs_ctx *ctx, const double *r0, int m, int method, int gs_iters, int precision, int on_device,
                   double *V, int64_t ldv, double *H, double *L, int *ncols, double *rho);

/* Fill *info.  Returns IGS_OK or IGS_EINVAL. */
int igs_get_info(const igs_ctx *ctx, igs_info *info);

/* Kernel-class timing.  While enabled, igs_solve and igs_arnoldi record CUDA events around
 * each kernel launch and accumulate per-class device time.  Classes: 0 SpMV, 1 block
 * reduction (multi-dot), 2 basis update, 3 small serial steps, 4 cycle set-up/finish. */
enum { IGS_KCLASS_SPMV = 0, IGS_KCLASS_DOTS = 1, IGS_KCLASS_UPDATE = 2, IGS_KCLASS_SMALL = 3,
       IGS_KCLASS_CYCLE = 4, IGS_KCLASS_COUNT = 5 };
typedef struct {
    double ms[IGS_KCLASS_COUNT];        /* summed device time per class                 */
    int64_t launches[IGS_KCLASS_COUNT]; /* kernel launches per class                    */
    double bytes[IGS_KCLASS_COUNT];     /* algorithmic bytes moved per class            */
    double flops[IGS_KCLASS_COUNT];     /* algorithmic floating-point operations        */
} igs_profile;
int igs_profile_enable(igs_ctx *ctx, int enable); /* enabling also clears the counters */
int igs_profile_get(igs_ctx *ctx, igs_profile *out);

/* Total kernel launches issued by this context since creation (for launch accounting). */
int64_t igs_launch_count(const igs_ctx *ctx);

/* Block multi-dot that allocates no device memory.  The paper has no counterpart: this is a
 * service for callers that may not call cudaMalloc (a host application that owns all device
 * memory and forbids plug-ins from allocating; code running while another thread captures
 * a CUDA graph in global capture mode; loops that cannot take cudaMalloc's implicit device
 * synchronisation).
 *   out[c]     = V[:, c]^T x0   for c < p
 *   out[p + c] = V[:, c]^T x1   for c < p (only when x1 != NULL)
 * V (n x p column-major, leading dimension ldv), x0, x1 and out are DEVICE pointers on the
 * current device; V, x0 and x1 must be 16-byte aligned, n a multiple of 4 and ldv even and
 * >= n.  The work runs on `stream` (a cudaStream_t; NULL = legacy default stream) and the
 * call returns after it completes.  Same kernel and summation order as the library's
 * step-5 reduction.
 * The per-block partial sums live in a fixed file-scope device array of 16384 doubles
 * (128 KiB) that every GPU loading the library holds until the process exits.  Largest p:
 * 24 x (the GPU's SM count), capped at 8192 -- 3648 on a 152-SM GB300, with or without x1
 * (the kernel's column groups take at most 8 columns each, at most 3 groups per SM; the
 * partial sums of every accepted launch then fit the array).  A larger p is rejected with
 * IGS_EINVAL before anything is launched.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture.  All calls share the array: calls whose GPU work
 * overlaps race on it.  Nothing in it must start at zero (each call writes every partial it
 * reads).  Returns IGS_OK, IGS_EINVAL (bad pointer, size, alignment, or too large) or
 * IGS_ECUDA. */
int igs_block_dots_static(const double *V, int64_t ldv, int p, int64_t n, const double *x0,
                          const double *x1, double *out, void *stream);

/* Arithmetic-pipe probe (measurement support; the paper has no counterpart): the FP64 and
 * FP32 fused multiply-add throughput of `device`, in FMAs per second: the best over 2, 4 and 8
 * blocks of 256 threads per SM with 4, 8 and 16 independent FMA chains per thread (about
 * 1 s of GPU time; allocates a few KB).  On GB300 the
 * FP64 rate bounds this library's FP64 streaming kernels, so the benchmark reports it beside
 * the unit-count FP64 peak.  Returns IGS_OK, IGS_EINVAL (NULL output) or IGS_ECUDA. */
int igs_probe_fma(int device, double *fp64_fma_per_s, double *fp32_fma_per_s);

/* Text of a status code, and of the last error met by ctx (never NULL). */
const char *igs_status_string(int status);
const char *igs_last_error(const igs_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* IGS_H */
