/*
 * igs_serve.h -- IGS-GMRES request server on one GPU (sm_103a): a continuous-batching request
 * loop for solves that arrive over time.
 *
 * Each request is one sparse FP64 system A x = b solved by restarted IGS-GMRES(m) (Alg. 4.1
 * of arXiv 2205.07805, with the readings of the single-system solver in igs.h), in FP64 or
 * in the precision form (FP32 basis inside FP64 iterative refinement, IGS_PREC_FP32_IR).
 *
 * How the server works
 *  - Submitting copies the request to the host side of the server; nothing waits on the GPU.
 *  - igs_server_pump admits queued requests in arrival order while a launch slot (one CUDA
 *    stream each) is free, the request's device memory fits in the server's arena (the
 *    "HBM budget": A, b, x, the Krylov basis, the Givens factors and exchange buffers of the
 *    request are carved out of one device allocation made at create), and its gang fits on
 *    the GPU beside the running gangs (the CTA budget: all running gangs are co-resident at
 *    once, so a large gang is never starved by smaller ones launched after it).  An admitted request is
 *    copied to the GPU and solved by ONE kernel launch: a cooperative gang of G CTAs (G grows
 *    with n, about rows_per_cta rows per CTA) that runs all cycles on the device, keeping the
 *    basis, the Hessenberg/Givens state and every scalar there.  Requests on different slots
 *    run concurrently; a request that arrives while others run starts as soon as a slot and
 *    memory free up.
 *  - The same pump call finds finished requests (CUDA events), copies x to host memory held by
 *    the server, releases their device memory, and queues a completion record.
 *  - Large requests (n >= graph_min_n, when set) take a graph lane instead: a worker thread
 *    of the server solves each with the single-system library of igs.h (its whole-GPU kernels
 *    are the faster executor for one large system).  graph_lanes lanes run concurrently, each
 *    on its own stream, so that large requests overlap on the device with each other (one
 *    fills the others' single-block steps) and with the gangs of the other requests.
 *  - A request's result depends only on the request (its matrix, b, x0 and options) and the
 *    server's options: it is bitwise the same alone and in any mix (its lane and gang size are
 *    functions of n, and no arithmetic of one request touches another's data).
 *
 * Calls on one server must be serialised by the caller (one thread drives it; the graph lane's
 * worker is internal and synchronised with the calls).  Status codes
 * are the IGS_* codes of igs.h; IGS_ETIMEOUT in a completion means the request's gang could
 * not synchronise within its bounded wait (no GPU hang: every wait in the kernel is bounded).
 */
#ifndef IGS_SERVE_H
#define IGS_SERVE_H

#include <stdint.h>

#include "igs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct igs_server igs_server;

enum { IGS_SERVE_MAX_M = 128 };

typedef struct {
    int device;             /* CUDA device ordinal                                           */
    int max_restart_m;      /* largest restart length of any request, 1..IGS_SERVE_MAX_M      */
    int64_t arena_bytes;    /* device memory for admitted requests (the admission budget)    */
    int slots;              /* requests in flight at once (one stream each), 1..256; 0: 8     */
    int rows_per_cta;       /* target rows per CTA of a request's gang (>= 256, multiple of
                               32); 0: 4096                                                  */
    int max_queue;          /* requests waiting for admission at most; a submit beyond it is
                               refused with IGS_ENOMEM ("queue full").  0: no limit          */
    int64_t graph_min_n;    /* requests with n >= graph_min_n take the graph lane: one at a
                               time, on a worker thread of the server, through igs_create /
                               igs_solve (igs.h: whole-GPU kernels, graph-captured cycles,
                               pooled device memory outside the arena), beside the gangs.
                               0: no graph lane                                              */
    int graph_lanes;        /* graph-lane requests in flight at once (one worker thread and
                               stream each, 1..16), so that large requests overlap on the
                               device; 0: 1                                                  */
} igs_server_opts;

typedef struct {
    int64_t n, nnz;         /* system size; rowptr/colind/vals as in igs_create (host arrays) */
    const int64_t *rowptr;
    const int32_t *colind;
    const double *vals;
    const double *b;        /* host, n entries                                               */
    const double *x0;       /* host, n entries, nullable (zero start)                        */
    double A_norm2;         /* ||A||_2 for beta (eq. "nrbe"); <= 0: estimated on the GPU by the
                               library's power iteration on A^T A (as igs_create does), on a
                               worker thread of the server, before the request is admitted
                               (a failed estimate falls back to the bound
                               sqrt(||A||_1 ||A||_inf) >= ||A||_2); the completion record
                               carries the value used                                        */
    int restart_m;          /* 1..max_restart_m                                               */
    int gs_iters;           /* 1 or 2                                                         */
    double tol_beta;        /* stop when beta(x) <= tol_beta                                  */
    int max_restarts;       /* cycles (FP64) or refinement steps (FP32_IR), >= 1              */
    int precision;          /* IGS_PREC_FP64 or IGS_PREC_FP32_IR                              */
    double inner_tol;       /* FP32_IR: residual reduction per FP32 cycle (<= 0: 1e-6)        */
} igs_request;

typedef struct {
    int64_t id;             /* as returned by igs_server_submit                               */
    int status;             /* IGS_OK, IGS_NOT_CONVERGED, IGS_BREAKDOWN, IGS_ENUMERIC,
                               IGS_ETIMEOUT, or IGS_ECUDA (launch failed)                     */
    double beta;            /* backward error of the returned x (eq. "nrbe")                  */
    int64_t steps;          /* Arnoldi columns built over all cycles                          */
    int cycles;
    int gang_ctas;          /* G, the CTAs of the request's launch                            */
    int64_t device_bytes;   /* arena bytes the request held                                   */
    double t_submit, t_admit, t_done;  /* server clock (seconds since create): submitted,
                               launched, and found finished by igs_server_pump               */
    int path;               /* IGS_SERVE_PATH_GANG or IGS_SERVE_PATH_GRAPH (gang_ctas is 0 and
                               device_bytes the context's memory on the graph lane)          */
    double A_norm2;         /* the ||A||_2 the request's beta used                            */
} igs_completion;

enum { IGS_SERVE_PATH_GANG = 0, IGS_SERVE_PATH_GRAPH = 1 };

typedef struct {
    int64_t submitted, queued, running, completed;
    int64_t arena_bytes, arena_used, arena_peak;
    int64_t launches;       /* kernel launches issued (one per admitted request)              */
} igs_server_stats;

/* Create a server: allocates the arena and the launch slots.  Errors: IGS_EINVAL, IGS_ENOMEM,
 * IGS_ECUDA.  *out is NULL on error. */
int igs_server_create(igs_server **out, const igs_server_opts *opts);

/* Release everything (waits for running requests).  NULL-safe. */
void igs_server_destroy(igs_server *srv);

/* Queue a request (validates and copies it; A is converted to SELL-32 here).  *id_out gets
 * the request id.  Errors: IGS_EINVAL (malformed CSR, bad options, a request that can never
 * fit the arena or the GPU), IGS_ENUMERIC (non-finite entry), IGS_ENOMEM (queue full: the
 * request is refused, nothing is kept). */
int igs_server_submit(igs_server *srv, const igs_request *req, int64_t *id_out);

/* Admit and launch what fits; collect finished requests.  *running (nullable) gets the
 * number of requests on the GPU afterwards.  Returns IGS_OK or IGS_ECUDA. */
int igs_server_pump(igs_server *srv, int *running);

/* Completion records not yet returned, oldest first (at most max_out).  *n_out gets the
 * count. */
int igs_server_poll(igs_server *srv, igs_completion *out, int max_out, int *n_out);

/* Copy the solution of a completed request to x (host, n entries) and forget the request.
 * Returns IGS_OK, or IGS_EINVAL (unknown id, not finished, or already taken). */
int igs_server_take_result(igs_server *srv, int64_t id, double *x);

int igs_server_get_stats(const igs_server *srv, igs_server_stats *out);

/* The server clock (seconds since create), for stamping arrivals. */
double igs_server_clock(const igs_server *srv);

const char *igs_server_last_error(const igs_server *srv);

/* Self-test of the gangs' bounded waits (no server needed).  Launches a cooperative gang of
 * G CTAs (2 <= G <= the SM count) on `device` through four of the solver's gang barriers.
 * stall = 0: they complete; returns IGS_OK.  stall = 1: the barrier's arrival counter
 * starts at a value no arrival brings to G (a flag nothing sets), so every CTA's wait runs
 * out after its bound (a few seconds), raises the gang's abort flag and returns; the call then
 * returns IGS_ETIMEOUT with *abort_out = 1 (nullable) and the device stays usable.  This is
 * how the timeout path is tested without faulting or hanging a GPU.  Errors: IGS_EINVAL,
 * IGS_ECUDA. */
int igs_server_gang_selftest(int device, int G, int stall, int *abort_out);

#ifdef __cplusplus
}
#endif
#endif /* IGS_SERVE_H */
