// C interface of the GB300 IGS-GMRES library (declared in include/igs.h).
//
// A solve is a host loop over restart cycles.  Each cycle -- Alg. 4.1 steps 1-18 for
// k = 3..m+1, the final normalisation, the Givens least squares, x_m = x_0 + V_m y_m and the
// backward error of the new x -- is one CUDA graph launch, captured once per (m, gs) and
// replayed; every per-step scalar stays in device memory, so the host waits only once per
// cycle.  The Givens rotation of each completed Hessenberg column runs on a parallel graph
// branch, overlapping the next basis update; its stop decision is consumed one iteration
// later, and the cycle's least squares uses exactly the columns up to the stop.
#include "../../include/igs.h"
#include "igs_internal.h"

#include <algorithm>
#include <cmath>
#include <new>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

using igs::KClass;

struct igs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;  // user-visible ordering stream
    bool own_stream = false;
    bool stream_alloc = false;  // device memory from the stream-ordered pool
    cudaStream_t cap = nullptr;     // private capture stream
    cudaStream_t side = nullptr;    // private side stream (Givens branch during capture)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    igs::Workspace w;
    double normA = 0.0;
    int normA_est = 0;
    int64_t device_bytes = 0;
    std::vector<void *> allocs;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int kernels = 0;
    };
    std::map<std::pair<int, int>, Graph> graphs;
    // profiling (eager execution with events)
    bool profiling = false;
    igs_profile prof{};
    int64_t launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_err;

int fail(igs_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_err = buf;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? IGS_ENOMEM : IGS_ECUDA,    \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                        \
    } while (0)

template <class T>
int dalloc(igs_ctx *ctx, T **p, size_t count)
{
    void *q = nullptr;
    const size_t bytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = ctx->stream_alloc ? cudaMallocAsync(&q, bytes, ctx->stream) : cudaMalloc(&q, bytes);
    if (e != cudaSuccess)
        return fail(ctx, IGS_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    e = ctx->stream_alloc ? cudaMemsetAsync(q, 0, bytes, ctx->stream) : cudaMemset(q, 0, bytes);
    if (e != cudaSuccess) {
        if (ctx->stream_alloc)
            cudaFreeAsync(q, ctx->stream);
        else
            cudaFree(q);
        return fail(ctx, IGS_ECUDA, "cudaMemset failed: %s", cudaGetErrorString(e));
    }
    ctx->allocs.push_back(q);
    ctx->device_bytes += (int64_t)bytes;
    *p = static_cast<T *>(q);
    return IGS_OK;
}

// Issues kernels either while a graph is being captured (count only) or eagerly with
// CUDA events around every kernel (profiling).
struct Issuer {
    igs_ctx *ctx;
    cudaStream_t s;      // main stream
    cudaStream_t side;   // Givens branch (== s when not capturing)
    bool capture;
    int kernels = 0;
    struct Pending {
        cudaEvent_t a, b;
        int cls;
        double bytes, flops;
    };
    std::vector<Pending> pend;

    template <class F>
    cudaError_t run(int cls, double bytes, double flops, F &&fn, cudaStream_t on)
    {
        ++kernels;
        if (capture || !ctx->profiling) return fn(on);
        Pending p{};
        p.cls = cls;
        p.bytes = bytes;
        p.flops = flops;
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        cudaEventRecord(p.a, on);
        cudaError_t e = fn(on);
        cudaEventRecord(p.b, on);
        pend.push_back(p);
        return e;
    }
    void collect()
    {
        for (auto &p : pend) {
            float ms = 0.f;
            cudaEventSynchronize(p.b);
            cudaEventElapsedTime(&ms, p.a, p.b);
            ctx->prof.ms[p.cls] += ms;
            ctx->prof.launches[p.cls] += 1;
            ctx->prof.bytes[p.cls] += p.bytes;
            ctx->prof.flops[p.cls] += p.flops;
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        pend.clear();
    }
};

// Algorithmic traffic / work models (FP64, int32 CSR) used by the profile.
double spmv_bytes(const igs::Workspace &w) { return 12.0 * w.nnz + 4.0 * (w.n + 1) + 16.0 * w.n; }
double dots_bytes(const igs::Workspace &w, int p, int nq) { return 8.0 * w.n * (p + nq); }
double upd_bytes(const igs::Workspace &w, int p) { return 8.0 * w.n * (p + 2); }

// Enqueue one restart cycle (see the file comment).  Precondition: ctx->w.r = b - A x,
// st->rnorm/xnorm/bnorm set (by the solve set-up or the previous cycle's end).
cudaError_t enqueue_cycle32(igs_ctx *ctx, Issuer &is, int m, int gs);
cudaError_t enqueue_cycle_1r(igs_ctx *ctx, Issuer &is, int m, bool df);
cudaError_t enqueue_cycle_vdf(igs_ctx *ctx, Issuer &is, int m, int gs);
cudaError_t enqueue_cycle_1r_vdf(igs_ctx *ctx, Issuer &is, int m);

// The block multi-dot of the FP64 cycles: FP64 FMAs, or double-float products on the FP32
// pipes for the IGS_PREC_FP64_DF form (from kDfMinRows rows on; same partial-sum layout).
using DotsLauncher = cudaError_t (*)(const igs::Workspace &, int, const double *, const double *, bool,
                                     cudaStream_t, igs::DotsPlan *);
DotsLauncher dots_launcher(const igs::Workspace &w, bool df)
{
    return df && igs::dots_df_applies(w) ? igs::launch_dots_df : igs::launch_dots;
}

// gs = 0 selects Alg. 4.2 (one-reduce); 1 or 2 Alg. 4.1 with that many GS iterations.
cudaError_t enqueue_cycle(igs_ctx *ctx, Issuer &is, int m, int gs, int prec)
{
    if (gs == 0 && prec == IGS_PREC_FP64_DF && igs::dots_df_applies(ctx->w)) return enqueue_cycle_1r_vdf(ctx, is, m);
    if (gs == 0) return enqueue_cycle_1r(ctx, is, m, prec == IGS_PREC_FP64_DF);
    if (prec == IGS_PREC_FP32_IR) return enqueue_cycle32(ctx, is, m, gs);
    if (prec == IGS_PREC_FP64_DF && igs::dots_df_applies(ctx->w)) return enqueue_cycle_vdf(ctx, is, m, gs);
    const igs::Workspace &w = ctx->w;
    const DotsLauncher dots = igs::launch_dots;
    cudaStream_t s = is.s;
    const int64_t ld = w.ld;
    double *V = w.V;
    auto col = [&](int c) { return V + (int64_t)c * ld; };
    cudaError_t e;
#define RUN(cls, bytes, flops, on, expr)                                          \
    do {                                                                          \
        e = is.run((cls), (bytes), (flops), [&](cudaStream_t st_) { (void)st_; return (expr); }, (on)); \
        if (e != cudaSuccess) return e;                                           \
    } while (0)

    // Step 1: rho = ||r0||, v1 = r0 / rho.
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_cycle_start(w, 0, st_));
    RUN(igs::KC_CYCLE, 16.0 * w.n, w.n, s, igs::launch_scale(w, w.r, col(0), 0, false, st_));
    // Step 2: w2 = A v1, H11 = v1^T w2, w2 -= H11 v1.
    igs::DotsPlan pl{};
    RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, col(0), col(1), nullptr, false, st_));
    RUN(igs::KC_DOTS, dots_bytes(w, 1, 1), 2.0 * w.n, s, dots(w, 1, col(1), nullptr, false, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_prime(w, pl, st_));
    RUN(igs::KC_UPDATE, upd_bytes(w, 1), 2.0 * w.n, s,
        igs::launch_update(w, 1, w.r1v, false, 1.0, col(1), col(1), false, false, false, st_));

    bool pending_join = false;
    auto join_side = [&]() -> cudaError_t {
        if (pending_join && is.capture) {
            cudaError_t ee = cudaStreamWaitEvent(s, ctx->ev_join, 0);
            if (ee != cudaSuccess) return ee;
        }
        pending_join = false;
        return cudaSuccess;
    };
    auto fork_givens = [&](int j) -> cudaError_t {
        cudaStream_t on = s;
        if (is.capture) {
            cudaError_t ee = cudaEventRecord(ctx->ev_fork, s);
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(is.side, ctx->ev_fork, 0);
            if (ee != cudaSuccess) return ee;
            on = is.side;
        }
        cudaError_t ee = is.run(igs::KC_SMALL, 0, 0, [&](cudaStream_t st_) { return igs::launch_givens(w, j, st_); }, on);
        if (ee != cudaSuccess) return ee;
        if (is.capture) {
            ee = cudaEventRecord(ctx->ev_join, is.side);
            if (ee != cudaSuccess) return ee;
            pending_join = true;
        }
        return cudaSuccess;
    };

    for (int k = 3; k <= m + 1; ++k) {
        const int p = k - 1;
        // the previous column's Givens kernel (side branch) is complete before this
        // column's step kernel reads its stop decision
        if ((e = join_side()) != cudaSuccess) return e;
        double *wv = col(p - 1);
        // Step 4: v_k = A w_{k-1}.
        RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, wv, w.z, nullptr, true, st_));
        // Step 5: [V_{k-2}, w_{k-1}]^T [w_{k-1}, v_k] (block partial sums).
        RUN(igs::KC_DOTS, dots_bytes(w, p, 2), 4.0 * w.n * p, s, dots(w, p, wv, w.z, true, st_, &pl));
        // Steps 6-12 (+ step 17 for one iteration).
        RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_a(w, k, gs, pl, st_));
        // Givens least squares for the column completed by step 6 (column k-2, 1-based).
        if ((e = fork_givens(k - 3)) != cudaSuccess) return e;
        // Steps 7, 11, 13: v_{k-1} = w/gamma in place, u_k = v_k/gamma - V_{k-1} r^(1).
        double *uout = gs == 1 ? col(p) : w.u;
        RUN(igs::KC_UPDATE, upd_bytes(w, p) + 8.0 * w.n, 2.0 * w.n * p, s,
            igs::launch_update(w, p, w.r1v, false, 0.0, w.z, uout, true, false, true, st_));
        if (gs == 2) {
            // Step 14: r^(2) = V_{k-1}^T u_k.
            RUN(igs::KC_DOTS, dots_bytes(w, p, 1), 2.0 * w.n * p, s, dots(w, p, w.u, nullptr, true, st_, &pl));
            // Steps 15, 17.
            RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_b(w, k, pl, st_));
            // Step 16: w_k = u_k - V_{k-1} r^(3).
            RUN(igs::KC_UPDATE, upd_bytes(w, p), 2.0 * w.n * p, s,
                igs::launch_update(w, p, w.r3v, false, 1.0, w.u, col(p), false, false, true, st_));
        }
    }
    // Flush: gamma_{m+1} = ||w_{m+1}||, H_{m+1,m}, last L row, v_{m+1} = w_{m+1}/gamma.
    if ((e = join_side()) != cudaSuccess) return e;
    RUN(igs::KC_DOTS, dots_bytes(w, m + 1, 1), 2.0 * w.n * (m + 1), s,
        dots(w, m + 1, col(m), nullptr, true, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_flush(w, m, pl, st_));
    RUN(igs::KC_CYCLE, 16.0 * w.n, w.n, s, igs::launch_scale(w, col(m), col(m), 1, true, st_));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_givens(w, m - 1, st_));
    // Least squares y = argmin ||rho e1 - H y||, x_m = x_0 + V_m y_m.
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_lsq(w, m, st_));
    RUN(igs::KC_CYCLE, upd_bytes(w, m), 2.0 * w.n * m, s,
        igs::launch_update(w, 0, w.y, true, 1.0, w.x, w.x, false, true, false, st_));
    // r = b - A x, ||r||, ||x||, beta(x).
    RUN(igs::KC_CYCLE, spmv_bytes(w) + 8.0 * w.n, 2.0 * w.nnz, s, igs::launch_spmv(w, w.x, w.r, w.b, false, st_));
    int nblk = 0;
    RUN(igs::KC_CYCLE, 16.0 * w.n, 4.0 * w.n, s, igs::launch_norms(w, w.r, w.x, nullptr, &nblk, st_));
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_beta(w, nblk, st_));
#undef RUN
    return cudaSuccess;
}

// One Alg. 4.1 cycle of the double-float form (IGS_PREC_FP64_DF, n >= kDfMinRows): the same
// steps and single-block kernels as the FP64 cycle, with the basis stored split (each element
// as its FP32 (hi, lo) pair in V's bytes, written once when its column is formed) and the
// multi-dots and basis updates in double-float arithmetic.  FP64 vectors: the current
// unnormalised w (in w.t; the SpMV input and the source of step 7's v = w / gamma), z = A w,
// u, x and r.  z is also kept split (in w.u's bytes: step 5 reads it before step 13 writes
// u), and u (in w.r's bytes, which hold r only at the cycle's start and end) for step 14.
// x = x0 + V y and r = b - A x stay FP64.
cudaError_t enqueue_cycle_vdf(igs_ctx *ctx, Issuer &is, int m, int gs)
{
    const igs::Workspace &w = ctx->w;
    cudaStream_t s = is.s;
    const int64_t ld = w.ld;
    auto col = [&](int c) { return w.V + (int64_t)c * ld; };
    auto cold = [&](int c) { return reinterpret_cast<float2 *>(w.V + (int64_t)c * ld); };
    double *wb = w.t;                               // FP64 w
    float2 *ud = reinterpret_cast<float2 *>(w.r);   // split u (between the cycle's start and end)
    float2 *zd = reinterpret_cast<float2 *>(w.u);   // split z (from the SpMV until step 13 writes u)
    const double *zdd = reinterpret_cast<const double *>(zd);
    cudaError_t e;
#define RUN(cls, bytes, flops, on, expr)                                          \
    do {                                                                          \
        e = is.run((cls), (bytes), (flops), [&](cudaStream_t st_) { (void)st_; return (expr); }, (on)); \
        if (e != cudaSuccess) return e;                                           \
    } while (0)
    // Step 1: rho = ||r0||, v1 = r0 / rho (split into the basis, FP64 into wb).
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_cycle_start(w, 0, st_));
    RUN(igs::KC_CYCLE, 16.0 * w.n, w.n, s, igs::launch_scale_df(w, w.r, cold(0), wb, 0, false, st_));
    // Step 2: w2 = A v1, H11 = v1^T w2, w2 -= H11 v1.
    igs::DotsPlan pl{};
    RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, wb, w.z, nullptr, false, st_, zd));
    RUN(igs::KC_DOTS, dots_bytes(w, 1, 1), 2.0 * w.n, s, igs::launch_dots_df_ex(w, 1, zdd, nullptr, false, true, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_prime(w, pl, st_));
    RUN(igs::KC_UPDATE, upd_bytes(w, 1), 2.0 * w.n, s,
        igs::launch_update_df_ex(w, 1, w.r1v, false, 1.0, w.z, wb, cold(1), nullptr, false, false, true, st_));

    bool pending_join = false;
    auto join_side = [&]() -> cudaError_t {
        if (pending_join && is.capture) {
            cudaError_t ee = cudaStreamWaitEvent(s, ctx->ev_join, 0);
            if (ee != cudaSuccess) return ee;
        }
        pending_join = false;
        return cudaSuccess;
    };
    auto fork_givens = [&](int j) -> cudaError_t {
        cudaStream_t on = s;
        if (is.capture) {
            cudaError_t ee = cudaEventRecord(ctx->ev_fork, s);
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(is.side, ctx->ev_fork, 0);
            if (ee != cudaSuccess) return ee;
            on = is.side;
        }
        cudaError_t ee = is.run(igs::KC_SMALL, 0, 0, [&](cudaStream_t st_) { return igs::launch_givens(w, j, st_); }, on);
        if (ee != cudaSuccess) return ee;
        if (is.capture) {
            ee = cudaEventRecord(ctx->ev_join, is.side);
            if (ee != cudaSuccess) return ee;
            pending_join = true;
        }
        return cudaSuccess;
    };

    for (int k = 3; k <= m + 1; ++k) {
        const int p = k - 1;
        // the previous column's Givens kernel (side branch) is complete before this
        // column's step kernel reads its stop decision
        if ((e = join_side()) != cudaSuccess) return e;
        // Step 4: v_k = A w_{k-1} (FP64 w; z in FP64 and split).
        RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, wb, w.z, nullptr, true, st_, zd));
        // Step 5: [V_{k-2}, w_{k-1}]^T [w_{k-1}, v_k]: the split basis (w is its column p-1) and z.
        RUN(igs::KC_DOTS, dots_bytes(w, p, 2), 4.0 * w.n * p, s,
            igs::launch_dots_df_ex(w, p, col(p - 1), zdd, true, true, st_, &pl));
        // Steps 6-12 (+ step 17 for one iteration).
        RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_a(w, k, gs, pl, st_));
        if ((e = fork_givens(k - 3)) != cudaSuccess) return e;
        // Steps 7, 11, 13: column p-1 = split(w / gamma), u = z / gamma - V_{k-1} r^(1) (FP64 and
        // split; with one iteration u is w_k: FP64 into wb, split into column p).
        double *uout = gs == 1 ? wb : w.u;
        float2 *udf = gs == 1 ? cold(p) : ud;
        RUN(igs::KC_UPDATE, upd_bytes(w, p) + 8.0 * w.n, 2.0 * w.n * p, s,
            igs::launch_update_df_ex(w, p, w.r1v, false, 0.0, w.z, uout, udf, wb, true, false, true, st_));
        if (gs == 2) {
            // Step 14: r^(2) = V_{k-1}^T u_k.
            RUN(igs::KC_DOTS, dots_bytes(w, p, 1), 2.0 * w.n * p, s,
                igs::launch_dots_df_ex(w, p, reinterpret_cast<const double *>(ud), nullptr, true, true, st_, &pl));
            // Steps 15, 17.
            RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_b(w, k, pl, st_));
            // Step 16: w_k = u_k - V_{k-1} r^(3) (FP64 into wb, split into column p).
            RUN(igs::KC_UPDATE, upd_bytes(w, p), 2.0 * w.n * p, s,
                igs::launch_update_df_ex(w, p, w.r3v, false, 1.0, w.u, wb, cold(p), nullptr, false, false, true, st_));
        }
    }
    // Flush: gamma_{m+1} = ||w_{m+1}||, H_{m+1,m}, last L row, v_{m+1} = split(w_{m+1} / gamma).
    if ((e = join_side()) != cudaSuccess) return e;
    RUN(igs::KC_DOTS, dots_bytes(w, m + 1, 1), 2.0 * w.n * (m + 1), s,
        igs::launch_dots_df_ex(w, m + 1, col(m), nullptr, true, true, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_flush(w, m, pl, st_));
    RUN(igs::KC_CYCLE, 16.0 * w.n, w.n, s, igs::launch_scale_df(w, wb, cold(m), nullptr, 1, true, st_));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_givens(w, m - 1, st_));
    // Least squares y = argmin ||rho e1 - H y||, x_m = x_0 + V_m y_m (FP64).
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_lsq(w, m, st_));
    RUN(igs::KC_CYCLE, upd_bytes(w, m), 2.0 * w.n * m, s, igs::launch_xupdate_vdf(w, st_));
    // r = b - A x, ||r||, ||x||, beta(x).
    RUN(igs::KC_CYCLE, spmv_bytes(w) + 8.0 * w.n, 2.0 * w.nnz, s, igs::launch_spmv(w, w.x, w.r, w.b, false, st_));
    int nblk = 0;
    RUN(igs::KC_CYCLE, 16.0 * w.n, 4.0 * w.n, s, igs::launch_norms(w, w.r, w.x, nullptr, &nblk, st_));
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_beta(w, nblk, st_));
#undef RUN
    return cudaSuccess;
}

// One Alg. 4.2 cycle of the double-float form (n >= kDfMinRows): the FP64 Alg. 4.2 cycle's
// steps and single-block kernels on the split basis of enqueue_cycle_vdf.  The current u is
// kept in FP64 in w.t (the SpMV input and the source of v = (u - V r^(2)) / gamma) and split in
// basis column nb (the one reduction reads it there, where the FP64 cycle keeps u); z = A u in
// FP64 and split (w.u's bytes: Alg. 4.2 keeps no other u).
cudaError_t enqueue_cycle_1r_vdf(igs_ctx *ctx, Issuer &is, int m)
{
    const igs::Workspace &w = ctx->w;
    cudaStream_t s = is.s;
    const int64_t ld = w.ld;
    auto col = [&](int c) { return w.V + (int64_t)c * ld; };
    auto cold = [&](int c) { return reinterpret_cast<float2 *>(w.V + (int64_t)c * ld); };
    double *wu = w.t;                               // FP64 u
    float2 *zd = reinterpret_cast<float2 *>(w.u);   // split z
    const double *zdd = reinterpret_cast<const double *>(zd);
    cudaError_t e;
#define RUN(cls, bytes, flops, on, expr)                                          \
    do {                                                                          \
        e = is.run((cls), (bytes), (flops), [&](cudaStream_t st_) { (void)st_; return (expr); }, (on)); \
        if (e != cudaSuccess) return e;                                           \
    } while (0)
    // Step 1: rho = ||r0||, v1 = r0 / rho (split into the basis, FP64 into wu).
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_cycle_start(w, 0, st_));
    RUN(igs::KC_CYCLE, 16.0 * w.n, w.n, s, igs::launch_scale_df(w, w.r, cold(0), wu, 0, false, st_));
    // Step 2: w2 = A v1, H11 = v1^T w2, u_2 = w2 - v1 H11 (FP64 into wu, split into column 1).
    igs::DotsPlan pl{};
    RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, wu, w.z, nullptr, false, st_, zd));
    RUN(igs::KC_DOTS, dots_bytes(w, 1, 1), 2.0 * w.n, s, igs::launch_dots_df_ex(w, 1, zdd, nullptr, false, true, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_prime(w, pl, st_));
    RUN(igs::KC_UPDATE, upd_bytes(w, 1), 2.0 * w.n, s,
        igs::launch_update_df_ex(w, 1, w.r1v, false, 1.0, w.z, wu, cold(1), nullptr, false, false, true, st_));

    bool pending_join = false;
    auto join_side = [&]() -> cudaError_t {
        if (pending_join && is.capture) {
            cudaError_t ee = cudaStreamWaitEvent(s, ctx->ev_join, 0);
            if (ee != cudaSuccess) return ee;
        }
        pending_join = false;
        return cudaSuccess;
    };
    auto fork_givens = [&](int j) -> cudaError_t {
        cudaStream_t on = s;
        if (is.capture) {
            cudaError_t ee = cudaEventRecord(ctx->ev_fork, s);
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(is.side, ctx->ev_fork, 0);
            if (ee != cudaSuccess) return ee;
            on = is.side;
        }
        cudaError_t ee = is.run(igs::KC_SMALL, 0, 0, [&](cudaStream_t st_) { return igs::launch_givens(w, j, st_); }, on);
        if (ee != cudaSuccess) return ee;
        if (is.capture) {
            ee = cudaEventRecord(ctx->ev_join, is.side);
            if (ee != cudaSuccess) return ee;
            pending_join = true;
        }
        return cudaSuccess;
    };
    for (int k = 3; k <= m + 1; ++k) {
        const int nb = k - 2;
        // the previous column's Givens kernel (side branch) is complete before this
        // column's step kernel reads its stop decision
        if ((e = join_side()) != cudaSuccess) return e;
        // Step 4: A u_{k-1} (FP64 u; z in FP64 and split), then the one reduction
        // [V_nb, u]^T [u, A u] over the split basis (u is its column nb).
        RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, wu, w.z, nullptr, true, st_, zd));
        RUN(igs::KC_DOTS, dots_bytes(w, nb + 1, 2), 4.0 * w.n * (nb + 1), s,
            igs::launch_dots_df_ex(w, nb + 1, col(nb), zdd, true, true, st_, &pl));
        // Steps 5, 9, 14, 15 of the previous iteration (column nb-2 complete; in the launch's
        // prologue) and steps 6-8, 12 of this one; column nb-2's Givens rotation on the side.
        RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_1r(w, nb, false, pl, st_));
        if (nb >= 2 && (e = fork_givens(nb - 2)) != cudaSuccess) return e;
        // Steps 10-11, 13: v_{k-1} and u_k in one pass over the split basis.
        RUN(igs::KC_UPDATE, 8.0 * w.n * (nb + 4), 4.0 * w.n * nb, s, igs::launch_update_1r_df(w, nb, w.z, wu, false, st_));
    }
    // Flush: the reduction of u_{m+1} (no product), columns m-2 and m-1 complete, v_{m+1}.
    if ((e = join_side()) != cudaSuccess) return e;
    RUN(igs::KC_DOTS, dots_bytes(w, m + 1, 1), 2.0 * w.n * (m + 1), s,
        igs::launch_dots_df_ex(w, m + 1, col(m), nullptr, true, true, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_1r(w, m, true, pl, st_));
    RUN(igs::KC_UPDATE, 8.0 * w.n * (m + 2), 2.0 * w.n * m, s, igs::launch_update_1r_df(w, m, w.z, wu, true, st_));
    if (m >= 2) RUN(igs::KC_SMALL, 0, 0, s, igs::launch_givens(w, m - 2, st_));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_givens(w, m - 1, st_));
    // Least squares y = argmin ||rho e1 - H y||, x_m = x_0 + V_m y_m (FP64).
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_lsq(w, m, st_));
    RUN(igs::KC_CYCLE, upd_bytes(w, m), 2.0 * w.n * m, s, igs::launch_xupdate_vdf(w, st_));
    // r = b - A x, ||r||, ||x||, beta(x).
    RUN(igs::KC_CYCLE, spmv_bytes(w) + 8.0 * w.n, 2.0 * w.nnz, s, igs::launch_spmv(w, w.x, w.r, w.b, false, st_));
    int nblk = 0;
    RUN(igs::KC_CYCLE, 16.0 * w.n, 4.0 * w.n, s, igs::launch_norms(w, w.r, w.x, nullptr, &nblk, st_));
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_beta(w, nblk, st_));
#undef RUN
    return cudaSuccess;
}

// One cycle of the precision form (IGS_PREC_FP32_IR): the same steps and single-block
// kernels as the FP64 cycle, with the SpMV, the basis, z and u in FP32 (igs_fp32.cu); the
// cycle's residual r = b - A x (FP64, from the previous cycle) enters as v_1 = r / rho and the
// cycle ends with x = x + V y and r = b - A x in FP64: one step of iterative refinement.
cudaError_t enqueue_cycle32(igs_ctx *ctx, Issuer &is, int m, int gs)
{
    const igs::Workspace &w = ctx->w;
    cudaStream_t s = is.s;
    const int64_t ld = w.ld;
    float *V = w.V32;
    auto col = [&](int c) { return V + (int64_t)c * ld; };
    cudaError_t e;
    const double spmv32b = 8.0 * w.nnz + 4.0 * (w.n + 1) + 8.0 * w.n;
    auto dots32b = [&](int p, int nq) { return 4.0 * w.n * (p + nq); };
    auto upd32b = [&](int p) { return 4.0 * w.n * (p + 2); };
#define RUN(cls, bytes, flops, on, expr)                                          \
    do {                                                                          \
        e = is.run((cls), (bytes), (flops), [&](cudaStream_t st_) { (void)st_; return (expr); }, (on)); \
        if (e != cudaSuccess) return e;                                           \
    } while (0)

    // Step 1: rho = ||r0|| (FP64), v1 = r0 / rho (to FP32).
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_cycle_start(w, 0, st_));
    RUN(igs::KC_CYCLE, 12.0 * w.n, w.n, s, igs::launch_scale_to32(w, w.r, col(0), st_));
    // Step 2: w2 = A v1, H11 = v1^T w2, w2 -= H11 v1.
    igs::DotsPlan pl{};
    RUN(igs::KC_SPMV, spmv32b, 2.0 * w.nnz, s, igs::launch_spmv32(w, col(0), col(1), st_));
    RUN(igs::KC_DOTS, dots32b(1, 1), 2.0 * w.n, s, igs::launch_dots32(w, 1, col(1), nullptr, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_prime(w, pl, st_));
    RUN(igs::KC_UPDATE, upd32b(1), 2.0 * w.n, s, igs::launch_update32(w, 1, w.r1v, 1.0, col(1), col(1), false, st_));

    bool pending_join = false;
    auto join_side = [&]() -> cudaError_t {
        if (pending_join && is.capture) {
            cudaError_t ee = cudaStreamWaitEvent(s, ctx->ev_join, 0);
            if (ee != cudaSuccess) return ee;
        }
        pending_join = false;
        return cudaSuccess;
    };
    auto fork_givens = [&](int j) -> cudaError_t {
        cudaStream_t on = s;
        if (is.capture) {
            cudaError_t ee = cudaEventRecord(ctx->ev_fork, s);
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(is.side, ctx->ev_fork, 0);
            if (ee != cudaSuccess) return ee;
            on = is.side;
        }
        cudaError_t ee = is.run(igs::KC_SMALL, 0, 0, [&](cudaStream_t st_) { return igs::launch_givens(w, j, st_); }, on);
        if (ee != cudaSuccess) return ee;
        if (is.capture) {
            ee = cudaEventRecord(ctx->ev_join, is.side);
            if (ee != cudaSuccess) return ee;
            pending_join = true;
        }
        return cudaSuccess;
    };

    for (int k = 3; k <= m + 1; ++k) {
        const int p = k - 1;
        // the previous column's Givens kernel (side branch) is complete before this
        // column's step kernel reads its stop decision
        if ((e = join_side()) != cudaSuccess) return e;
        float *wv = col(p - 1);
        // Step 4: z = A w_{k-1} (FP32).
        RUN(igs::KC_SPMV, spmv32b, 2.0 * w.nnz, s, igs::launch_spmv32(w, wv, w.z32, st_));
        // Step 5: [V_{k-2}, w_{k-1}]^T [w_{k-1}, z] (FP32 chunks, FP64 partial sums).
        RUN(igs::KC_DOTS, dots32b(p, 2), 4.0 * w.n * p, s, igs::launch_dots32(w, p, wv, w.z32, st_, &pl));
        // Steps 6-12 (+ step 17 for one iteration), FP64.
        RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_a(w, k, gs, pl, st_));
        if ((e = fork_givens(k - 3)) != cudaSuccess) return e;
        // Steps 7, 11, 13: v_{k-1} = w/gamma in place, u = z/gamma - V_{k-1} r^(1) (FP32).
        float *uout = gs == 1 ? col(p) : w.u32;
        RUN(igs::KC_UPDATE, upd32b(p) + 4.0 * w.n, 2.0 * w.n * p, s,
            igs::launch_update32(w, p, w.r1v, 0.0, w.z32, uout, true, st_));
        if (gs == 2) {
            // Step 14: r^(2) = V_{k-1}^T u.
            RUN(igs::KC_DOTS, dots32b(p, 1), 2.0 * w.n * p, s, igs::launch_dots32(w, p, w.u32, nullptr, st_, &pl));
            // Steps 15, 17.
            RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_b(w, k, pl, st_));
            // Step 16: w_k = u - V_{k-1} r^(3).
            RUN(igs::KC_UPDATE, upd32b(p), 2.0 * w.n * p, s,
                igs::launch_update32(w, p, w.r3v, 1.0, w.u32, col(p), false, st_));
        }
    }
    // Flush: gamma_{m+1} = ||w_{m+1}||, H_{m+1,m}, last L row, v_{m+1} = w_{m+1}/gamma.
    if ((e = join_side()) != cudaSuccess) return e;
    RUN(igs::KC_DOTS, dots32b(m + 1, 1), 2.0 * w.n * (m + 1), s,
        igs::launch_dots32(w, m + 1, col(m), nullptr, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_flush(w, m, pl, st_));
    RUN(igs::KC_CYCLE, 8.0 * w.n, w.n, s, igs::launch_scale32(w, col(m), st_));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_givens(w, m - 1, st_));
    // y = argmin ||rho e1 - H y||; x = x + V y in FP64 (the refinement step).
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_lsq(w, m, st_));
    RUN(igs::KC_CYCLE, 4.0 * w.n * m + 16.0 * w.n, 2.0 * w.n * m, s, igs::launch_xupdate32(w, st_));
    // r = b - A x, ||r||, ||x||, beta(x) in FP64.
    RUN(igs::KC_CYCLE, spmv_bytes(w) + 8.0 * w.n, 2.0 * w.nnz, s, igs::launch_spmv(w, w.x, w.r, w.b, false, st_));
    int nblk = 0;
    RUN(igs::KC_CYCLE, 16.0 * w.n, 4.0 * w.n, s, igs::launch_norms(w, w.r, w.x, nullptr, &nblk, st_));
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_beta(w, nblk, st_));
#undef RUN
    return cudaSuccess;
}

// One cycle of Alg. 4.2 (one-reduce hybrid MGS-CGS GMRES; the readings are the oracle's).
// Per column: the SpMV on u_{k-1} (held in V[:, nb]), the one reduction [V_nb, u]^T [u, A u]
// (the step-5 multi-dot), the single-block step (the lagged norm and Stephen's trick for
// r^(1); its prologue completes the previous column: r^(3), H, L, q), and one fused pass over
// V_nb forming v_{k-1} and u_k.  The Givens rotation of each completed column runs on a side
// branch as in Alg. 4.1.
cudaError_t enqueue_cycle_1r(igs_ctx *ctx, Issuer &is, int m, bool df)
{
    const igs::Workspace &w = ctx->w;
    const DotsLauncher dots = dots_launcher(w, df);
    cudaStream_t s = is.s;
    const int64_t ld = w.ld;
    double *V = w.V;
    auto col = [&](int c) { return V + (int64_t)c * ld; };
    cudaError_t e;
#define RUN(cls, bytes, flops, on, expr)                                          \
    do {                                                                          \
        e = is.run((cls), (bytes), (flops), [&](cudaStream_t st_) { (void)st_; return (expr); }, (on)); \
        if (e != cudaSuccess) return e;                                           \
    } while (0)
    // Step 1: rho = ||r0||, v1 = r0 / rho.
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_cycle_start(w, 0, st_));
    RUN(igs::KC_CYCLE, 16.0 * w.n, w.n, s, igs::launch_scale(w, w.r, col(0), 0, false, st_));
    // Step 2: w2 = A v1, H11 = v1^T w2, u_2 = w2 - v1 H11 (into V[:, 1]).
    igs::DotsPlan pl{};
    RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, col(0), col(1), nullptr, false, st_));
    RUN(igs::KC_DOTS, dots_bytes(w, 1, 1), 2.0 * w.n, s, dots(w, 1, col(1), nullptr, false, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_prime(w, pl, st_));
    RUN(igs::KC_UPDATE, upd_bytes(w, 1), 2.0 * w.n, s,
        igs::launch_update(w, 1, w.r1v, false, 1.0, col(1), col(1), false, false, false, st_));

    bool pending_join = false;
    auto join_side = [&]() -> cudaError_t {
        if (pending_join && is.capture) {
            cudaError_t ee = cudaStreamWaitEvent(s, ctx->ev_join, 0);
            if (ee != cudaSuccess) return ee;
        }
        pending_join = false;
        return cudaSuccess;
    };
    auto fork_givens = [&](int j) -> cudaError_t {
        cudaStream_t on = s;
        if (is.capture) {
            cudaError_t ee = cudaEventRecord(ctx->ev_fork, s);
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(is.side, ctx->ev_fork, 0);
            if (ee != cudaSuccess) return ee;
            on = is.side;
        }
        cudaError_t ee = is.run(igs::KC_SMALL, 0, 0, [&](cudaStream_t st_) { return igs::launch_givens(w, j, st_); }, on);
        if (ee != cudaSuccess) return ee;
        if (is.capture) {
            ee = cudaEventRecord(ctx->ev_join, is.side);
            if (ee != cudaSuccess) return ee;
            pending_join = true;
        }
        return cudaSuccess;
    };
    for (int k = 3; k <= m + 1; ++k) {
        const int nb = k - 2;
        // the previous column's Givens kernel (side branch) is complete before this
        // column's step kernel reads its stop decision
        if ((e = join_side()) != cudaSuccess) return e;
        double *u = col(nb);
        // Step 4: A u_{k-1}, then the one reduction [V_nb, u]^T [u, A u].
        RUN(igs::KC_SPMV, spmv_bytes(w), 2.0 * w.nnz, s, igs::launch_spmv(w, u, w.z, nullptr, true, st_));
        RUN(igs::KC_DOTS, dots_bytes(w, nb + 1, 2), 4.0 * w.n * (nb + 1), s,
            dots(w, nb + 1, u, w.z, true, st_, &pl));
        // Steps 5, 9, 14, 15 of the previous iteration (column nb-2 complete; in the launch's
        // prologue) and steps 6-8, 12 of this one; column nb-2's Givens rotation on the side.
        RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_1r(w, nb, false, pl, st_));
        if (nb >= 2 && (e = fork_givens(nb - 2)) != cudaSuccess) return e;
        // Steps 10-11, 13: v_{k-1} and u_k in one pass.
        RUN(igs::KC_UPDATE, 8.0 * w.n * (nb + 4), 4.0 * w.n * nb, s, igs::launch_update_1r(w, nb, w.z, false, st_));
    }
    // Flush: the reduction of u_{m+1} (no product), columns m-2 and m-1 complete, v_{m+1}.
    if ((e = join_side()) != cudaSuccess) return e;
    RUN(igs::KC_DOTS, dots_bytes(w, m + 1, 1), 2.0 * w.n * (m + 1), s,
        dots(w, m + 1, col(m), nullptr, true, st_, &pl));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_step_1r(w, m, true, pl, st_));
    RUN(igs::KC_UPDATE, 8.0 * w.n * (m + 2), 2.0 * w.n * m, s, igs::launch_update_1r(w, m, w.z, true, st_));
    if (m >= 2) RUN(igs::KC_SMALL, 0, 0, s, igs::launch_givens(w, m - 2, st_));
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_givens(w, m - 1, st_));
    // Least squares y = argmin ||rho e1 - H y||, x_m = x_0 + V_m y_m.
    RUN(igs::KC_SMALL, 0, 0, s, igs::launch_lsq(w, m, st_));
    RUN(igs::KC_CYCLE, upd_bytes(w, m), 2.0 * w.n * m, s,
        igs::launch_update(w, 0, w.y, true, 1.0, w.x, w.x, false, true, false, st_));
    // r = b - A x, ||r||, ||x||, beta(x).
    RUN(igs::KC_CYCLE, spmv_bytes(w) + 8.0 * w.n, 2.0 * w.nnz, s, igs::launch_spmv(w, w.x, w.r, w.b, false, st_));
    int nblk = 0;
    RUN(igs::KC_CYCLE, 16.0 * w.n, 4.0 * w.n, s, igs::launch_norms(w, w.r, w.x, nullptr, &nblk, st_));
    RUN(igs::KC_CYCLE, 0, 0, s, igs::launch_beta(w, nblk, st_));
#undef RUN
    return cudaSuccess;
}

// Solve-level set-up: state, ||b||, r = b - A x, beta(x).  b and x are already in w.b, w.x.
cudaError_t enqueue_setup(igs_ctx *ctx, Issuer &is, double tol, double inner_tol)
{
    const igs::Workspace &w = ctx->w;
    cudaError_t e;
    int nblk = 0;
    e = is.run(igs::KC_CYCLE, 0, 0, [&](cudaStream_t s) { return igs::launch_init_state(w, tol, ctx->normA, inner_tol, s); }, is.s);
    if (e != cudaSuccess) return e;
    e = is.run(igs::KC_CYCLE, 8.0 * w.n, 2.0 * w.n, [&](cudaStream_t s) { return igs::launch_norms(w, w.b, nullptr, nullptr, &nblk, s); }, is.s);
    if (e != cudaSuccess) return e;
    e = is.run(igs::KC_CYCLE, 0, 0, [&](cudaStream_t s) { return igs::launch_bnorm(w, nblk, s); }, is.s);
    if (e != cudaSuccess) return e;
    e = is.run(igs::KC_CYCLE, spmv_bytes(w), 2.0 * w.nnz, [&](cudaStream_t s) { return igs::launch_spmv(w, w.x, w.r, w.b, false, s); }, is.s);
    if (e != cudaSuccess) return e;
    e = is.run(igs::KC_CYCLE, 16.0 * w.n, 4.0 * w.n, [&](cudaStream_t s) { return igs::launch_norms(w, w.r, w.x, nullptr, &nblk, s); }, is.s);
    if (e != cudaSuccess) return e;
    return is.run(igs::KC_CYCLE, 0, 0, [&](cudaStream_t s) { return igs::launch_beta(w, nblk, s); }, is.s);
}

int get_graph(igs_ctx *ctx, int m, int gs, int prec, igs_ctx::Graph **out)
{
    auto key = std::make_pair(m, gs + 4 * prec);
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
        *out = &it->second;
        return IGS_OK;
    }
    Issuer is{ctx, ctx->cap, ctx->side, true};
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_cycle(ctx, is, m, gs, prec);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(ctx, IGS_ECUDA, "capturing the cycle failed: %s", cudaGetErrorString(e));
    }
    if (e2 != cudaSuccess) return fail(ctx, IGS_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
    igs_ctx::Graph gr;
    e = cudaGraphInstantiate(&gr.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, IGS_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    gr.kernels = is.kernels;
    auto res = ctx->graphs.emplace(key, gr);
    *out = &res.first->second;
    return IGS_OK;
}

// Run one cycle: replay the graph, or issue eagerly with events when profiling.
int run_cycle(igs_ctx *ctx, int m, int gs, int prec)
{
    if (ctx->profiling) {
        Issuer is{ctx, ctx->stream, ctx->stream, false};
        cudaError_t e = enqueue_cycle(ctx, is, m, gs, prec);
        ctx->launches += is.kernels;
        CK(e);
        CK(cudaStreamSynchronize(ctx->stream));
        is.collect();
        return IGS_OK;
    }
    igs_ctx::Graph *g = nullptr;
    int rc = get_graph(ctx, m, gs, prec, &g);
    if (rc != IGS_OK) return rc;
    CK(cudaGraphLaunch(g->exec, ctx->stream));
    ctx->launches += g->kernels;
    return IGS_OK;
}

int run_setup(igs_ctx *ctx, double tol, double inner_tol)
{
    Issuer is{ctx, ctx->stream, ctx->stream, false};
    cudaError_t e = enqueue_setup(ctx, is, tol, inner_tol);
    ctx->launches += is.kernels;
    CK(e);
    if (ctx->profiling) {
        CK(cudaStreamSynchronize(ctx->stream));
        is.collect();
    }
    return IGS_OK;
}

int copy_vec_in(igs_ctx *ctx, double *dst, const double *src, bool on_device)
{
    const size_t bytes = sizeof(double) * (size_t)ctx->w.n;
    if (!src) {
        CK(cudaMemsetAsync(dst, 0, bytes, ctx->stream));
        return IGS_OK;
    }
    CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
    return IGS_OK;
}

int read_state(igs_ctx *ctx, igs::DevState *hs)
{
    CK(cudaMemcpyAsync(hs, ctx->w.st, sizeof(igs::DevState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return IGS_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

const char *igs_status_string(int status)
{
    switch (status) {
    case IGS_OK: return "converged";
    case IGS_NOT_CONVERGED: return "not converged (maximum number of restarts reached)";
    case IGS_BREAKDOWN: return "breakdown (invariant Krylov subspace; x is valid)";
    case IGS_EINVAL: return "invalid argument";
    case IGS_ENOMEM: return "out of memory";
    case IGS_ECUDA: return "CUDA error";
    case IGS_ENUMERIC: return "non-finite value met";
    case IGS_ETIMEOUT: return "device wait timed out";
    case IGS_ENOTIMPL: return "not implemented";
    default: return "unknown status";
    }
}

const char *igs_last_error(const igs_ctx *ctx)
{
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

void igs_destroy(igs_ctx *ctx)
{
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (ctx->stream_alloc && ctx->stream) {
        for (void *p : ctx->allocs) cudaFreeAsync(p, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    } else {
        for (void *p : ctx->allocs) cudaFree(p);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    cudaSetDevice(cur);
    delete ctx;
}

int igs_create(igs_ctx **out, int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
               const double *vals, const igs_create_opts *opts)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            igs_ctx *ctx = nullptr;
            if (!out) return fail(nullptr, IGS_EINVAL, "out is NULL");
            *out = nullptr;
            if (!rowptr || (nnz > 0 && (!colind || !vals))) return fail(nullptr, IGS_EINVAL, "null CSR array");
            if (n < 1 || nnz < 0 || nnz >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31))
                return fail(nullptr, IGS_EINVAL, "bad sizes n=%lld nnz=%lld", (long long)n, (long long)nnz);
            if (rowptr[0] != 0 || rowptr[n] != nnz) return fail(nullptr, IGS_EINVAL, "rowptr[0] must be 0 and rowptr[n] = nnz");
            for (int64_t i = 0; i < n; ++i)
                if (rowptr[i + 1] < rowptr[i]) return fail(nullptr, IGS_EINVAL, "rowptr decreases at row %lld", (long long)i);
            for (int64_t q = 0; q < nnz; ++q) {
                if (colind[q] < 0 || colind[q] >= n) return fail(nullptr, IGS_EINVAL, "column index out of range at %lld", (long long)q);
                if (!std::isfinite(vals[q])) return fail(nullptr, IGS_ENUMERIC, "non-finite matrix value at %lld", (long long)q);
            }
            igs_create_opts o{};
            o.device = -1;
            o.max_restart_m = 100;
            if (opts) o = *opts;
            if (o.max_restart_m <= 0) o.max_restart_m = 100;
            if (o.max_restart_m > igs::kMaxRestart)
                return fail(nullptr, IGS_EINVAL, "max_restart_m %d exceeds %d", o.max_restart_m, igs::kMaxRestart);
            if (o.norm2_iters <= 0) o.norm2_iters = 100;

            ctx = new igs_ctx();
            int rc = IGS_OK;
            auto bail = [&](int code) {
                if (!ctx->err.empty()) g_create_err = ctx->err;
                igs_destroy(ctx);
                return code;
            };
            {
                int dev = o.device;
                if (dev < 0) {
                    if (cudaGetDevice(&dev) != cudaSuccess) {
                        ctx->err = "no CUDA device";
                        return bail(IGS_ECUDA);
                    }
                }
                ctx->device = dev;
                cudaError_t e = cudaSetDevice(dev);
                if (e != cudaSuccess) {
                    fail(ctx, IGS_ECUDA, "cudaSetDevice(%d): %s", dev, cudaGetErrorString(e));
                    return bail(IGS_ECUDA);
                }
                int sms = 0;
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                ctx->w.num_sms = sms > 0 ? sms : 1;
            }
            if (o.stream) {
                ctx->stream = (cudaStream_t)o.stream;
            } else {
                if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
                    ctx->err = "cudaStreamCreate failed";
                    return bail(IGS_ECUDA);
                }
                ctx->own_stream = true;
            }
            ctx->stream_alloc = o.stream_alloc != 0;
            if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
                ctx->err = "stream/event creation failed";
                return bail(IGS_ECUDA);
            }
            igs::Workspace &w = ctx->w;
            w.n = n;
            w.nnz = nnz;
            w.ld = (n + 31) & ~int64_t(31);
            w.mmax = o.max_restart_m;
            w.spmv_warp_rows = nnz >= 16 * n;
            const int M = w.mmax;
            int *rp = nullptr, *ci = nullptr;
            double *va = nullptr;
            if ((rc = dalloc(ctx, &rp, (size_t)n + 1)) || (rc = dalloc(ctx, &ci, (size_t)nnz)) ||
                (rc = dalloc(ctx, &va, (size_t)nnz)) || (rc = dalloc(ctx, &w.V, (size_t)w.ld * (M + 1))) ||
                (rc = dalloc(ctx, &w.z, (size_t)w.ld)) || (rc = dalloc(ctx, &w.u, (size_t)w.ld)) ||
                (rc = dalloc(ctx, &w.r, (size_t)w.ld)) || (rc = dalloc(ctx, &w.b, (size_t)w.ld)) ||
                (rc = dalloc(ctx, &w.x, (size_t)w.ld)) || (rc = dalloc(ctx, &w.t, (size_t)w.ld)) ||
                (rc = dalloc(ctx, &w.H, (size_t)(M + 1) * M)) || (rc = dalloc(ctx, &w.R, (size_t)(M + 1) * M)) ||
                (rc = dalloc(ctx, &w.L, (size_t)(M + 1) * (M + 1))) ||
                (rc = dalloc(ctx, &w.Lrow, (size_t)(M + 1) * M / 2 + 2)) ||
                (rc = dalloc(ctx, &w.Lout, (size_t)(M + 1) * (M + 1))) || (rc = dalloc(ctx, &w.cs, (size_t)M)) ||
                (rc = dalloc(ctx, &w.sn, (size_t)M)) || (rc = dalloc(ctx, &w.g, (size_t)M + 1)) ||
                (rc = dalloc(ctx, &w.lfro2, (size_t)M + 1)) ||
                (rc = dalloc(ctx, &w.r1v, (size_t)M + 1)) || (rc = dalloc(ctx, &w.r2v, (size_t)M + 1)) ||
                (rc = dalloc(ctx, &w.r3v, (size_t)M + 1)) || (rc = dalloc(ctx, &w.y, (size_t)M + 1)) ||
                (rc = dalloc(ctx, &w.hist_res, (size_t)M)) || (rc = dalloc(ctx, &w.hist_lfro, (size_t)M)) ||
                (rc = dalloc(ctx, &w.st, 1)))
                return bail(rc);
            // partial-sum buffer: largest multi-dot launch (two vectors, up to m+1 columns) or norms
            int64_t cap = 3 * (int64_t)w.num_sms;
            for (int p = 1; p <= M + 1; ++p) {
                const igs::DotsPlan pl = igs::plan_dots(w, p);
                const int64_t need = 2 * (int64_t)p * pl.rblocks;
                if (need > cap) cap = need;
            }
            if ((rc = dalloc(ctx, &w.part, (size_t)cap))) return bail(rc);
            w.part_cap = cap;
            // host -> device copies; with pooled memory they follow the allocations on the stream
            auto upload = [&](void *dst, const void *src, size_t bytes) {
                if (!ctx->stream_alloc) return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
                cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
                return e == cudaSuccess ? cudaStreamSynchronize(ctx->stream) : e;
            };
            {
                std::vector<int> rp32((size_t)n + 1);
                for (int64_t i = 0; i <= n; ++i) rp32[(size_t)i] = (int)rowptr[i];
                cudaError_t e = upload(rp, rp32.data(), sizeof(int) * rp32.size());
                if (e == cudaSuccess && nnz > 0) e = upload(ci, colind, sizeof(int) * (size_t)nnz);
                if (e == cudaSuccess && nnz > 0) e = upload(va, vals, sizeof(double) * (size_t)nnz);
                if (e != cudaSuccess) {
                    fail(ctx, IGS_ECUDA, "copying A: %s", cudaGetErrorString(e));
                    return bail(IGS_ECUDA);
                }
            }
            w.rowptr = rp;
            w.colind = ci;
            w.val = va;
            if (!w.spmv_warp_rows) {
                // SELL-32 copy of A: the FP64 hot-path SpMV loads columns and values coalesced
                // (the FP32 SpMV of the precision form keeps the CSR thread-per-row kernel: the
                // SELL form of it measured 33 % slower on the 3-D 7-point matrices)
                const int64_t nsl = (n + 31) / 32;
                std::vector<int64_t> soff((size_t)nsl + 1, 0);
                int64_t wall = 0;
                for (int64_t k = 0; k < nsl; ++k) {
                    int64_t wmax = 0;
                    for (int64_t i = 32 * k; i < std::min<int64_t>(n, 32 * k + 32); ++i)
                        wmax = std::max<int64_t>(wmax, rowptr[i + 1] - rowptr[i]);
                    soff[(size_t)k + 1] = soff[(size_t)k] + 32 * wmax;
                    wall = std::max(wall, wmax);
                }
                // ELL (every slice as wide as the widest) when that is narrow and costs little
                // padding: the SpMV then computes slice offsets instead of loading them
                if (wall >= 1 && wall <= igs::kMaxEllWidth &&
                    (double)(32 * wall * nsl) <= igs::kEllMaxPadding * (double)soff[(size_t)nsl]) {
                    for (int64_t k = 0; k <= nsl; ++k) soff[(size_t)k] = 32 * wall * k;
                    w.ell_width = (int)wall;
                }
                const int64_t ne = std::max<int64_t>(soff[(size_t)nsl], 1);
                std::vector<int> scol((size_t)ne, -1);
                std::vector<double> sval((size_t)ne, 0.0);
                for (int64_t i = 0; i < n; ++i)
                    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                        const size_t e = (size_t)(soff[(size_t)(i >> 5)] + 32 * (q - rowptr[i]) + (i & 31));
                        scol[e] = colind[q];
                        sval[e] = vals[q];
                    }
                int64_t *d_off = nullptr;
                int *d_col = nullptr;
                double *d_val = nullptr;
                if ((rc = dalloc(ctx, &d_off, soff.size())) || (rc = dalloc(ctx, &d_col, (size_t)ne)) ||
                    (rc = dalloc(ctx, &d_val, (size_t)ne)))
                    return bail(rc);
                cudaError_t e = upload(d_off, soff.data(), sizeof(int64_t) * soff.size());
                if (e == cudaSuccess) e = upload(d_col, scol.data(), sizeof(int) * scol.size());
                if (e == cudaSuccess) e = upload(d_val, sval.data(), sizeof(double) * sval.size());
                if (e != cudaSuccess) {
                    fail(ctx, IGS_ECUDA, "copying A (SELL-32): %s", cudaGetErrorString(e));
                    return bail(IGS_ECUDA);
                }
                w.sell_off = d_off;
                w.sell_col = d_col;
                w.sell_val = d_val;
            }
            if (o.fp32_basis) {
                // precision form: FP32 basis, Krylov vectors and A's values (rounded to nearest)
                if ((rc = dalloc(ctx, &w.V32, (size_t)w.ld * (M + 1))) || (rc = dalloc(ctx, &w.z32, (size_t)w.ld)) ||
                    (rc = dalloc(ctx, &w.u32, (size_t)w.ld)) || (rc = dalloc(ctx, &w.val32, (size_t)nnz)))
                    return bail(rc);
                std::vector<float> v32((size_t)(nnz > 0 ? nnz : 1));
                for (int64_t q = 0; q < nnz; ++q) v32[(size_t)q] = (float)vals[q];
                cudaError_t e = nnz > 0 ? upload(w.val32, v32.data(), sizeof(float) * (size_t)nnz) : cudaSuccess;
                if (e != cudaSuccess) {
                    fail(ctx, IGS_ECUDA, "copying A (FP32): %s", cudaGetErrorString(e));
                    return bail(IGS_ECUDA);
                }
            }
            {
                cudaError_t e = igs::configure_kernels(w);
                if (e == cudaSuccess) e = igs::configure_df_kernels();
                if (e != cudaSuccess) {
                    fail(ctx, IGS_ECUDA, "kernel configuration: %s", cudaGetErrorString(e));
                    return bail(IGS_ECUDA);
                }
            }
            if (o.A_norm2 > 0.0) {
                ctx->normA = o.A_norm2;
            } else {
                // A^T in CSR (counting sort), uploaded for the power iteration only.
                std::vector<int> trp((size_t)n + 1, 0), tci((size_t)nnz);
                std::vector<double> tva((size_t)nnz);
                for (int64_t q = 0; q < nnz; ++q) trp[(size_t)colind[q] + 1]++;
                for (int64_t i = 0; i < n; ++i) trp[(size_t)i + 1] += trp[(size_t)i];
                std::vector<int> pos(trp.begin(), trp.end() - 1);
                for (int64_t i = 0; i < n; ++i)
                    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                        const int c = colind[q];
                        tci[(size_t)pos[(size_t)c]] = (int)i;
                        tva[(size_t)pos[(size_t)c]++] = vals[q];
                    }
                // scratch from the stream-ordered pool when the context's memory is (so that
                // neither allocating nor freeing it waits for other streams' work)
                const bool pooled = ctx->stream_alloc;
                auto salloc = [&](void **q, size_t bytes) {
                    return pooled ? cudaMallocAsync(q, bytes, ctx->stream) : cudaMalloc(q, bytes);
                };
                auto sfree = [&](void *q) {
                    if (q) pooled ? cudaFreeAsync(q, ctx->stream) : cudaFree(q);
                };
                auto up = [&](void *dst, const void *src, size_t bytes) {
                    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
                };
                int *d_trp = nullptr, *d_tci = nullptr;
                double *d_tva = nullptr;
                cudaError_t e = salloc((void **)&d_trp, sizeof(int) * (n + 1));
                if (e == cudaSuccess) e = salloc((void **)&d_tci, sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
                if (e == cudaSuccess) e = salloc((void **)&d_tva, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
                if (e == cudaSuccess) e = up(d_trp, trp.data(), sizeof(int) * (n + 1));
                if (e == cudaSuccess && nnz > 0) e = up(d_tci, tci.data(), sizeof(int) * (size_t)nnz);
                if (e == cudaSuccess && nnz > 0) e = up(d_tva, tva.data(), sizeof(double) * (size_t)nnz);
                double est = 0.0;
                // (synchronises the stream before returning, so the host copies above are done)
                if (e == cudaSuccess) e = igs::estimate_norm2(w, d_trp, d_tci, d_tva, o.norm2_iters, &est, ctx->stream);
                if (e != cudaSuccess) cudaStreamSynchronize(ctx->stream);
                sfree(d_trp);
                sfree(d_tci);
                sfree(d_tva);
                if (e != cudaSuccess) {
                    fail(ctx, IGS_ECUDA, "norm estimate: %s", cudaGetErrorString(e));
                    return bail(IGS_ECUDA);
                }
                ctx->normA = est;
                ctx->normA_est = 1;
            }
            if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
                ctx->err = "create: stream sync failed";
                return bail(IGS_ECUDA);
            }
            *out = ctx;
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

int igs_get_info(const igs_ctx *ctx, igs_info *info)
{
    if (!ctx || !info) return IGS_EINVAL;
    info->n = ctx->w.n;
    info->nnz = ctx->w.nnz;
    info->max_restart_m = ctx->w.mmax;
    info->device = ctx->device;
    info->A_norm2 = ctx->normA;
    info->A_norm2_estimated = ctx->normA_est;
    info->device_bytes = ctx->device_bytes;
    return IGS_OK;
}

int igs_profile_enable(igs_ctx *ctx, int enable)
{
    if (!ctx) return IGS_EINVAL;
    ctx->profiling = enable != 0;
    if (enable) ctx->prof = igs_profile{};
    return IGS_OK;
}

int igs_profile_get(igs_ctx *ctx, igs_profile *out)
{
    if (!ctx || !out) return IGS_EINVAL;
    *out = ctx->prof;
    return IGS_OK;
}

int64_t igs_launch_count(const igs_ctx *ctx) { return ctx ? ctx->launches : -1; }

int igs_spmv(igs_ctx *ctx, const double *x, double *y, int on_device)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!ctx || !x || !y) return IGS_EINVAL;
            CK(cudaSetDevice(ctx->device));
            igs::Workspace &w = ctx->w;
            const size_t bytes = sizeof(double) * (size_t)w.n;
            const double *xd = x;
            double *yd = y;
            if (!on_device) {
                CK(cudaMemcpyAsync(w.t, x, bytes, cudaMemcpyHostToDevice, ctx->stream));
                xd = w.t;
                yd = w.z;
            }
            CK(igs::launch_spmv(w, xd, yd, nullptr, false, ctx->stream));
            ctx->launches += 1;
            if (!on_device) CK(cudaMemcpyAsync(y, w.z, bytes, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

int igs_solve(igs_ctx *ctx, const double *b, const double *x0, const igs_solve_opts *opts, igs_result *res)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!ctx || !b || !opts || !res || !res->x) return ctx ? fail(ctx, IGS_EINVAL, "null argument") : IGS_EINVAL;
            const int m = opts->restart_m;
            const int method = opts->method == 0 ? IGS_METHOD_IGS : opts->method;
            if (method != IGS_METHOD_IGS && method != IGS_METHOD_ONE_REDUCE) return fail(ctx, IGS_EINVAL, "unknown method");
            if (m < 1 || m > ctx->w.mmax) return fail(ctx, IGS_EINVAL, "restart_m %d outside [1, %d]", m, ctx->w.mmax);
            if (method == IGS_METHOD_IGS && opts->gs_iters != 1 && opts->gs_iters != 2)
                return fail(ctx, IGS_EINVAL, "gs_iters must be 1 or 2");
            if (method == IGS_METHOD_ONE_REDUCE && opts->precision == IGS_PREC_FP32_IR)
                return fail(ctx, IGS_EINVAL, "the one-reduce method runs in FP64 (or FP64_DF) only");
            const int gs = method == IGS_METHOD_ONE_REDUCE ? 0 : opts->gs_iters;  // 0: Alg. 4.2 cycle
            if (opts->max_restarts < 1) return fail(ctx, IGS_EINVAL, "max_restarts must be >= 1");
            if (!(opts->tol_beta >= 0.0)) return fail(ctx, IGS_EINVAL, "tol_beta must be >= 0");
            if (res->H && res->H_ld < m + 1) return fail(ctx, IGS_EINVAL, "H_ld < m+1");
            const int prec = opts->precision;
            if (prec != IGS_PREC_FP64 && prec != IGS_PREC_FP32_IR && prec != IGS_PREC_FP64_DF)
                return fail(ctx, IGS_EINVAL, "unknown precision %d", prec);
            if (prec == IGS_PREC_FP32_IR && !ctx->w.V32)
                return fail(ctx, IGS_EINVAL, "precision FP32_IR needs a context created with fp32_basis");
            const double inner_tol = prec == IGS_PREC_FP32_IR ? (opts->inner_tol > 0.0 ? opts->inner_tol : 1e-6) : 0.0;
            CK(cudaSetDevice(ctx->device));
            igs::Workspace &w = ctx->w;
            const bool dev = opts->inputs_on_device != 0;
            int rc;
            if ((rc = copy_vec_in(ctx, w.b, b, dev)) != IGS_OK) return rc;
            if ((rc = copy_vec_in(ctx, w.x, x0, dev)) != IGS_OK) return rc;
            if ((rc = run_setup(ctx, opts->tol_beta, inner_tol)) != IGS_OK) return rc;
            igs::DevState hs{};
            if ((rc = read_state(ctx, &hs)) != IGS_OK) return rc;
            res->hist_len = 0;
            res->steps = 0;
            res->cycles = 0;
            res->rho0 = hs.rnorm;
            int status = IGS_NOT_CONVERGED;
            std::vector<double> hres((size_t)m), hlf((size_t)m);
            if (!std::isfinite(hs.beta)) {
                status = IGS_ENUMERIC;
            } else if (hs.beta <= opts->tol_beta) {
                status = IGS_OK;
            } else {
                for (int cyc = 0; cyc < opts->max_restarts; ++cyc) {
                    if ((rc = run_cycle(ctx, m, gs, prec)) != IGS_OK) return rc;
                    if ((rc = read_state(ctx, &hs)) != IGS_OK) return rc;
                    res->cycles += 1;
                    const int nc = hs.ncols;
                    res->steps += nc;
                    if ((res->arnoldi_hist || res->lfro_hist) && nc > 0) {
                        CK(cudaMemcpyAsync(hres.data(), w.hist_res, sizeof(double) * nc, cudaMemcpyDeviceToHost, ctx->stream));
                        CK(cudaMemcpyAsync(hlf.data(), w.hist_lfro, sizeof(double) * nc, cudaMemcpyDeviceToHost, ctx->stream));
                        CK(cudaStreamSynchronize(ctx->stream));
                        for (int j = 0; j < nc && res->hist_len < res->hist_cap; ++j) {
                            if (res->arnoldi_hist) res->arnoldi_hist[res->hist_len] = hres[(size_t)j];
                            if (res->lfro_hist) res->lfro_hist[res->hist_len] = hlf[(size_t)j];
                            res->hist_len++;
                        }
                    }
                    if (hs.stop_reason < 0 || !std::isfinite(hs.beta)) {
                        status = IGS_ENUMERIC;
                        break;
                    }
                    if (hs.beta <= opts->tol_beta) {
                        status = IGS_OK;
                        break;
                    }
                    if (hs.stop_reason == 2) {
                        status = IGS_BREAKDOWN;
                        break;
                    }
                }
            }
            const size_t bytes = sizeof(double) * (size_t)w.n;
            CK(cudaMemcpyAsync(res->x, w.x, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
            if (res->H && res->cycles > 0)
                CK(cudaMemcpy2DAsync(res->H, sizeof(double) * res->H_ld, w.H, sizeof(double) * w.ldh(),
                                     sizeof(double) * (m + 1), m, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            res->beta = hs.beta;
            return status;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

int igs_arnoldi(igs_ctx *ctx, const double *r0, int m, int gs, int on_device, double *V, int64_t ldv,
                double *H, double *L, int *ncols, double *rho)
{
    return igs_arnoldi_ex(ctx, r0, m, IGS_METHOD_IGS, gs, IGS_PREC_FP64, on_device, V, ldv, H, L, ncols, rho);
}

int igs_arnoldi_ex(igs_ctx *ctx, const double *r0, int m, int method, int gs, int precision, int on_device,
                   double *V, int64_t ldv, double *H, double *L, int *ncols, double *rho)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!ctx || !r0) return ctx ? fail(ctx, IGS_EINVAL, "null argument") : IGS_EINVAL;
            if (m < 1 || m > ctx->w.mmax) return fail(ctx, IGS_EINVAL, "m %d outside [1, %d]", m, ctx->w.mmax);
            if (method != IGS_METHOD_IGS && method != IGS_METHOD_ONE_REDUCE) return fail(ctx, IGS_EINVAL, "unknown method");
            if (method == IGS_METHOD_IGS && gs != 1 && gs != 2) return fail(ctx, IGS_EINVAL, "gs_iters must be 1 or 2");
            if (method == IGS_METHOD_ONE_REDUCE) gs = 0;  // the Alg. 4.2 cycle
            if (precision != IGS_PREC_FP64 && precision != IGS_PREC_FP64_DF)
                return fail(ctx, IGS_EINVAL, "igs_arnoldi_ex runs FP64 or FP64_DF cycles only");
            if (V && ldv < ctx->w.n) return fail(ctx, IGS_EINVAL, "ldv < n");
            CK(cudaSetDevice(ctx->device));
            igs::Workspace &w = ctx->w;
            const int M = w.mmax;
            CK(cudaMemsetAsync(w.H, 0, sizeof(double) * (size_t)(M + 1) * M, ctx->stream));
            CK(cudaMemsetAsync(w.L, 0, sizeof(double) * (size_t)(M + 1) * (M + 1), ctx->stream));
            CK(cudaMemsetAsync(w.V, 0, sizeof(double) * (size_t)w.ld * (M + 1), ctx->stream));
            int rc;
            if ((rc = copy_vec_in(ctx, w.b, r0, on_device != 0)) != IGS_OK) return rc;
            if ((rc = copy_vec_in(ctx, w.x, nullptr, false)) != IGS_OK) return rc;
            if ((rc = run_setup(ctx, 0.0, 0.0)) != IGS_OK) return rc;
            if ((rc = run_cycle(ctx, m, gs, precision)) != IGS_OK) return rc;
            igs::DevState hs{};
            if ((rc = read_state(ctx, &hs)) != IGS_OK) return rc;
            const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            if (V && precision == IGS_PREC_FP64_DF && igs::dots_df_applies(w)) {
                // the double-float cycles keep the basis split: hand it out in FP64
                CK(igs::launch_df_to_f64(w.V, w.ld * (int64_t)(m + 1), w.num_sms, ctx->stream));
                ctx->launches += 1;
            }
            if (V)
                CK(cudaMemcpy2DAsync(V, sizeof(double) * ldv, w.V, sizeof(double) * w.ld, sizeof(double) * w.n,
                                     m + 1, kind, ctx->stream));
            if (H)
                CK(cudaMemcpy2DAsync(H, sizeof(double) * (m + 1), w.H, sizeof(double) * w.ldh(),
                                     sizeof(double) * (m + 1), m, kind, ctx->stream));
            if (L) {
                // the device keeps L column-major; hand it out row-major
                double *dst = on_device ? L : w.Lout;
                CK(igs::launch_transpose(w.L, w.ldl(), m + 1, m + 1, dst, m + 1, ctx->stream));
                ctx->launches += 1;
                if (!on_device)
                    CK(cudaMemcpyAsync(L, w.Lout, sizeof(double) * (size_t)(m + 1) * (m + 1),
                                       cudaMemcpyDeviceToHost, ctx->stream));
            }
            CK(cudaStreamSynchronize(ctx->stream));
            if (ncols) *ncols = hs.ncols;
            if (rho) *rho = hs.rho;
            if (hs.stop_reason < 0) return IGS_ENUMERIC;
            return hs.stop_reason == 2 ? IGS_BREAKDOWN : IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

}  // extern "C"
