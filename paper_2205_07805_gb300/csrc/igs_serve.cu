// Request server (include/igs_serve.h): continuous batching of IGS-GMRES solves on one GPU.
//
// Device side: one cooperative launch per request, a gang of G CTAs running the device solver
// of igs_sysdev.cuh (FP64 basis, or FP32 basis inside FP64 refinement) over the whole solve.
// Host side (native runtime): an arena allocator over one device allocation (admission by
// the bytes a request needs), a pool of launch slots (one stream and event each), FIFO
// admission, completion detection by event queries, and result collection.
#include "../../include/igs.h"
#include "../../include/igs_serve.h"
#include "igs_internal.h"
#include "igs_sysdev.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <condition_variable>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace igs {
namespace serve {

constexpr int kThreads = 256;  // threads per CTA of a request's gang

template <typename T>
struct ServeArgs {
    sysdev::SysArgs<T> sys;
    sysdev::GangSync *sync;
    double *gpart;     // 2 x G x gld exchange buffer
    int gld;
    double *Rbase;     // G x rstride: each CTA's Givens factor
    int64_t rstride;
    int chunk;         // rows per CTA (multiple of 32)
    int n2;            // n rounded up to even
};

// One request's solve by a gang of gridDim.x CTAs (all co-resident: cooperative launch).
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_serve_solve(ServeArgs<T> a)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ sysdev::Shared sh;
    if (threadIdx.x == 0) sysdev::init_shared(sh);
    __syncthreads();
    const sysdev::SmemLayout L = sysdev::smem_layout<T>(a.chunk, a.sys.m);
    sysdev::Gang gg;
    gg.G = gridDim.x;
    gg.g = blockIdx.x;
    gg.lo = min(a.n2, (int)blockIdx.x * a.chunk);
    gg.hi = min(a.n2, gg.lo + a.chunk);
    gg.sync = a.sync;
    gg.gpart = a.gpart;
    gg.gld = a.gld;
    gg.R = a.Rbase + (int64_t)blockIdx.x * a.rstride;
    sysdev::d_solve<T>(a.sys, gg, sm, L, sh);
}

// Four gang barriers of the solver (igs_server_gang_selftest); ok[g] = 1 if CTA g passed
// them all, 0 if its bounded wait gave up or saw another CTA's abort.
__global__ void __launch_bounds__(kThreads) k_gang_selftest(sysdev::GangSync *sync, int *ok)
{
    __shared__ sysdev::Shared sh;
    if (threadIdx.x == 0) sysdev::init_shared(sh);
    __syncthreads();
    sysdev::Gang gg{};
    gg.G = gridDim.x;
    gg.g = blockIdx.x;
    gg.sync = sync;
    bool pass = true;
    for (int r = 0; r < 4 && pass; ++r) pass = sysdev::gang_barrier(gg, sh);
    if (threadIdx.x == 0) ok[blockIdx.x] = pass ? 1 : 0;
}

// First-fit allocator over [0, size) with coalescing free ranges (256-byte granules).
class Arena {
public:
    void init(int64_t size)
    {
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(int64_t bytes, int64_t *off)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const int64_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest > 0) free_[at] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(int64_t off, int64_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t size() const { return size_; }
    int64_t used() const { return used_; }
    int64_t peak() const { return peak_; }

private:
    int64_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<int64_t, int64_t> free_;
};

// Device result block of a request.
struct ResultBlock {
    double beta;
    int64_t steps;
    int status;
    int cycles;
};

// A request on the graph lane: its own copies of the inputs, and the results the worker
// thread writes (only the worker touches a job between hand-over and completion).
struct GraphJob {
    int64_t id = 0;
    igs_request opt{};
    double normA = 0.0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colind;
    std::vector<double> vals, b, x0, x;
    int status = IGS_OK;
    double beta = 0.0;
    int64_t steps = 0, device_bytes = 0;
    int cycles = 0;
};

// A gang request whose ||A||_2 the server estimates (no A_norm2 given): a copy of its CSR
// matrix for the norm worker, and the estimate it hands back.
struct NormJob {
    int64_t id = 0, n = 0, nnz = 0;
    int device = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colind;
    std::vector<double> vals;
    double normA = 0.0;
    int status = IGS_OK;
};

struct Request {
    int64_t id = 0;
    bool graph = false;  // runs on the graph lane (whole-GPU kernels, one request at a time)
    std::unique_ptr<GraphJob> job;
    igs_request opt{};
    int n = 0, n2 = 0, ldv = 0, G = 1, chunk = 32, nslices = 0;
    bool f32 = false, has_x0 = false;
    double normA = 0.0;
    // host copies until admission
    std::vector<int64_t> sell_off;
    std::vector<int> sell_col;
    std::vector<double> sell_val;
    std::vector<float> sell_val32;
    std::vector<double> b, x0;
    // device layout (offsets in the arena)
    int64_t arena_off = -1, bytes = 0;
    struct Off {
        int64_t off, col, val, val32, b, x0, x, V, r64, R, gpart, sync, res;
    } o{};
    size_t smem = 0;
    int slot = -1;
    std::vector<double> x_host;
    ResultBlock res{};
    int status = IGS_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    bool done = false, polled = false;
    bool norm_pending = false;  // waiting for the norm worker's ||A||_2 estimate
};

}  // namespace serve
}  // namespace igs

using igs::serve::Request;

struct igs_server {
    int device = 0, num_sms = 1, max_m = 0, slots = 8, rows_per_cta = 4096, max_queue = 0;
    char *arena_base = nullptr;
    igs::serve::Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<int64_t> slot_req;  // request id on each slot, -1 free
    std::unordered_map<int64_t, Request> reqs;
    std::deque<int64_t> queue;
    std::deque<int64_t> completions;
    int64_t next_id = 1, submitted = 0, completed = 0, launches = 0;
    int max_gang[2] = {1, 1};       // largest co-resident gang (FP64, FP32 kernels)
    int cta_budget = 1;             // CTAs of all running gangs at most (all co-resident at once)
    int running_ctas = 0;
    // graph lanes: requests with n >= graph_min_n, each solved by a worker thread of its lane
    // through igs_create/igs_solve (the whole-GPU kernels and CUDA graphs of igs.h); the lanes
    // run concurrently (their streams overlap on the device) and beside the gangs
    struct Lane {
        std::thread thread;
        cudaStream_t stream = nullptr;
        int64_t busy = -1;                                    // request on the lane, -1: idle
        std::unique_ptr<igs::serve::GraphJob> in, out;        // hand-over / finished (under graph_mu)
    };
    // norm worker: ||A||_2 of gang requests that come without one, estimated on the GPU by
    // the library's power iteration (igs_create with A_norm2 = 0) on its own stream
    std::thread norm_thread;
    cudaStream_t norm_stream = nullptr;
    std::deque<std::unique_ptr<igs::serve::NormJob>> norm_in, norm_out;  // under graph_mu
    std::condition_variable norm_cv;
    int64_t graph_min_n = 0;
    std::deque<int64_t> graph_queue;       // waiting for a lane (FIFO)
    std::vector<Lane> lanes;
    std::mutex graph_mu;
    std::condition_variable graph_cv;
    bool graph_stop = false;
    size_t smem_max[2] = {0, 0};
    std::chrono::steady_clock::time_point t0;
    std::string err;
};

namespace {

int sfail(igs_server *s, int code, const std::string &what, cudaError_t e = cudaSuccess)
{
    if (s) {
        s->err = what;
        if (e != cudaSuccess) s->err += std::string(": ") + cudaGetErrorString(e);
    }
    return code;
}

double now_s(const igs_server *s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

template <typename T>
void *kernel_ptr()
{
    return reinterpret_cast<void *>(igs::serve::k_serve_solve<T>);
}

// Device bytes and buffer offsets of a request (relative to its arena block).
int64_t plan_request(Request &r, int gld)
{
    int64_t o = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = o;
        o += (bytes + 255) / 256 * 256;
        return at;
    };
    const int64_t ne = (int64_t)r.sell_col.size();
    const int m = r.opt.restart_m;
    r.o.off = take(sizeof(int64_t) * r.sell_off.size());
    r.o.col = take(sizeof(int) * ne);
    r.o.val = take(sizeof(double) * ne);
    r.o.val32 = r.f32 ? take(sizeof(float) * ne) : -1;
    r.o.b = take(sizeof(double) * r.n);
    r.o.x0 = r.has_x0 ? take(sizeof(double) * r.n) : -1;
    r.o.x = take(sizeof(double) * r.n2);
    r.o.V = take((int64_t)(r.f32 ? sizeof(float) : sizeof(double)) * r.ldv * (m + 1));
    r.o.r64 = r.f32 ? take(sizeof(double) * r.ldv) : -1;
    r.o.R = take(sizeof(double) * (int64_t)r.G * (m * (m + 1) / 2 + 1));
    r.o.gpart = take(sizeof(double) * 2 * (int64_t)r.G * gld);
    r.o.sync = take(sizeof(igs::sysdev::GangSync));
    r.o.res = take(sizeof(igs::serve::ResultBlock));
    return o;
}

template <typename T>
int launch_request(igs_server *s, Request &r, cudaStream_t st)
{
    using namespace igs;
    char *base = s->arena_base + r.arena_off;
    const int m = r.opt.restart_m;
    const int gld = 2 * (m + 1) + 2;
    serve::ServeArgs<T> a;
    sysdev::SysArgs<T> &sa = a.sys;
    sa.n = r.n;
    sa.m = m;
    sa.gs = r.opt.gs_iters;
    sa.max_cycles = r.opt.max_restarts;
    sa.ldv = r.ldv;
    sa.tol = r.opt.tol_beta;
    sa.inner_tol = r.f32 ? (r.opt.inner_tol > 0.0 ? r.opt.inner_tol : 1e-6) : 0.0;
    sa.normA = r.normA;
    sa.sell_off = reinterpret_cast<const int64_t *>(base + r.o.off);
    sa.sell_col = reinterpret_cast<const int *>(base + r.o.col);
    sa.sell_val = reinterpret_cast<const double *>(base + r.o.val);
    sa.sell_val32 = r.f32 ? reinterpret_cast<const float *>(base + r.o.val32) : nullptr;
    sa.b = reinterpret_cast<const double *>(base + r.o.b);
    sa.x0 = r.has_x0 ? reinterpret_cast<const double *>(base + r.o.x0) : nullptr;
    sa.x = reinterpret_cast<double *>(base + r.o.x);
    sa.V = reinterpret_cast<T *>(base + r.o.V);
    sa.r64 = r.f32 ? reinterpret_cast<double *>(base + r.o.r64) : nullptr;
    serve::ResultBlock *rb = reinterpret_cast<serve::ResultBlock *>(base + r.o.res);
    sa.beta_out = &rb->beta;
    sa.status_out = &rb->status;
    sa.steps_out = &rb->steps;
    sa.cycles_out = &rb->cycles;
    a.sync = reinterpret_cast<sysdev::GangSync *>(base + r.o.sync);
    a.gpart = reinterpret_cast<double *>(base + r.o.gpart);
    a.gld = gld;
    a.Rbase = reinterpret_cast<double *>(base + r.o.R);
    a.rstride = m * (m + 1) / 2 + 1;
    a.chunk = r.chunk;
    a.n2 = r.n2;
    // uploads (the host copies are released afterwards)
    cudaError_t e = cudaSuccess;
    auto up = [&](int64_t off, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, st);
    };
    up(r.o.off, r.sell_off.data(), sizeof(int64_t) * r.sell_off.size());
    up(r.o.col, r.sell_col.data(), sizeof(int) * r.sell_col.size());
    up(r.o.val, r.sell_val.data(), sizeof(double) * r.sell_val.size());
    if (r.f32) up(r.o.val32, r.sell_val32.data(), sizeof(float) * r.sell_val32.size());
    up(r.o.b, r.b.data(), sizeof(double) * r.b.size());
    if (r.has_x0) up(r.o.x0, r.x0.data(), sizeof(double) * r.x0.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(base + r.o.sync, 0, sizeof(sysdev::GangSync), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + r.o.res, 0, sizeof(serve::ResultBlock), st);
    if (e != cudaSuccess) return sfail(s, IGS_ECUDA, "request upload", e);
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(kernel_ptr<T>(), dim3(r.G), dim3(serve::kThreads), args, r.smem, st);
    if (e != cudaSuccess) return sfail(s, IGS_ECUDA, "request launch", e);
    return IGS_OK;
}

// One graph-lane request through the single-system library on the lane's stream (pooled
// device memory, so that creating and destroying the context never waits for the gangs).
void run_graph_job(igs_server *s, cudaStream_t stream, igs::serve::GraphJob &j)
{
    const igs_request &q = j.opt;
    j.x.assign((size_t)q.n, 0.0);
    igs_create_opts co{};
    co.stream = stream;
    co.device = s->device;
    co.max_restart_m = q.restart_m;
    co.A_norm2 = j.normA;
    co.fp32_basis = q.precision == IGS_PREC_FP32_IR;
    co.stream_alloc = 1;
    igs_ctx *ctx = nullptr;
    int rc = igs_create(&ctx, q.n, q.nnz, j.rowptr.data(), j.colind.data(), j.vals.data(), &co);
    if (rc != IGS_OK) {
        j.status = rc;
        return;
    }
    igs_info info{};
    if (igs_get_info(ctx, &info) == IGS_OK) {
        j.device_bytes = info.device_bytes;
        j.normA = info.A_norm2;  // the given norm, or the context's GPU estimate
    }
    igs_solve_opts so{};
    so.restart_m = q.restart_m;
    so.gs_iters = q.gs_iters;
    so.tol_beta = q.tol_beta;
    so.max_restarts = q.max_restarts;
    so.inputs_on_device = 0;
    so.precision = q.precision;
    so.inner_tol = q.inner_tol;
    so.method = IGS_METHOD_IGS;
    igs_result res{};
    res.x = j.x.data();
    rc = igs_solve(ctx, j.b.data(), j.x0.empty() ? nullptr : j.x0.data(), &so, &res);
    j.status = rc;
    j.beta = res.beta;
    j.steps = res.steps;
    j.cycles = res.cycles;
    igs_destroy(ctx);
}

// ||A||_2 of one matrix by the library's estimator: a context of the smallest restart length
// (its power iteration on A^T A runs at create, on the given stream, with pooled memory).
void estimate_norm(cudaStream_t stream, igs::serve::NormJob &j)
{
    igs_create_opts co{};
    co.stream = stream;
    co.device = j.device;
    co.max_restart_m = 1;
    co.A_norm2 = 0.0;
    co.stream_alloc = 1;
    igs_ctx *ctx = nullptr;
    j.status = igs_create(&ctx, j.n, j.nnz, j.rowptr.data(), j.colind.data(), j.vals.data(), &co);
    if (j.status != IGS_OK) return;
    igs_info info{};
    j.status = igs_get_info(ctx, &info);
    j.normA = info.A_norm2;
    igs_destroy(ctx);
    std::vector<int64_t>().swap(j.rowptr);
    std::vector<int32_t>().swap(j.colind);
    std::vector<double>().swap(j.vals);
}

// The norm worker thread: estimates ||A||_2 for queued gang requests, in arrival order.
void norm_worker(igs_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::unique_ptr<igs::serve::NormJob> job;
        {
            std::unique_lock<std::mutex> lk(s->graph_mu);
            s->norm_cv.wait(lk, [&] { return s->graph_stop || !s->norm_in.empty(); });
            if (s->graph_stop) return;
            job = std::move(s->norm_in.front());
            s->norm_in.pop_front();
        }
        estimate_norm(s->norm_stream, *job);
        std::lock_guard<std::mutex> lk(s->graph_mu);
        s->norm_out.push_back(std::move(job));
    }
}

// A graph lane's worker thread: takes the job handed to its lane, solves it on the lane's
// stream, hands it back.
void graph_worker(igs_server *s, int lane)
{
    cudaSetDevice(s->device);
    igs_server::Lane &L = s->lanes[(size_t)lane];
    for (;;) {
        std::unique_ptr<igs::serve::GraphJob> job;
        {
            std::unique_lock<std::mutex> lk(s->graph_mu);
            s->graph_cv.wait(lk, [&] { return s->graph_stop || L.in != nullptr; });
            if (s->graph_stop) return;
            job = std::move(L.in);
        }
        run_graph_job(s, L.stream, *job);
        std::lock_guard<std::mutex> lk(s->graph_mu);
        L.out = std::move(job);
    }
}

// Finished requests: collect results, release memory.
int collect(igs_server *s)
{
    for (;;) {
        std::unique_ptr<igs::serve::NormJob> nj;
        {
            std::lock_guard<std::mutex> lk(s->graph_mu);
            if (s->norm_out.empty()) break;
            nj = std::move(s->norm_out.front());
            s->norm_out.pop_front();
        }
        Request &r = s->reqs[nj->id];
        r.norm_pending = false;
        if (nj->status == IGS_OK && nj->normA > 0.0 && std::isfinite(nj->normA)) r.normA = nj->normA;
        // (an estimate that failed leaves the bound sqrt(||A||_1 ||A||_inf) >= ||A||_2 in place)
    }
    for (auto &L : s->lanes) {
        std::unique_ptr<igs::serve::GraphJob> fin;
        {
            std::lock_guard<std::mutex> lk(s->graph_mu);
            fin = std::move(L.out);
        }
        if (!fin) continue;
        Request &r = s->reqs[fin->id];
        r.status = fin->status;
        r.res.status = fin->status;
        r.res.beta = fin->beta;
        r.res.steps = fin->steps;
        r.res.cycles = fin->cycles;
        r.bytes = fin->device_bytes;
        if (fin->normA > 0.0) r.normA = fin->normA;
        r.x_host = std::move(fin->x);
        r.t_done = now_s(s);
        r.done = true;
        L.busy = -1;
        s->completions.push_back(r.id);
        s->completed++;
    }
    for (int k = 0; k < s->slots; ++k) {
        const int64_t id = s->slot_req[(size_t)k];
        if (id < 0) continue;
        cudaError_t q = cudaEventQuery(s->events[(size_t)k]);
        if (q == cudaErrorNotReady) continue;
        Request &r = s->reqs[id];
        if (q != cudaSuccess) {
            r.status = IGS_ECUDA;
            s->err = std::string("request ") + std::to_string(id) + ": " + cudaGetErrorString(q);
        } else {
            char *base = s->arena_base + r.arena_off;
            r.x_host.resize((size_t)r.n);
            cudaError_t e = cudaMemcpyAsync(&r.res, base + r.o.res, sizeof(r.res), cudaMemcpyDeviceToHost,
                                            s->streams[(size_t)k]);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r.x_host.data(), base + r.o.x, sizeof(double) * r.n, cudaMemcpyDeviceToHost,
                                    s->streams[(size_t)k]);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->streams[(size_t)k]);
            if (e != cudaSuccess) return sfail(s, IGS_ECUDA, "collecting a result", e);
            r.status = r.res.status;
        }
        r.t_done = now_s(s);
        r.done = true;
        s->running_ctas -= r.G;
        s->arena.release(r.arena_off, r.bytes);
        r.arena_off = -1;
        s->slot_req[(size_t)k] = -1;
        s->completions.push_back(id);
        s->completed++;
    }
    return IGS_OK;
}

// Admit queued requests (FIFO) while a slot is free, the arena has room and the request's
// gang fits beside the running ones (the CTA budget: every admitted gang is co-resident at
// once, so no cooperative launch waits for SMs that later, smaller gangs could take first).
int admit(igs_server *s)
{
    for (auto &L : s->lanes) {
        if (L.busy >= 0 || s->graph_queue.empty()) continue;
        const int64_t id = s->graph_queue.front();
        s->graph_queue.pop_front();
        Request &r = s->reqs[id];
        {
            std::lock_guard<std::mutex> lk(s->graph_mu);
            L.in = std::move(r.job);
        }
        s->graph_cv.notify_all();
        L.busy = id;
        s->launches++;
        r.t_admit = now_s(s);
    }
    while (!s->queue.empty()) {
        int k = -1;
        for (int j = 0; j < s->slots; ++j)
            if (s->slot_req[(size_t)j] < 0) {
                k = j;
                break;
            }
        if (k < 0) return IGS_OK;
        Request &r = s->reqs[s->queue.front()];
        if (r.norm_pending) return IGS_OK;  // admitted in arrival order, once its norm is known
        if (s->running_ctas + r.G > s->cta_budget) return IGS_OK;
        int64_t off = 0;
        if (!s->arena.alloc(r.bytes, &off)) return IGS_OK;
        r.arena_off = off;
        r.slot = k;
        cudaStream_t st = s->streams[(size_t)k];
        const int rc = r.f32 ? launch_request<float>(s, r, st) : launch_request<double>(s, r, st);
        if (rc != IGS_OK) {  // the request completes with IGS_ECUDA
            cudaStreamSynchronize(st);
            s->arena.release(r.arena_off, r.bytes);
            r.arena_off = -1;
            r.status = IGS_ECUDA;
            r.t_admit = r.t_done = now_s(s);
            r.done = true;
            s->completions.push_back(r.id);
            s->completed++;
            s->queue.pop_front();
            return rc;
        }
        cudaError_t e = cudaEventRecord(s->events[(size_t)k], st);
        if (e != cudaSuccess) return sfail(s, IGS_ECUDA, "event record", e);
        s->launches++;
        s->running_ctas += r.G;
        r.t_admit = now_s(s);
        // host copies are on the device now
        std::vector<int64_t>().swap(r.sell_off);
        std::vector<int>().swap(r.sell_col);
        std::vector<double>().swap(r.sell_val);
        std::vector<float>().swap(r.sell_val32);
        std::vector<double>().swap(r.b);
        std::vector<double>().swap(r.x0);
        s->slot_req[(size_t)k] = r.id;
        s->queue.pop_front();
    }
    return IGS_OK;
}

}  // namespace

extern "C" {

int igs_server_create(igs_server **out, const igs_server_opts *opts)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            using namespace igs;
            if (!out) return IGS_EINVAL;
            *out = nullptr;
            if (!opts) return IGS_EINVAL;
            if (opts->max_restart_m < 1 || opts->max_restart_m > IGS_SERVE_MAX_M || opts->arena_bytes <= 0)
                return IGS_EINVAL;
            const int slots = opts->slots > 0 ? opts->slots : 8;
            const int rpc = opts->rows_per_cta > 0 ? opts->rows_per_cta : 4096;
            const int lanes = opts->graph_lanes > 0 ? opts->graph_lanes : 1;
            if (slots > 256 || rpc < 256 || rpc % 32 != 0 || opts->graph_min_n < 0 || lanes > 16) return IGS_EINVAL;
            igs_server *s = new (std::nothrow) igs_server();
            if (!s) return IGS_ENOMEM;
            auto bail = [&](int code) {
                igs_server_destroy(s);
                return code;
            };
            s->device = opts->device;
            s->max_m = opts->max_restart_m;
            s->slots = slots;
            s->rows_per_cta = rpc;
            s->max_queue = opts->max_queue > 0 ? opts->max_queue : 0;
            s->graph_min_n = opts->graph_min_n;
            s->t0 = std::chrono::steady_clock::now();
            if (cudaSetDevice(s->device) != cudaSuccess) return bail(IGS_ECUDA);
            cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
            int optin = 0;
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
            s->smem_max[0] = sizeof(double) * (size_t)sysdev::smem_layout<double>(rpc, s->max_m).total;
            s->smem_max[1] = sizeof(double) * (size_t)sysdev::smem_layout<float>(rpc, s->max_m).total;
            void *kern[2] = {kernel_ptr<double>(), kernel_ptr<float>()};
            for (int t = 0; t < 2; ++t) {
                cudaFuncAttributes fa;
                if (cudaFuncGetAttributes(&fa, kern[t]) != cudaSuccess) return bail(IGS_ECUDA);
                if (s->smem_max[t] + fa.sharedSizeBytes > (size_t)optin) return bail(IGS_EINVAL);
                if (igs::raise_smem_limit(kern[t], s->smem_max[t]) != cudaSuccess) return bail(IGS_ECUDA);
                int nb = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern[t], serve::kThreads, s->smem_max[t]) !=
                    cudaSuccess)
                    return bail(IGS_ECUDA);
                s->max_gang[t] = std::max(1, nb) * s->num_sms;
            }
            s->cta_budget = std::min(s->max_gang[0], s->max_gang[1]);
            if (cudaMalloc(reinterpret_cast<void **>(&s->arena_base), (size_t)opts->arena_bytes) != cudaSuccess)
                return bail(IGS_ENOMEM);
            s->arena.init(opts->arena_bytes);
            s->streams.assign((size_t)slots, nullptr);
            s->events.assign((size_t)slots, nullptr);
            s->slot_req.assign((size_t)slots, -1);
            for (int k = 0; k < slots; ++k)
                if (cudaStreamCreateWithFlags(&s->streams[(size_t)k], cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&s->events[(size_t)k], cudaEventDisableTiming) != cudaSuccess)
                    return bail(IGS_ECUDA);
            if (cudaStreamCreateWithFlags(&s->norm_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(IGS_ECUDA);
            try {
                s->norm_thread = std::thread(norm_worker, s);
            } catch (...) {
                return bail(IGS_ENOMEM);
            }
            if (s->graph_min_n > 0) {
                s->lanes = std::vector<igs_server::Lane>((size_t)lanes);
                for (int l = 0; l < lanes; ++l) {
                    if (cudaStreamCreateWithFlags(&s->lanes[(size_t)l].stream, cudaStreamNonBlocking) != cudaSuccess)
                        return bail(IGS_ECUDA);
                    try {
                        s->lanes[(size_t)l].thread = std::thread(graph_worker, s, l);
                    } catch (...) {
                        return bail(IGS_ENOMEM);
                    }
                }
            }
            *out = s;
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

void igs_server_destroy(igs_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->graph_mu);
        s->graph_stop = true;
        for (auto &L : s->lanes) L.in.reset();
    }
    s->graph_cv.notify_all();
    s->norm_cv.notify_all();
    for (auto &L : s->lanes)
        if (L.thread.joinable()) L.thread.join();  // a running graph-lane solve ends first
    if (s->norm_thread.joinable()) s->norm_thread.join();
    cudaSetDevice(s->device);
    if (s->norm_stream) {
        cudaStreamSynchronize(s->norm_stream);
        cudaStreamDestroy(s->norm_stream);
    }
    for (auto &L : s->lanes)
        if (L.stream) {
            cudaStreamSynchronize(L.stream);
            cudaStreamDestroy(L.stream);
        }
    for (auto st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto ev : s->events)
        if (ev) cudaEventDestroy(ev);
    if (s->arena_base) cudaFree(s->arena_base);
    delete s;
}

int igs_server_submit(igs_server *s, const igs_request *q, int64_t *id_out)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            using namespace igs;
            if (!s) return IGS_EINVAL;
            if (!q || !id_out) return sfail(s, IGS_EINVAL, "null argument");
            const int64_t n = q->n, nnz = q->nnz;
            if (n < 1 || n >= ((int64_t)1 << 30) || nnz < 0 || nnz >= ((int64_t)1 << 31) || !q->rowptr || !q->b ||
                (nnz > 0 && (!q->colind || !q->vals)))
                return sfail(s, IGS_EINVAL, "bad sizes or null arrays");
            if (q->restart_m < 1 || q->restart_m > s->max_m || (q->gs_iters != 1 && q->gs_iters != 2) ||
                !(q->tol_beta >= 0.0) || q->max_restarts < 1 ||
                (q->precision != IGS_PREC_FP64 && q->precision != IGS_PREC_FP32_IR))
                return sfail(s, IGS_EINVAL, "bad request options");
            if (q->rowptr[0] != 0 || q->rowptr[n] != nnz) return sfail(s, IGS_EINVAL, "rowptr[0] must be 0, rowptr[n] = nnz");
            if (s->max_queue > 0 && (int64_t)(s->queue.size() + s->graph_queue.size()) >= s->max_queue)
                return sfail(s, IGS_ENOMEM, "queue full");
            std::vector<double> rowabs((size_t)n, 0.0), colabs((size_t)n, 0.0);
            for (int64_t i = 0; i < n; ++i) {
                if (q->rowptr[i + 1] < q->rowptr[i]) return sfail(s, IGS_EINVAL, "rowptr decreases");
                for (int64_t k = q->rowptr[i]; k < q->rowptr[i + 1]; ++k) {
                    if (q->colind[k] < 0 || q->colind[k] >= n) return sfail(s, IGS_EINVAL, "column index out of range");
                    if (!std::isfinite(q->vals[k])) return sfail(s, IGS_ENUMERIC, "non-finite matrix value");
                    rowabs[(size_t)i] += std::fabs(q->vals[k]);
                    colabs[(size_t)q->colind[k]] += std::fabs(q->vals[k]);
                }
            }
            Request r;
            r.id = s->next_id++;
            r.opt = *q;
            r.opt.rowptr = nullptr;
            r.opt.colind = nullptr;
            r.opt.vals = nullptr;
            r.opt.b = nullptr;
            r.opt.x0 = nullptr;
            r.n = (int)n;
            r.n2 = (int)((n + 1) / 2 * 2);
            r.ldv = (int)((n + 3) / 4 * 4);
            r.f32 = q->precision == IGS_PREC_FP32_IR;
            r.has_x0 = q->x0 != nullptr;
            const bool estimate = !(q->A_norm2 > 0.0);
            if (!estimate) {
                r.normA = q->A_norm2;
            } else {
                // placeholder until the GPU estimate arrives: ||A||_2 <= sqrt(||A||_1 ||A||_inf)
                const double n1 = *std::max_element(colabs.begin(), colabs.end());
                const double ninf = *std::max_element(rowabs.begin(), rowabs.end());
                r.normA = std::sqrt(n1 * ninf);
            }
            if (s->graph_min_n > 0 && n >= s->graph_min_n) {
                // graph lane: the library solves it with whole-GPU kernels; keep the CSR form
                auto job = std::make_unique<igs::serve::GraphJob>();
                job->id = r.id;
                job->opt = r.opt;
                job->opt.colind = nullptr;
                job->opt.vals = nullptr;
                job->opt.b = nullptr;
                job->opt.x0 = nullptr;
                job->normA = estimate ? 0.0 : r.normA;  // 0: the lane's igs_create estimates it
                job->rowptr.assign(q->rowptr, q->rowptr + n + 1);
                job->colind.assign(q->colind, q->colind + nnz);
                job->vals.assign(q->vals, q->vals + nnz);
                job->b.assign(q->b, q->b + n);
                if (r.has_x0) job->x0.assign(q->x0, q->x0 + n);
                r.graph = true;
                r.G = 0;
                r.job = std::move(job);
                r.t_submit = now_s(s);
                const int64_t id = r.id;
                s->reqs.emplace(id, std::move(r));
                s->graph_queue.push_back(id);
                s->submitted++;
                *id_out = id;
                return IGS_OK;
            }
            // gang: about rows_per_cta rows per CTA, rows split on multiples of 32.  A gang of more
            // CTAs than SMs is rounded up to a whole number of CTAs per SM (within the CTA budget),
            // so that when it runs alone no SM carries more of its rows than another.
            int G = (r.n2 + s->rows_per_cta - 1) / s->rows_per_cta;
            if (G > s->num_sms) G = std::min((G + s->num_sms - 1) / s->num_sms * s->num_sms, std::max(G, s->cta_budget));
            int chunk = ((r.n2 + G - 1) / G + 31) / 32 * 32;
            G = (r.n2 + chunk - 1) / chunk;
            if (G > s->cta_budget) return sfail(s, IGS_EINVAL, "system too large for one co-resident gang");
            r.G = G;
            r.chunk = chunk;
            r.smem = r.f32 ? sizeof(double) * (size_t)sysdev::smem_layout<float>(chunk, r.opt.restart_m).total
                           : sizeof(double) * (size_t)sysdev::smem_layout<double>(chunk, r.opt.restart_m).total;
            // SELL-32 (32-row slices, each as wide as its longest row, CSR order, padding -1)
            const int64_t nsl = (n + 31) / 32;
            r.sell_off.assign((size_t)nsl + 1, 0);
            for (int64_t k = 0; k < nsl; ++k) {
                int64_t w = 0;
                for (int64_t i = 32 * k; i < std::min(n, 32 * k + 32); ++i) w = std::max(w, q->rowptr[i + 1] - q->rowptr[i]);
                r.sell_off[(size_t)k + 1] = r.sell_off[(size_t)k] + 32 * w;
            }
            const int64_t ne = r.sell_off[(size_t)nsl];
            r.sell_col.assign((size_t)std::max<int64_t>(ne, 1), -1);
            r.sell_val.assign((size_t)std::max<int64_t>(ne, 1), 0.0);
            for (int64_t i = 0; i < n; ++i)
                for (int64_t j = 0; j < q->rowptr[i + 1] - q->rowptr[i]; ++j) {
                    const size_t e = (size_t)(r.sell_off[(size_t)(i >> 5)] + 32 * j + (i & 31));
                    r.sell_col[e] = q->colind[q->rowptr[i] + j];
                    r.sell_val[e] = q->vals[q->rowptr[i] + j];
                }
            if (r.f32) {
                r.sell_val32.resize(r.sell_val.size());
                for (size_t e = 0; e < r.sell_val.size(); ++e) r.sell_val32[e] = (float)r.sell_val[e];
            }
            r.b.assign(q->b, q->b + n);
            if (r.has_x0) r.x0.assign(q->x0, q->x0 + n);
            r.bytes = plan_request(r, 2 * (r.opt.restart_m + 1) + 2);
            if (r.bytes > s->arena.size()) return sfail(s, IGS_EINVAL, "request larger than the arena");
            if (estimate) {
                auto nj = std::make_unique<igs::serve::NormJob>();
                nj->id = r.id;
                nj->n = n;
                nj->nnz = nnz;
                nj->device = s->device;
                nj->rowptr.assign(q->rowptr, q->rowptr + n + 1);
                nj->colind.assign(q->colind, q->colind + nnz);
                nj->vals.assign(q->vals, q->vals + nnz);
                r.norm_pending = true;
                {
                    std::lock_guard<std::mutex> lk(s->graph_mu);
                    s->norm_in.push_back(std::move(nj));
                }
                s->norm_cv.notify_one();
            }
            r.t_submit = now_s(s);
            const int64_t id = r.id;
            s->reqs.emplace(id, std::move(r));
            s->queue.push_back(id);
            s->submitted++;
            *id_out = id;
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

int igs_server_pump(igs_server *s, int *running)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!s) return IGS_EINVAL;
            if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, IGS_ECUDA, "cudaSetDevice");
            int rc = collect(s);
            if (rc == IGS_OK) rc = admit(s);
            if (running) {
                int k = 0;
                for (auto &L : s->lanes) k += L.busy >= 0;
                for (auto id : s->slot_req) k += id >= 0;
                *running = k;
            }
            return rc;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

int igs_server_poll(igs_server *s, igs_completion *out, int max_out, int *n_out)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!s || !n_out || (max_out > 0 && !out)) return IGS_EINVAL;
            int k = 0;
            while (k < max_out && !s->completions.empty()) {
                const int64_t id = s->completions.front();
                s->completions.pop_front();
                Request &r = s->reqs[id];
                igs_completion &c = out[k++];
                c.id = id;
                c.status = r.status;
                c.beta = r.res.beta;
                c.steps = r.res.steps;
                c.cycles = r.res.cycles;
                c.gang_ctas = r.G;
                c.device_bytes = r.bytes;
                c.path = r.graph ? IGS_SERVE_PATH_GRAPH : IGS_SERVE_PATH_GANG;
                c.t_submit = r.t_submit;
                c.t_admit = r.t_admit;
                c.t_done = r.t_done;
                c.A_norm2 = r.normA;
                r.polled = true;
            }
            *n_out = k;
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

int igs_server_take_result(igs_server *s, int64_t id, double *x)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!s || !x) return IGS_EINVAL;
            auto it = s->reqs.find(id);
            if (it == s->reqs.end() || !it->second.done) return sfail(s, IGS_EINVAL, "unknown or unfinished request");
            std::memcpy(x, it->second.x_host.data(), sizeof(double) * it->second.x_host.size());
            s->reqs.erase(it);
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

int igs_server_get_stats(const igs_server *s, igs_server_stats *o)
{
    if (!s || !o) return IGS_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->submitted = s->submitted;
    o->queued = (int64_t)(s->queue.size() + s->graph_queue.size());
    o->running = 0;
    for (auto &L : s->lanes) o->running += L.busy >= 0;
    for (auto id : s->slot_req) o->running += id >= 0;
    o->completed = s->completed;
    o->arena_bytes = s->arena.size();
    o->arena_used = s->arena.used();
    o->arena_peak = s->arena.peak();
    o->launches = s->launches;
    return IGS_OK;
}

double igs_server_clock(const igs_server *s) { return s ? now_s(s) : 0.0; }

int igs_server_gang_selftest(int device, int G, int stall, int *abort_out)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            using namespace igs;
            if (G < 2 || (stall != 0 && stall != 1)) return IGS_EINVAL;
            if (cudaSetDevice(device) != cudaSuccess) return IGS_ECUDA;
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || G > sms)
                return IGS_EINVAL;
            sysdev::GangSync *sync = nullptr;
            int *ok = nullptr;
            cudaStream_t st = nullptr;
            int rc = IGS_ECUDA;
            std::vector<int> h((size_t)G, 0);
            sysdev::GangSync hs{};
            // stalled: an arrival count that no arrival brings to G, so that every wait runs out
            hs.count = stall ? 0x40000000u : 0u;
            if (cudaMalloc(&sync, sizeof(sysdev::GangSync)) == cudaSuccess && cudaMalloc(&ok, sizeof(int) * G) == cudaSuccess &&
                cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
                cudaMemcpyAsync(sync, &hs, sizeof(hs), cudaMemcpyHostToDevice, st) == cudaSuccess &&
                cudaMemsetAsync(ok, 0, sizeof(int) * G, st) == cudaSuccess) {
                void *args[] = {&sync, &ok};
                if (cudaLaunchCooperativeKernel(reinterpret_cast<void *>(serve::k_gang_selftest), dim3(G),
                                                dim3(serve::kThreads), args, 0, st) == cudaSuccess &&
                    cudaMemcpyAsync(h.data(), ok, sizeof(int) * G, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                    cudaMemcpyAsync(&hs, sync, sizeof(hs), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess) {
                    int passed = 0;
                    for (int v : h) passed += v;
                    if (abort_out) *abort_out = hs.abort;
                    rc = passed == G ? IGS_OK : IGS_ETIMEOUT;
                }
            }
            if (st) cudaStreamDestroy(st);
            cudaFree(ok);
            cudaFree(sync);
            return rc;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

const char *igs_server_last_error(const igs_server *s) { return s ? s->err.c_str() : "null server"; }

}  // extern "C"
