// Batched IGS-GMRES (include/igs_batch.h): many independent sparse systems solved by one
// persistent kernel launch.
//
// Each CTA takes systems from a device work queue (largest first) and runs the whole
// restarted IGS-GMRES(m) of Alg. 4.1 on one system at a time: the device solver of
// igs_sysdev.cuh with a gang of one CTA (cycle start and the backward error of eq. "nrbe",
// steps 1-18, the Givens least squares with the in-cycle stop test, the flush, x_m = x_0 +
// V_m y_m, breakdown and restarts, with the single-system path's control flow).  Every
// per-step scalar lives in shared memory, so a step costs no kernel launch and no host round
// trip.
//
// Determinism: the arithmetic of a system depends only on that system (its n, its CSR rows
// and the solve options), never on the CTA, the block size, the number of resident CTAs or
// the other systems of the batch (igs_sysdev.cuh: fixed slices and orders, fixed lane roles).
// So a system's x, beta and step count are bitwise the same whether it is solved alone or
// in a batch, and under every launch configuration the tuner may pick.
//
// Memory: each CTA (slot) owns a basis V of (m+1) columns with leading dimension
// round_up(n, 4) and the Givens factor R (packed upper, column-major) in HBM (re-read from
// L2 when the working set fits); the Krylov vector z/u, the slice partial sums, L (packed
// strictly-lower, column-major) and the small vectors are in shared memory.  A is kept in
// SELL-32 (32-row slices, each as wide as its longest row, entries in CSR order).
#include "../../include/igs.h"
#include "../../include/igs_batch.h"
#include "igs_internal.h"
#include "igs_sysdev.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace igs {
namespace batch {

using sysdev::round_up;
using sysdev::SmemLayout;

constexpr int kMaxM = IGS_BATCH_MAX_M;  // largest restart length of the batched solver
constexpr int kMaxN = IGS_BATCH_MAX_N;  // largest system (the Krylov vector is kept in shared memory)
constexpr int kMaxSlotsPerSM = 8;       // largest resident CTAs per SM any configuration uses
static_assert(kMaxM <= sysdev::kMaxM, "restart length beyond the device solver's limit");

__host__ __device__ inline SmemLayout smem_layout(int nmax, int m)
{
    return sysdev::smem_layout<double>(round_up(nmax, 2), m);
}

// Matrix and workspace of a batch (kernel argument, by value).
struct Args {
    int m;
    int nmax;
    const int64_t *sys_row0;  // count+1 row offsets into the concatenated vectors
    // A in sliced ELL (SELL-32): slice k (32 consecutive rows of one system) holds its
    // entries at sell_off[k] .. sell_off[k+1]-1, entry j of lane r at sell_off[k] + 32 j + r,
    // in the row's CSR order; padding has column -1.  sys_slice0[s] is system s's first slice.
    const int64_t *sell_off;
    const int *sys_slice0;
    const int *sell_col;      // column index local to the system, or -1
    const double *sell_val;
    const double *normA;      // per system ||A_s||_2
    double *vslots;           // per-CTA basis storage: V, then R at r_offset
    int64_t slot_stride;      // doubles per slot
    int64_t r_offset;         // doubles from a slot's start to its R
    unsigned int *queue;      // work counter (zeroed before each launch)
    unsigned long long *summary;  // [0] total steps, [1+k] systems with status code k-6
};

// Per-call parameters, copied to the device before each launch.
struct Run {
    const int *order;   // systems in solve order
    int count;          // entries of order
    int gs;
    int max_cycles;
    int x0_given;
    double tol;
    const double *b;    // N, concatenated
    const double *x0;   // N or null
    double *x;          // N
    double *beta;       // per system (indexed by system id), nullable
    int *status;        // nullable
    int64_t *steps;     // nullable
    int *cycles;        // nullable
};

// The solve arguments of system sid in CTA slot V / R.
__device__ sysdev::SysArgs<double> sys_args(const Args &a, const Run &run, int sid, double *V)
{
    sysdev::SysArgs<double> s;
    const int64_t row0 = a.sys_row0[sid];
    s.n = (int)(a.sys_row0[sid + 1] - row0);
    s.m = a.m;
    s.gs = run.gs;
    s.max_cycles = run.max_cycles;
    s.ldv = round_up(s.n, 4);
    s.tol = run.tol;
    s.inner_tol = 0.0;
    s.normA = a.normA[sid];
    s.sell_off = a.sell_off + a.sys_slice0[sid];
    s.sell_col = a.sell_col;
    s.sell_val = a.sell_val;
    s.sell_val32 = nullptr;
    s.b = run.b + row0;
    s.x0 = run.x0_given ? run.x0 + row0 : nullptr;
    s.x = run.x + row0;
    s.V = V;
    s.r64 = nullptr;
    s.beta_out = run.beta ? run.beta + sid : nullptr;
    s.status_out = run.status ? run.status + sid : nullptr;
    s.steps_out = run.steps ? run.steps + sid : nullptr;
    s.cycles_out = run.cycles ? run.cycles + sid : nullptr;
    return s;
}

// The persistent batched solver: CTAs take systems from the queue until it is empty.
// Instantiated per block size T with the register budget of MINB resident CTAs per SM.
template <int T, int MINB>
__global__ void __launch_bounds__(T, MINB) k_batch_solve(Args a, const Run *__restrict__ runp)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ sysdev::Shared sh;
    __shared__ Run run;
    __shared__ int s_next;
    if (threadIdx.x == 0) {
        run = *runp;
        sysdev::init_shared(sh);
    }
    const SmemLayout L = smem_layout(a.nmax, a.m);
    double *V = a.vslots + (int64_t)blockIdx.x * a.slot_stride;
    for (;;) {
        if (threadIdx.x == 0) s_next = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int q = s_next;
        __syncthreads();
        if (q >= run.count) break;
        const int sid = run.order[q];
        const sysdev::SysArgs<double> sa = sys_args(a, run, sid, V);
        sysdev::Gang gg;
        gg.G = 1;
        gg.g = 0;
        gg.lo = 0;
        gg.hi = round_up(sa.n, 2);
        gg.sync = nullptr;
        gg.gpart = nullptr;
        gg.gld = 0;
        gg.R = V + a.r_offset;
        sysdev::d_solve<double>(sa, gg, sm, L, sh);
        if (threadIdx.x == 0) {
            atomicAdd(&a.summary[0], (unsigned long long)sh.steps);
            const int k = sh.status + 6;  // status codes -6..2 -> 0..8
            if (k >= 0 && k < 9) atomicAdd(&a.summary[1 + k], 1ull);
        }
        __syncthreads();
    }
}

// ||A_s||_2 by power iteration on A_s^T A_s (one CTA per system; At = A^T in the same
// sliced form).  Start vector: a fixed hash of the row index.
__global__ void __launch_bounds__(256) k_batch_norm2(Args a, const int64_t *__restrict__ at_off,
                                                     const int *__restrict__ at_col,
                                                     const double *__restrict__ at_val, int count,
                                                     int iters, double *__restrict__ out)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ sysdev::Shared sh;
    __shared__ double s_lam;
    if (threadIdx.x == 0) sysdev::init_shared(sh);
    __syncthreads();
    const SmemLayout L = smem_layout(a.nmax, a.m);
    double *V = a.vslots + (int64_t)blockIdx.x * a.slot_stride;
    for (int sid = blockIdx.x; sid < count; sid += gridDim.x) {
        const int64_t row0 = a.sys_row0[sid];
        const int n = (int)(a.sys_row0[sid + 1] - row0);
        const int ldv = round_up(n, 4);
        sysdev::SysArgs<double> sa{}, st{};
        sa.n = st.n = n;
        sa.sell_off = a.sell_off + a.sys_slice0[sid];
        sa.sell_col = a.sell_col;
        sa.sell_val = a.sell_val;
        st.sell_off = at_off + a.sys_slice0[sid];
        st.sell_col = at_col;
        st.sell_val = at_val;
        sysdev::Gang gg{};
        gg.G = 1;
        gg.hi = round_up(n, 2);
        double *xv = V, *yv = V + ldv, *uv = V + 2 * (int64_t)ldv;
        const double sc = 1.0 / sqrt((double)n);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            uint64_t hsh = (uint64_t)i * 0x9E3779B97F4A7C15ull;
            hsh ^= hsh >> 29;
            xv[i] = sc * (0.5 + (double)(hsh >> 11) * 0x1p-53);
        }
        __syncthreads();
        double lam = 0.0;
        for (int it = 0; it < iters; ++it) {
            sysdev::d_spmv<double, double, double, double, false>(sa, gg, sa.sell_val, xv, nullptr, yv);
            __syncthreads();
            sysdev::d_spmv<double, double, double, double, false>(st, gg, st.sell_val, yv, nullptr, uv);
            __syncthreads();
            sysdev::d_sumsq<double, double>(gg, sh, n, uv, (const double *)nullptr, 1, sm + L.part, sm + L.red);
            if (threadIdx.x == 0) s_lam = sqrt(sm[L.red]);
            __syncthreads();
            lam = s_lam;
            const double f = lam > 0.0 ? 1.0 / lam : 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) xv[i] = uv[i] * f;
            __syncthreads();
        }
        if (threadIdx.x == 0) out[sid] = sqrt(lam);
        __syncthreads();
    }
}

using BatchKernel = void (*)(Args, const Run *);

// Kernel instance for a block size (128, 256 or 512 threads), else null.
inline BatchKernel batch_kernel(int threads)
{
    switch (threads) {
    case 128: return k_batch_solve<128, 5>;
    case 256: return k_batch_solve<256, 2>;
    case 512: return k_batch_solve<512, 1>;
    default: return nullptr;
    }
}

}  // namespace batch
}  // namespace igs

// =====================================================================================
// Host side.
// =====================================================================================
using igs::batch::Args;
using igs::batch::Run;

struct igs_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int count = 0, m = 0, nmax = 0, num_sms = 0;
    int64_t N = 0, nnz = 0;
    size_t smem = 0;
    int max_smem_optin = 0;
    // device data
    int64_t *sys_row0 = nullptr, *sell_off = nullptr;
    int *sys_slice0 = nullptr, *sell_col = nullptr, *order = nullptr, *order_sample = nullptr;
    double *sell_val = nullptr, *normA = nullptr, *vslots = nullptr;
    int64_t slot_stride = 0, r_offset = 0;
    int slots_alloc = 0;
    unsigned int *queue = nullptr;
    unsigned long long *summary = nullptr;
    Run *run_dev = nullptr;
    Run *run_host = nullptr;                // pinned
    unsigned long long *summary_host = nullptr;  // pinned, 10 entries
    double *b_dev = nullptr, *x_dev = nullptr, *x0_dev = nullptr, *beta_dev = nullptr;
    double *b_tune = nullptr;
    int *status_dev = nullptr, *cycles_dev = nullptr;
    int64_t *steps_dev = nullptr;
    int sample_count = 0;
    std::vector<double> normA_host;
    // launch configuration
    int threads = 256, bpsm = 2;
    std::vector<igs_batch_tune_entry> tune;
    // captured launch per configuration
    struct G {
        int threads, bpsm;
        cudaGraphExec_t exec;
    };
    std::vector<G> graphs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
};

namespace {

int fail(igs_batch *bt, int code, const char *what, cudaError_t e = cudaSuccess)
{
    if (bt) {
        bt->err = what;
        if (e != cudaSuccess) {
            bt->err += ": ";
            bt->err += cudaGetErrorString(e);
        }
    }
    return code;
}

#define BT_CUDA(call, what)                                          \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return fail(bt, IGS_ECUDA, what, e_); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
}

Args make_args(const igs_batch *bt)
{
    Args a;
    a.m = bt->m;
    a.nmax = bt->nmax;
    a.sys_row0 = bt->sys_row0;
    a.sell_off = bt->sell_off;
    a.sys_slice0 = bt->sys_slice0;
    a.sell_col = bt->sell_col;
    a.sell_val = bt->sell_val;
    a.normA = bt->normA;
    a.vslots = bt->vslots;
    a.slot_stride = bt->slot_stride;
    a.r_offset = bt->r_offset;
    a.queue = bt->queue;
    a.summary = bt->summary;
    return a;
}

int max_blocks_per_sm(igs_batch *bt, int threads, int *out)
{
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, igs::batch::batch_kernel(threads),
                                                                  threads, bt->smem);
    if (e != cudaSuccess) return fail(bt, IGS_ECUDA, "occupancy query", e);
    *out = nb < igs::batch::kMaxSlotsPerSM ? nb : igs::batch::kMaxSlotsPerSM;
    return IGS_OK;
}

// Capture (once per configuration) the launch: parameter copy, queue reset, persistent kernel.
int get_graph(igs_batch *bt, int threads, int bpsm, cudaGraphExec_t *out)
{
    for (auto &g : bt->graphs)
        if (g.threads == threads && g.bpsm == bpsm) {
            *out = g.exec;
            return IGS_OK;
        }
    const int grid = bt->num_sms * bpsm;
    if (grid > bt->slots_alloc) return fail(bt, IGS_EINVAL, "configuration needs more basis slots than allocated");
    cudaStream_t cs = nullptr;
    BT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemcpyAsync(bt->run_dev, bt->run_host, sizeof(Run), cudaMemcpyHostToDevice, cs);
        cudaMemsetAsync(bt->queue, 0, sizeof(unsigned int), cs);
        cudaMemsetAsync(bt->summary, 0, 10 * sizeof(unsigned long long), cs);
        igs::batch::batch_kernel(threads)<<<grid, threads, bt->smem, cs>>>(make_args(bt), bt->run_dev);
        cudaError_t le = cudaGetLastError();
        cudaMemcpyAsync(bt->summary_host, bt->summary, 10 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(bt, IGS_ECUDA, "capturing the batched launch", e);
    bt->graphs.push_back({threads, bpsm, exec});
    *out = exec;
    return IGS_OK;
}

// Launch with the current run parameters (run_host already filled); optionally time it.
int launch(igs_batch *bt, int threads, int bpsm, float *ms)
{
    cudaGraphExec_t exec = nullptr;
    int rc = get_graph(bt, threads, bpsm, &exec);
    if (rc != IGS_OK) return rc;
    BT_CUDA(cudaEventRecord(bt->ev0, bt->stream), "event");
    BT_CUDA(cudaGraphLaunch(exec, bt->stream), "graph launch");
    BT_CUDA(cudaEventRecord(bt->ev1, bt->stream), "event");
    BT_CUDA(cudaStreamSynchronize(bt->stream), "batched solve");
    if (ms) BT_CUDA(cudaEventElapsedTime(ms, bt->ev0, bt->ev1), "event time");
    return IGS_OK;
}

bool valid_threads(int t) { return t == 128 || t == 256 || t == 512; }

// Time every launch configuration on a sample of the batch (every 4th system in solve
// order) with b = A * ones, and keep the fastest.  Results never depend on the choice.
int autotune(igs_batch *bt, int gs, double tol, int max_restarts)
{
    bt->tune.clear();
    Run *r = bt->run_host;
    std::memset(r, 0, sizeof(Run));
    r->order = bt->order_sample;
    r->count = bt->sample_count;
    r->gs = gs;
    r->max_cycles = max_restarts;
    r->x0_given = 0;
    r->tol = tol;
    r->b = bt->b_tune;
    r->x = bt->x_dev;
    float best = 1e30f;
    int bt_threads = bt->threads, bt_bpsm = bt->bpsm;
    const int cand_threads[3] = {128, 256, 512};
    for (int ti = 0; ti < 3; ++ti) {
        const int t = cand_threads[ti];
        int maxb = 0;
        int rc = max_blocks_per_sm(bt, t, &maxb);
        if (rc != IGS_OK) return rc;
        for (int b = 1; b <= maxb; ++b) {
            if (bt->num_sms * b > bt->slots_alloc) break;
            float ms0 = 0.f, ms1 = 0.f;
            rc = launch(bt, t, b, &ms0);  // first run includes capture effects
            if (rc != IGS_OK) return rc;
            rc = launch(bt, t, b, &ms1);
            if (rc != IGS_OK) return rc;
            const float ms = std::min(ms0, ms1);
            igs_batch_tune_entry te;
            te.block_threads = t;
            te.blocks_per_sm = b;
            te.ms = ms;
            bt->tune.push_back(te);
            if (ms < best) {
                best = ms;
                bt_threads = t;
                bt_bpsm = b;
            }
        }
    }
    bt->threads = bt_threads;
    bt->bpsm = bt_bpsm;
    return IGS_OK;
}

}  // namespace

namespace {

// Sliced ELL (32-row slices, each as wide as its longest row) of a block-diagonal CSR with
// system-local column indices; entries keep each row's CSR order.
struct SellHost {
    std::vector<int> slice0;     // count+1
    std::vector<int64_t> off;    // slices+1
    std::vector<int> col;
    std::vector<double> val;
};

void build_sell(int count, const int64_t *sys_ptr, const int64_t *rp, const int *ci, const double *va,
                SellHost &out)
{
    out.slice0.assign((size_t)count + 1, 0);
    int64_t nsl = 0;
    for (int s = 0; s < count; ++s) {
        out.slice0[(size_t)s] = (int)nsl;
        nsl += (sys_ptr[s + 1] - sys_ptr[s] + 31) / 32;
    }
    out.slice0[(size_t)count] = (int)nsl;
    out.off.assign((size_t)nsl + 1, 0);
    int64_t k = 0;
    for (int s = 0; s < count; ++s)
        for (int64_t r0 = sys_ptr[s]; r0 < sys_ptr[s + 1]; r0 += 32, ++k) {
            const int64_t r1 = std::min(r0 + 32, sys_ptr[s + 1]);
            int64_t w = 0;
            for (int64_t i = r0; i < r1; ++i) w = std::max(w, rp[i + 1] - rp[i]);
            out.off[(size_t)k + 1] = out.off[(size_t)k] + 32 * w;
        }
    out.col.assign((size_t)std::max<int64_t>(out.off[(size_t)nsl], 1), -1);
    out.val.assign((size_t)std::max<int64_t>(out.off[(size_t)nsl], 1), 0.0);
    k = 0;
    for (int s = 0; s < count; ++s)
        for (int64_t r0 = sys_ptr[s]; r0 < sys_ptr[s + 1]; r0 += 32, ++k) {
            const int64_t r1 = std::min(r0 + 32, sys_ptr[s + 1]);
            for (int64_t i = r0; i < r1; ++i)
                for (int64_t j = 0; j < rp[i + 1] - rp[i]; ++j) {
                    const size_t e = (size_t)(out.off[(size_t)k] + 32 * j + (i - r0));
                    out.col[e] = ci[rp[i] + j];
                    out.val[e] = va[rp[i] + j];
                }
        }
}

int upload_sell(const SellHost &h, int64_t **off, int **slice0, int **col, double **val, cudaStream_t s)
{
    const size_t ne = h.col.size();
    if (dalloc(off, h.off.size()) || dalloc(col, ne) || dalloc(val, ne) ||
        (slice0 && dalloc(slice0, h.slice0.size())))
        return IGS_ENOMEM;
    if (cudaMemcpyAsync(*off, h.off.data(), sizeof(int64_t) * h.off.size(), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(*col, h.col.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(*val, h.val.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, s) ||
        (slice0 && cudaMemcpyAsync(*slice0, h.slice0.data(), sizeof(int) * h.slice0.size(),
                                   cudaMemcpyHostToDevice, s)))
        return IGS_ECUDA;
    return IGS_OK;
}

}  // namespace

extern "C" int igs_batch_create(igs_batch **out, int count, const int64_t *sys_ptr,
                                const int64_t *rowptr, const int32_t *colind, const double *vals,
                                const igs_batch_opts *opts)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            using namespace igs::batch;
            if (!out) return IGS_EINVAL;
            *out = nullptr;
            if (count < 1 || !sys_ptr || !rowptr || !opts) return IGS_EINVAL;
            const int m = opts->restart_m;
            if (m < 1 || m > kMaxM) return IGS_EINVAL;
            if (sys_ptr[0] != 0) return IGS_EINVAL;
            int nmax = 0;
            for (int s = 0; s < count; ++s) {
                const int64_t n = sys_ptr[s + 1] - sys_ptr[s];
                if (n < 1 || n > kMaxN) return IGS_EINVAL;
                nmax = std::max(nmax, (int)n);
            }
            const int64_t N = sys_ptr[count];
            if (rowptr[0] != 0) return IGS_EINVAL;
            for (int64_t i = 0; i < N; ++i)
                if (rowptr[i + 1] < rowptr[i]) return IGS_EINVAL;
            const int64_t nnz = rowptr[N];
            if (nnz >= ((int64_t)1 << 31)) return IGS_EINVAL;
            if (nnz > 0 && (!colind || !vals)) return IGS_EINVAL;
            // every entry of system s must lie in its diagonal block; store local column indices
            std::vector<int> loc((size_t)(nnz ? nnz : 1));
            for (int s = 0; s < count; ++s) {
                const int64_t r0 = sys_ptr[s], r1 = sys_ptr[s + 1];
                for (int64_t i = r0; i < r1; ++i)
                    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                        const int64_t c = colind[k];
                        if (c < r0 || c >= r1) return IGS_EINVAL;
                        if (!std::isfinite(vals[k])) return IGS_ENUMERIC;
                        loc[(size_t)k] = (int)(c - r0);
                    }
            }
            if (opts->A_norm2)
                for (int s = 0; s < count; ++s)
                    if (!(opts->A_norm2[s] >= 0.0) || !std::isfinite(opts->A_norm2[s])) return IGS_EINVAL;
            if (opts->block_threads != 0 && !valid_threads(opts->block_threads)) return IGS_EINVAL;
            if (opts->blocks_per_sm < 0 || opts->blocks_per_sm > kMaxSlotsPerSM) return IGS_EINVAL;

            igs_batch *bt = new (std::nothrow) igs_batch();
            if (!bt) return IGS_ENOMEM;
            int rc = IGS_OK;
            auto bail = [&](int code) {
                igs_batch_destroy(bt);
                return code;
            };
            bt->device = opts->device;
            if (cudaSetDevice(bt->device) != cudaSuccess) return bail(IGS_ECUDA);
            if (opts->stream) {
                bt->stream = static_cast<cudaStream_t>(opts->stream);
            } else {
                if (cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(IGS_ECUDA);
                bt->own_stream = true;
            }
            bt->count = count;
            bt->m = m;
            bt->nmax = nmax;
            bt->N = N;
            bt->nnz = nnz;
            if (cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, bt->device) != cudaSuccess)
                return bail(IGS_ECUDA);
            if (cudaDeviceGetAttribute(&bt->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, bt->device) !=
                cudaSuccess)
                return bail(IGS_ECUDA);
            const SmemLayout L = smem_layout(nmax, m);
            bt->smem = sizeof(double) * (size_t)L.total;
            for (int t : {128, 256, 512}) {
                cudaFuncAttributes fa;
                if (cudaFuncGetAttributes(&fa, batch_kernel(t)) != cudaSuccess) return bail(IGS_ECUDA);
                if (bt->smem + fa.sharedSizeBytes > (size_t)bt->max_smem_optin) return bail(IGS_EINVAL);
                if (igs::raise_smem_limit((const void *)batch_kernel(t), bt->smem) != cudaSuccess) return bail(IGS_ECUDA);
            }
            if (igs::raise_smem_limit((const void *)k_batch_norm2, bt->smem) != cudaSuccess) return bail(IGS_ECUDA);

            // slots: one per CTA of the largest configuration the GPU can hold (any block size)
            int slots_per_sm = 0;
            for (int t : {128, 256, 512}) {
                int nb = 0;
                rc = max_blocks_per_sm(bt, t, &nb);
                if (rc != IGS_OK) return bail(rc);
                slots_per_sm = std::max(slots_per_sm, nb);
            }
            if (slots_per_sm < 1) return bail(IGS_EINVAL);
            bt->slots_alloc = bt->num_sms * slots_per_sm;
            // (m+1) basis columns (at least three for the power iteration's vectors), then R
            bt->r_offset = (int64_t)std::max(m + 1, 3) * round_up(nmax, 4);
            bt->slot_stride = bt->r_offset + (int64_t)m * (m + 1) / 2;
            bt->slot_stride = (bt->slot_stride + 31) / 32 * 32;

            // solve order: largest system first (ties by index); the tuning sample is every 4th
            std::vector<int> order(count);
            for (int s = 0; s < count; ++s) order[s] = s;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                return sys_ptr[x + 1] - sys_ptr[x] > sys_ptr[y + 1] - sys_ptr[y];
            });
            std::vector<int> sample;
            for (int q = 0; q < count; q += 4) sample.push_back(order[q]);
            bt->sample_count = (int)sample.size();

            // b for tuning: A * ones
            std::vector<double> btune((size_t)N);
            for (int64_t i = 0; i < N; ++i) {
                double s = 0.0;
                for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += vals[k];
                btune[(size_t)i] = s;
            }

            if (dalloc(&bt->sys_row0, (size_t)count + 1) || dalloc(&bt->order, (size_t)count) || dalloc(&bt->order_sample, sample.size()) ||
                dalloc(&bt->normA, (size_t)count) ||
                dalloc(&bt->vslots, (size_t)bt->slots_alloc * (size_t)bt->slot_stride) ||
                dalloc(&bt->queue, 1) || dalloc(&bt->summary, 10) || dalloc(&bt->run_dev, 1) ||
                dalloc(&bt->b_dev, (size_t)N) || dalloc(&bt->x_dev, (size_t)N) || dalloc(&bt->x0_dev, (size_t)N) ||
                dalloc(&bt->b_tune, (size_t)N) || dalloc(&bt->beta_dev, (size_t)count) ||
                dalloc(&bt->status_dev, (size_t)count) || dalloc(&bt->cycles_dev, (size_t)count) ||
                dalloc(&bt->steps_dev, (size_t)count))
                return bail(IGS_ENOMEM);
            if (cudaMallocHost(reinterpret_cast<void **>(&bt->run_host), sizeof(Run)) != cudaSuccess ||
                cudaMallocHost(reinterpret_cast<void **>(&bt->summary_host), 10 * sizeof(unsigned long long)) !=
                    cudaSuccess)
                return bail(IGS_ENOMEM);
            std::memset(bt->run_host, 0, sizeof(Run));
            if (cudaEventCreate(&bt->ev0) != cudaSuccess || cudaEventCreate(&bt->ev1) != cudaSuccess)
                return bail(IGS_ECUDA);
            cudaStream_t s = bt->stream;
            {
                SellHost sh;
                build_sell(count, sys_ptr, rowptr, loc.data(), vals, sh);
                rc = upload_sell(sh, &bt->sell_off, &bt->sys_slice0, &bt->sell_col, &bt->sell_val, s);
                if (rc != IGS_OK) return bail(rc);
                if (cudaStreamSynchronize(s) != cudaSuccess) return bail(IGS_ECUDA);
            }
            if (cudaMemcpyAsync(bt->sys_row0, sys_ptr, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(bt->order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(bt->order_sample, sample.data(), sizeof(int) * sample.size(), cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(bt->b_tune, btune.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s) ||
                cudaMemsetAsync(bt->vslots, 0, sizeof(double) * (size_t)bt->slots_alloc * bt->slot_stride, s))
                return bail(IGS_ECUDA);

            // ||A_s||_2: given, or estimated on the GPU by power iteration on A_s^T A_s
            bt->normA_host.assign((size_t)count, 0.0);
            if (opts->A_norm2) {
                std::memcpy(bt->normA_host.data(), opts->A_norm2, sizeof(double) * count);
                if (cudaMemcpyAsync(bt->normA, opts->A_norm2, sizeof(double) * count, cudaMemcpyHostToDevice, s))
                    return bail(IGS_ECUDA);
            } else {
                // A^T in the same block-diagonal CSR form (local column indices)
                std::vector<int64_t> trp((size_t)N + 1, 0);
                for (int64_t k = 0; k < nnz; ++k) trp[(size_t)(colind[k] + 1)]++;
                for (int64_t i = 0; i < N; ++i) trp[(size_t)i + 1] += trp[(size_t)i];
                std::vector<int64_t> fillp(trp.begin(), trp.end() - 1);
                std::vector<int> tci((size_t)(nnz ? nnz : 1));
                std::vector<double> tva((size_t)(nnz ? nnz : 1));
                for (int sidx = 0; sidx < count; ++sidx)
                    for (int64_t i = sys_ptr[sidx]; i < sys_ptr[sidx + 1]; ++i)
                        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                            const int64_t dst = fillp[(size_t)colind[k]]++;
                            tci[(size_t)dst] = (int)(i - sys_ptr[sidx]);
                            tva[(size_t)dst] = vals[k];
                        }
                SellHost th;
                build_sell(count, sys_ptr, trp.data(), tci.data(), tva.data(), th);
                int64_t *at_rp = nullptr;
                int *at_ci = nullptr;
                double *at_va = nullptr;
                int urc = upload_sell(th, &at_rp, nullptr, &at_ci, &at_va, s);
                const int iters = opts->norm2_iters > 0 ? opts->norm2_iters : 100;
                cudaError_t e = urc == IGS_OK ? cudaSuccess : cudaErrorMemoryAllocation;
                if (e == cudaSuccess) {
                    const int grid = std::min(count, bt->slots_alloc);
                    k_batch_norm2<<<grid, 256, bt->smem, s>>>(make_args(bt), at_rp, at_ci, at_va, count, iters, bt->normA);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(bt->normA_host.data(), bt->normA, sizeof(double) * count, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                cudaFree(at_rp);
                cudaFree(at_ci);
                cudaFree(at_va);
                if (e != cudaSuccess) return bail(IGS_ECUDA);
            }
            if (cudaStreamSynchronize(s) != cudaSuccess) return bail(IGS_ECUDA);

            // launch configuration: given, else tuned
            if (opts->block_threads != 0 && opts->blocks_per_sm != 0) {
                bt->threads = opts->block_threads;
                bt->bpsm = opts->blocks_per_sm;
                int maxb = 0;
                rc = max_blocks_per_sm(bt, bt->threads, &maxb);
                if (rc != IGS_OK) return bail(rc);
                if (maxb < 1) return bail(IGS_EINVAL);
            } else {
                rc = autotune(bt, 2, 1e-12, 20);
                if (rc != IGS_OK) return bail(rc);
            }
            *out = bt;
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

extern "C" void igs_batch_destroy(igs_batch *bt)
{
    if (!bt) return;
    cudaSetDevice(bt->device);
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    for (auto &g : bt->graphs) cudaGraphExecDestroy(g.exec);
    cudaFree(bt->sys_row0);
    cudaFree(bt->sell_off);
    cudaFree(bt->sys_slice0);
    cudaFree(bt->sell_col);
    cudaFree(bt->sell_val);
    cudaFree(bt->order);
    cudaFree(bt->order_sample);
    cudaFree(bt->normA);
    cudaFree(bt->vslots);
    cudaFree(bt->queue);
    cudaFree(bt->summary);
    cudaFree(bt->run_dev);
    cudaFree(bt->b_dev);
    cudaFree(bt->x_dev);
    cudaFree(bt->x0_dev);
    cudaFree(bt->b_tune);
    cudaFree(bt->beta_dev);
    cudaFree(bt->status_dev);
    cudaFree(bt->cycles_dev);
    cudaFree(bt->steps_dev);
    if (bt->run_host) cudaFreeHost(bt->run_host);
    if (bt->summary_host) cudaFreeHost(bt->summary_host);
    if (bt->ev0) cudaEventDestroy(bt->ev0);
    if (bt->ev1) cudaEventDestroy(bt->ev1);
    if (bt->own_stream && bt->stream) cudaStreamDestroy(bt->stream);
    delete bt;
}

extern "C" int igs_batch_solve(igs_batch *bt, const double *b, const double *x0,
                               const igs_batch_solve_opts *opts, igs_batch_result *res)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!bt) return IGS_EINVAL;
            if (!b || !opts || !res || !res->x) return fail(bt, IGS_EINVAL, "null argument");
            if (opts->gs_iters < 1 || opts->gs_iters > 2 || !(opts->tol_beta >= 0.0) || opts->max_restarts < 1)
                return fail(bt, IGS_EINVAL, "invalid solve options");
            if (cudaSetDevice(bt->device) != cudaSuccess) return fail(bt, IGS_ECUDA, "cudaSetDevice");
            cudaStream_t s = bt->stream;
            const bool dev = opts->inputs_on_device != 0;
            Run *r = bt->run_host;
            std::memset(r, 0, sizeof(Run));
            r->order = bt->order;
            r->count = bt->count;
            r->gs = opts->gs_iters;
            r->max_cycles = opts->max_restarts;
            r->tol = opts->tol_beta;
            r->x0_given = x0 ? 1 : 0;
            const size_t vb = sizeof(double) * (size_t)bt->N;
            if (dev) {
                r->b = b;
                r->x0 = x0;
                r->x = res->x;
                r->beta = res->beta;
                r->status = res->status;
                r->steps = res->steps;
                r->cycles = res->cycles;
            } else {
                BT_CUDA(cudaMemcpyAsync(bt->b_dev, b, vb, cudaMemcpyHostToDevice, s), "copy b");
                if (x0) BT_CUDA(cudaMemcpyAsync(bt->x0_dev, x0, vb, cudaMemcpyHostToDevice, s), "copy x0");
                r->b = bt->b_dev;
                r->x0 = x0 ? bt->x0_dev : nullptr;
                r->x = bt->x_dev;
                r->beta = bt->beta_dev;
                r->status = bt->status_dev;
                r->steps = bt->steps_dev;
                r->cycles = bt->cycles_dev;
            }
            float ms = 0.f;
            int rc = launch(bt, bt->threads, bt->bpsm, &ms);
            if (rc != IGS_OK) return rc;
            if (!dev) {
                BT_CUDA(cudaMemcpyAsync(res->x, bt->x_dev, vb, cudaMemcpyDeviceToHost, s), "copy x");
                if (res->beta)
                    BT_CUDA(cudaMemcpyAsync(res->beta, bt->beta_dev, sizeof(double) * bt->count, cudaMemcpyDeviceToHost, s),
                            "copy beta");
                if (res->status)
                    BT_CUDA(cudaMemcpyAsync(res->status, bt->status_dev, sizeof(int) * bt->count, cudaMemcpyDeviceToHost, s),
                            "copy status");
                if (res->steps)
                    BT_CUDA(cudaMemcpyAsync(res->steps, bt->steps_dev, sizeof(int64_t) * bt->count, cudaMemcpyDeviceToHost, s),
                            "copy steps");
                if (res->cycles)
                    BT_CUDA(cudaMemcpyAsync(res->cycles, bt->cycles_dev, sizeof(int) * bt->count, cudaMemcpyDeviceToHost, s),
                            "copy cycles");
                BT_CUDA(cudaStreamSynchronize(s), "copy results");
            }
            const unsigned long long *sum = bt->summary_host;
            res->total_steps = (int64_t)sum[0];
            // summary[1 + status + 6]
            res->n_ok = (int)sum[1 + IGS_OK + 6];
            res->n_not_converged = (int)sum[1 + IGS_NOT_CONVERGED + 6];
            res->n_breakdown = (int)sum[1 + IGS_BREAKDOWN + 6];
            res->n_numeric = (int)sum[1 + IGS_ENUMERIC + 6];
            res->device_ms = ms;
            if (res->n_numeric > 0) return IGS_ENUMERIC;
            if (res->n_not_converged > 0) return IGS_NOT_CONVERGED;
            if (res->n_breakdown > 0) return IGS_BREAKDOWN;
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

extern "C" int igs_batch_set_config(igs_batch *bt, int block_threads, int blocks_per_sm)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!bt) return IGS_EINVAL;
            if (!valid_threads(block_threads) || blocks_per_sm < 1 ||
                bt->num_sms * blocks_per_sm > bt->slots_alloc)
                return fail(bt, IGS_EINVAL, "invalid launch configuration");
            int maxb = 0;
            int rc = max_blocks_per_sm(bt, block_threads, &maxb);
            if (rc != IGS_OK) return rc;
            if (blocks_per_sm > maxb) return fail(bt, IGS_EINVAL, "blocks_per_sm above occupancy");
            bt->threads = block_threads;
            bt->bpsm = blocks_per_sm;
            return IGS_OK;
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

extern "C" int igs_batch_tune(igs_batch *bt, int gs_iters, double tol_beta, int max_restarts)
{
    // no C++ exception crosses the C interface (allocation failures become IGS_ENOMEM)
    try {
        return [&]() -> int {
            if (!bt) return IGS_EINVAL;
            if (gs_iters < 1 || gs_iters > 2 || !(tol_beta >= 0.0) || max_restarts < 1)
                return fail(bt, IGS_EINVAL, "invalid tuning options");
            if (cudaSetDevice(bt->device) != cudaSuccess) return fail(bt, IGS_ECUDA, "cudaSetDevice");
            return autotune(bt, gs_iters, tol_beta, max_restarts);
        }();
    } catch (const std::bad_alloc &) {
        return IGS_ENOMEM;
    } catch (...) {
        return IGS_EINVAL;
    }
}

extern "C" int igs_batch_get_info(const igs_batch *bt, igs_batch_info *info)
{
    if (!bt || !info) return IGS_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->count = bt->count;
    info->total_rows = bt->N;
    info->nnz = bt->nnz;
    info->max_rows = bt->nmax;
    info->restart_m = bt->m;
    info->block_threads = bt->threads;
    info->blocks_per_sm = bt->bpsm;
    info->num_sms = bt->num_sms;
    info->smem_bytes = (int64_t)bt->smem;
    info->basis_bytes = (int64_t)bt->slots_alloc * bt->slot_stride * (int64_t)sizeof(double);
    const int nt = (int)std::min<size_t>(bt->tune.size(), IGS_BATCH_MAX_TUNE);
    info->n_tune = nt;
    for (int i = 0; i < nt; ++i) info->tune[i] = bt->tune[(size_t)i];
    return IGS_OK;
}

extern "C" int igs_batch_get_norms(const igs_batch *bt, double *out)
{
    if (!bt || !out) return IGS_EINVAL;
    std::memcpy(out, bt->normA_host.data(), sizeof(double) * bt->count);
    return IGS_OK;
}

extern "C" const char *igs_batch_last_error(const igs_batch *bt)
{
    if (!bt) return "null batch";
    return bt->err.c_str();
}
