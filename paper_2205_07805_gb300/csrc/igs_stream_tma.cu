// TMA-pipelined basis kernels of the GB300 IGS-GMRES library (sm_103a).
//
// Both kernels stream tiles of TR rows x p basis columns through shared memory with 1-D bulk
// copies (cp.async.bulk ... mbarrier::complete_tx), double buffered: while the block computes
// on tile j, the copies of tile j+1 are in flight, so HBM latency is hidden by the copy
// engine rather than by thread count.  This matters because the FP64 pipe, not HBM, bounds
// these kernels on GB300: few threads (4 warps, one per sub-partition) are enough to keep it
// busy once operands sit in shared memory.
//
//  * k_update_dots_tma -- Alg. 4.1 steps 7, 11, 13 and the partial sums of step 14 (two
//    Gauss-Seidel iterations): v_{k-1} = w_{k-1}/gamma in place, u = z/gamma - V r^(1),
//    partials of V^T u.  Each basis element is read once from HBM and feeds two FMAs.
//  * k_update_tma -- step 16 (and step 13 with one iteration):
//    out = a*src - V c, optionally normalising column p-1 in place first.
//
// Every mbarrier wait is bounded: on timeout the block records IGS status -5 in the device
// state, waits (bounded) for its own copies in flight and returns.
#include "igs_internal.h"

#include <cstdint>

namespace igs {

namespace {

constexpr uint32_t kWaitSpins = 1u << 20;

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses (made visible to it by a
// block barrier) before its later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            saddr(dst)),
        "l"(src), "r"(bytes), "r"(saddr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < kWaitSpins; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Tile geometry: TR rows per tile (16, 32 or 64, chosen per launch so that several blocks
// fit per SM); column c of a stage starts at c * (TR + 2) doubles -- 16-byte aligned, and
// consecutive columns land 4 banks apart, so column-per-thread reads conflict at most 4-way.
constexpr int kThreads = 128;        // 4 warps, one per sub-partition

__device__ __forceinline__ uint32_t round16(uint32_t bytes) { return (bytes + 15u) & ~15u; }

// Issue the bulk copies of one tile into a stage (called by all 32 lanes of warp 0): columns
// 0..p-1 of V for rows [row0, row0+len) and, when extra != nullptr, the same rows of `extra`
// after the columns.  Lane 0 arms the barrier with the expected byte count, then the lanes
// issue the copies in parallel (serial issue by one thread would stall its warp, and with it
// the tile, for ~p copy instructions).  Copy sizes are rounded up to 16 bytes (the vectors
// are padded to a multiple of 32 rows, so the rounding never leaves the allocation).
template <int kColStride>
__device__ __forceinline__ void issue_tile_warp(double *stage, const double *V, int64_t ld, int p,
                                                int64_t row0, int len, const double *extra,
                                                uint64_t *bar, int lane)
{
    const uint32_t bytes = round16((uint32_t)len * 8u);
    const int ncopies = p + (extra ? 1 : 0);
    if (lane == 0) mbar_expect_tx(bar, bytes * (uint32_t)ncopies);
    __syncwarp();
    for (int c = lane; c < ncopies; c += 32) {
        const double *src = c < p ? V + (int64_t)c * ld + row0 : extra + row0;
        bulk_g2s(stage + (size_t)c * kColStride, src, bytes, bar);
    }
}

__device__ void record_timeout(DevState *st)
{
    st->stop_reason = -5;
    st->halt = 1;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Fused steps 7, 11, 13 + step-14 partial sums.  Grid: one block per row range (1-2 per SM).
// Shared memory: 2 stages of (p+1) column segments, coefficients, u of the tile, tree space.
// Output: u, block partials bpart[blk*p + c], and (by the last block of each group of
// `group` blocks) group partials gpart[g*p + c].
// ------------------------------------------------------------------------------------------
template <int kTR>
__global__ void __launch_bounds__(kThreads)
k_update_dots_tma(double *V, int64_t ld, int p, int64_t n, int64_t rows_per_block,
                  const double *__restrict__ coef, const double *__restrict__ z, double *__restrict__ u,
                  double *__restrict__ bpart, double *__restrict__ gpart, int *__restrict__ counters,
                  int group, DevState *st)
{
    IGS_PDL_ENTER();
    if (st->halt) return;
    constexpr int kColStride = kTR + 2;
    constexpr int TPR = kThreads / kTR;  // threads per row in the row phase (2, 4 or 8)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);                 // 2 barriers
    double *stages = reinterpret_cast<double *>(smem_raw + 128);             // 2 stages
    const size_t stage_d = (size_t)(p + 1) * kColStride;
    double *sc = stages + 2 * stage_d;                                        // p coefficients
    double *us = sc + p;                                                      // kTR
    double *red = us + kTR;                                                   // kThreads
    __shared__ int s_last, s_fail;
    const int t = threadIdx.x;
    const double ig = st->inv_gamma;
    const int64_t r_lo = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r_hi = r_lo + rows_per_block < n ? r_lo + rows_per_block : n;
    const int ntiles = r_lo < r_hi ? (int)((r_hi - r_lo + kTR - 1) / kTR) : 0;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_fail = 0;
    }
    for (int c = t; c < p; c += kThreads) sc[c] = coef[c];
    __syncthreads();
    if (t < 32 && ntiles > 0)
        issue_tile_warp<kColStride>(stages, V, ld, p, r_lo, (int)(r_hi - r_lo < kTR ? r_hi - r_lo : kTR), z, &bars[0], t);
    // column-phase mapping: thread per column, with S row slices when p <= kThreads/2
    const bool narrow = p <= kThreads;
    const int S = narrow ? kThreads / p : 1;
    const int cmine = narrow ? t % p : t;
    const int sl = narrow ? t / p : 0;
    const bool act = narrow ? sl < S : true;
    double a0 = 0.0, a1 = 0.0;
    int issued = ntiles > 0 ? 1 : 0, fail_j = -1;
    for (int j = 0; j < ntiles; ++j) {
        const int s = j & 1;
        const int64_t row0 = r_lo + (int64_t)j * kTR;
        const int len = (int)(r_hi - row0 < kTR ? r_hi - row0 : kTR);
        double *stg = stages + s * stage_d;
        if (j + 1 < ntiles) {
            if (t < 32) {
                const int64_t nrow0 = row0 + kTR;
                fence_proxy_async();
                issue_tile_warp<kColStride>(stages + (s ^ 1) * stage_d, V, ld, p, nrow0,
                                (int)(r_hi - nrow0 < kTR ? r_hi - nrow0 : kTR), z, &bars[s ^ 1], t);
            }
            ++issued;
        }
        if (!mbar_wait(&bars[s], (uint32_t)((j >> 1) & 1))) {
            if (t == 0) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) {
            fail_j = j;
            break;
        }
        // step 7: normalise the lagged column in shared memory and in place in HBM
        double *lastc = stg + (size_t)(p - 1) * kColStride;
        if (t < len) {
            const double v = lastc[t] * ig;
            lastc[t] = v;
            V[(int64_t)(p - 1) * ld + row0 + t] = v;
        }
        __syncthreads();
        // steps 11, 13: u = z/gamma - V r^(1); TPR threads per row split the columns
        {
            const int r = t / TPR, h = t % TPR;
            double b0 = 0.0, b1 = 0.0;
            if (r < len) {
                int c = h;
                for (; c + TPR < p; c += 2 * TPR) {
                    b0 = fma(stg[(size_t)c * kColStride + r], sc[c], b0);
                    b1 = fma(stg[(size_t)(c + TPR) * kColStride + r], sc[c + TPR], b1);
                }
                if (c < p) b0 = fma(stg[(size_t)c * kColStride + r], sc[c], b0);
            }
            double acc = b0 + b1;
#pragma unroll
            for (int o = 1; o < TPR; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (r < len && h == 0) {
                const double zi = stg[(size_t)p * kColStride + r];
                const double ui = fma(ig, zi, -acc);
                u[row0 + r] = ui;
                us[r] = ui;
            }
        }
        __syncthreads();
        // partial sums of step 14 from the same tile
        if (narrow) {
            if (act) {
                const int rs = sl * len / S, re = (sl + 1) * len / S;
                const double *tc = stg + (size_t)cmine * kColStride;
                int r = rs;
                for (; r + 1 < re; r += 2) {
                    a0 = fma(tc[r], us[r], a0);
                    a1 = fma(tc[r + 1], us[r + 1], a1);
                }
                if (r < re) a0 = fma(tc[r], us[r], a0);
            }
        } else {
            const double *t0c = stg + (size_t)t * kColStride;
            const double *t1c = stg + (size_t)(t + kThreads) * kColStride;
            const bool second = t + kThreads < p;
            for (int r = 0; r < len; ++r) {
                a0 = fma(t0c[r], us[r], a0);
                if (second) a1 = fma(t1c[r], us[r], a1);
            }
        }
        __syncthreads();
    }
    if (fail_j >= 0) {
        // drain (bounded): only tile fail_j and the one issued after it can be in flight
        if (t == 0) {
            for (int j = fail_j; j < issued && j <= fail_j + 1; ++j)
                mbar_wait(&bars[j & 1], (uint32_t)((j >> 1) & 1));
            record_timeout(st);
        }
        return;
    }
    // block partials (slice tree when narrow)
    if (narrow) {
        red[t] = a0 + a1;
        int Sp = S;
        while (Sp > 1) {
            const int h = (Sp + 1) >> 1;
            __syncthreads();
            if (act && sl < Sp - h) red[t] += red[t + h * p];
            Sp = h;
        }
        __syncthreads();
        if (act && sl == 0) bpart[(int64_t)blockIdx.x * p + cmine] = red[t];
    } else {
        if (t < p) bpart[(int64_t)blockIdx.x * p + t] = a0;
        if (t + kThreads < p) bpart[(int64_t)blockIdx.x * p + t + kThreads] = a1;
    }
    // group combine by the last block of each group to finish (no block waits)
    __threadfence();
    __syncthreads();
    const int g = blockIdx.x / group;
    const int gb0 = g * group;
    const int gb1 = gb0 + group < (int)gridDim.x ? gb0 + group : (int)gridDim.x;
    if (t == 0) {
        const int prev = atomicAdd(&counters[g], 1);
        s_last = prev == gb1 - gb0 - 1;
        if (s_last) counters[g] = 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int c = t; c < p; c += kThreads) {
        double s0 = 0.0, s1 = 0.0;
        int b = gb0;
        for (; b + 1 < gb1; b += 2) {
            s0 += __ldcg(bpart + (int64_t)b * p + c);
            s1 += __ldcg(bpart + (int64_t)(b + 1) * p + c);
        }
        if (b < gb1) s0 += __ldcg(bpart + (int64_t)b * p + c);
        gpart[(int64_t)g * p + c] = s0 + s1;
    }
}

// ------------------------------------------------------------------------------------------
// out = a*src - V[:, 0:p] coef, tile-pipelined.  With norm_last, column p-1 is first scaled
// in place by st->inv_gamma and a = st->inv_gamma.
// ------------------------------------------------------------------------------------------
template <int kTR>
__global__ void __launch_bounds__(kThreads)
k_update_tma(double *V, int64_t ld, int p, int64_t n, int64_t rows_per_block,
             const double *__restrict__ coef, double alpha, const double *src, double *out,
             int norm_last, DevState *st)
{
    IGS_PDL_ENTER();
    if (st->halt) return;
    constexpr int kColStride = kTR + 2;
    constexpr int TPR = kThreads / kTR;  // threads per row (2, 4 or 8)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    double *stages = reinterpret_cast<double *>(smem_raw + 128);
    const size_t stage_d = (size_t)(p + 1) * kColStride;
    double *sc = stages + 2 * stage_d;
    __shared__ int s_fail;
    const int t = threadIdx.x;
    const double a = norm_last ? st->inv_gamma : alpha;
    const int64_t r_lo = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r_hi = r_lo + rows_per_block < n ? r_lo + rows_per_block : n;
    const int ntiles = r_lo < r_hi ? (int)((r_hi - r_lo + kTR - 1) / kTR) : 0;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_fail = 0;
    }
    for (int c = t; c < p; c += kThreads) sc[c] = coef[c];
    __syncthreads();
    if (t < 32 && ntiles > 0)
        issue_tile_warp<kColStride>(stages, V, ld, p, r_lo, (int)(r_hi - r_lo < kTR ? r_hi - r_lo : kTR), src, &bars[0], t);
    int issued = ntiles > 0 ? 1 : 0, fail_j = -1;
    for (int j = 0; j < ntiles; ++j) {
        const int s = j & 1;
        const int64_t row0 = r_lo + (int64_t)j * kTR;
        const int len = (int)(r_hi - row0 < kTR ? r_hi - row0 : kTR);
        double *stg = stages + s * stage_d;
        if (j + 1 < ntiles) {
            if (t < 32) {
                const int64_t nrow0 = row0 + kTR;
                fence_proxy_async();
                issue_tile_warp<kColStride>(stages + (s ^ 1) * stage_d, V, ld, p, nrow0,
                                (int)(r_hi - nrow0 < kTR ? r_hi - nrow0 : kTR), src, &bars[s ^ 1], t);
            }
            ++issued;
        }
        if (!mbar_wait(&bars[s], (uint32_t)((j >> 1) & 1))) {
            if (t == 0) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) {
            fail_j = j;
            break;
        }
        if (norm_last) {
            double *lastc = stg + (size_t)(p - 1) * kColStride;
            if (t < len) {
                const double v = lastc[t] * a;
                lastc[t] = v;
                V[(int64_t)(p - 1) * ld + row0 + t] = v;
            }
            __syncthreads();
        }
        const int r = t / TPR, h = t % TPR;
        double b0 = 0.0, b1 = 0.0;
        if (r < len) {
            int c = h;
            for (; c + TPR < p; c += 2 * TPR) {
                b0 = fma(stg[(size_t)c * kColStride + r], sc[c], b0);
                b1 = fma(stg[(size_t)(c + TPR) * kColStride + r], sc[c + TPR], b1);
            }
            if (c < p) b0 = fma(stg[(size_t)c * kColStride + r], sc[c], b0);
        }
        double acc = b0 + b1;
#pragma unroll
        for (int o = 1; o < TPR; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (r < len && h == 0) out[row0 + r] = fma(a, stg[(size_t)p * kColStride + r], -acc);
        __syncthreads();
    }
    if (fail_j >= 0 && t == 0) {
        for (int j = fail_j; j < issued && j <= fail_j + 1; ++j) mbar_wait(&bars[j & 1], (uint32_t)((j >> 1) & 1));
        record_timeout(st);
    }
}

// ------------------------------------------------------------------------------------------
// Launchers.  The tile height is chosen per launch: the tallest of 64/32/16 rows whose
// double-buffered stage still lets at least four blocks share an SM (16 warps).
// ------------------------------------------------------------------------------------------
static size_t smem_for(int p, int tr, bool with_dots)
{
    size_t d = 2 * (size_t)(p + 1) * (tr + 2) + (size_t)p;
    if (with_dots) d += tr + kThreads;
    return 128 + sizeof(double) * d;
}

static int pick_tr(int p, bool with_dots)
{
    const size_t per_sm = 228 * 1024;
    for (int tr : {64, 32})
        if (4 * (smem_for(p, tr, with_dots) + 1024) <= per_sm) return tr;
    return 16;
}

size_t tma_smem(int p, bool with_dots)
{
    return smem_for(p, pick_tr(p, with_dots), with_dots);
}

bool tma_fits(int p)
{
    return smem_for(p, 16, true) <= kTmaMaxSmem;
}

static int tma_blocks(const Workspace &w, const void *fn, size_t smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (per_sm > kTmaMaxBlocksPerSM) per_sm = kTmaMaxBlocksPerSM;
    return w.num_sms * per_sm;
}

static int64_t tma_rows(int64_t n, int blocks)
{
    int64_t rows = (n + blocks - 1) / blocks;
    return (rows + 1) & ~int64_t(1);  // even: every tile starts 16-byte aligned
}

template <int TR>
static cudaError_t launch_ud(const Workspace &w, int p, const double *coef, const double *z, double *u,
                             cudaStream_t s, int *ngroups_out)
{
    const size_t smem = smem_for(p, TR, true);
    const int blocks = tma_blocks(w, (const void *)k_update_dots_tma<TR>, smem);
    const int64_t rows = tma_rows(w.n, blocks);
    const int nblk = (int)((w.n + rows - 1) / rows);
    launch_k(false, k_update_dots_tma<TR>, dim3(nblk), dim3(kThreads), smem, s, w.V, w.ld, p, w.n, rows, coef, z, u, w.bpart, w.part,
                                                       w.counters, kFusedGroup, w.st);
    if (ngroups_out) *ngroups_out = (nblk + kFusedGroup - 1) / kFusedGroup;
    return cudaGetLastError();
}

template <int TR>
static cudaError_t launch_u(const Workspace &w, int p, const double *coef, double alpha, const double *src,
                            double *out, bool norm_last, cudaStream_t s)
{
    const size_t smem = smem_for(p, TR, false);
    const int blocks = tma_blocks(w, (const void *)k_update_tma<TR>, smem);
    const int64_t rows = tma_rows(w.n, blocks);
    const int nblk = (int)((w.n + rows - 1) / rows);
    launch_k(false, k_update_tma<TR>, dim3(nblk), dim3(kThreads), smem, s, w.V, w.ld, p, w.n, rows, coef, alpha, src, out,
                                                  norm_last ? 1 : 0, w.st);
    return cudaGetLastError();
}

cudaError_t launch_update_dots_tma(const Workspace &w, int p, const double *coef, const double *z,
                                   double *u, cudaStream_t s, int *ngroups_out)
{
    switch (pick_tr(p, true)) {
    case 64: return launch_ud<64>(w, p, coef, z, u, s, ngroups_out);
    case 32: return launch_ud<32>(w, p, coef, z, u, s, ngroups_out);
    default: return launch_ud<16>(w, p, coef, z, u, s, ngroups_out);
    }
}

cudaError_t launch_update_tma(const Workspace &w, int p, const double *coef, double alpha,
                              const double *src, double *out, bool norm_last, cudaStream_t s)
{
    switch (pick_tr(p, false)) {
    case 64: return launch_u<64>(w, p, coef, alpha, src, out, norm_last, s);
    case 32: return launch_u<32>(w, p, coef, alpha, src, out, norm_last, s);
    default: return launch_u<16>(w, p, coef, alpha, src, out, norm_last, s);
    }
}

template <int TR>
static cudaError_t set_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_update_dots_tma<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTmaMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_update_tma<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaMaxSmem);
    return e;
}

cudaError_t configure_tma_kernels()
{
    cudaError_t e = set_attrs<64>();
    if (e == cudaSuccess) e = set_attrs<32>();
    if (e == cudaSuccess) e = set_attrs<16>();
    return e;
}

}  // namespace igs
