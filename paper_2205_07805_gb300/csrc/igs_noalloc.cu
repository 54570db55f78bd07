// Block multi-dot that allocates no device memory (igs_block_dots_static in include/igs.h).
//
// Who needs this: callers that are not allowed to call cudaMalloc -- a host application
// that owns all device memory through its own pool and forbids plug-ins from allocating,
// code that runs while another thread captures a CUDA graph in global capture mode (where
// cudaMalloc is an error), and latency-critical loops that cannot afford cudaMalloc's
// implicit device synchronisation.  They pass their own inputs and outputs; the per-block
// partial sums, which the regular path keeps in a context workspace, live here in a fixed
// file-scope device array instead.
//
// The scratch array: kStaticScratch doubles (128 KiB), allocated by the CUDA runtime when
// the library is loaded on a device and held by every device that loads the library until
// the process exits.  All calls share it and it keeps the last call's contents; nothing has
// to start at zero, because each call writes every partial it later reads.  Two calls whose
// GPU work overlaps (different streams or threads without ordering) race on it.
#include "../../include/igs.h"
#include "igs_internal.h"

#include <mutex>

namespace {

constexpr int64_t kStaticScratch = 16384;  // doubles
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_dots_scratch[kStaticScratch];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// out[v] = sum over rb of part[rb * nv + v] (the multi-dot's row-block-major partials),
// fixed order (one block).
__global__ void __launch_bounds__(256) k_sum_partials(const double *__restrict__ part, int nv, int nrb,
                                                     double *__restrict__ out)
{
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        double a0 = 0.0, a1 = 0.0;
        int rb = 0;
        for (; rb + 1 < nrb; rb += 2) {
            a0 += part[(int64_t)rb * nv + v];
            a1 += part[(int64_t)(rb + 1) * nv + v];
        }
        if (rb < nrb) a0 += part[(int64_t)rb * nv + v];
        out[v] = a0 + a1;
    }
}

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return IGS_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dots_scratch) != cudaSuccess || !p) return IGS_ECUDA;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return IGS_OK;
}

// Largest p one launch can take on a GPU with `sms` SMs: the plan's column groups (at most
// kDotsBlocksPerSM blocks per SM) of at most kDotsMaxGroupCols columns each, and the partial
// sums of the widest plan (one row block) within the scratch array for two vectors.
int64_t max_columns(int sms)
{
    const int64_t by_groups = (int64_t)sms * igs::kDotsBlocksPerSM * igs::kDotsMaxGroupCols;
    const int64_t by_scratch = kStaticScratch / 2;
    return by_groups < by_scratch ? by_groups : by_scratch;
}

}  // namespace

extern "C" int igs_block_dots_static(const double *V, int64_t ldv, int p, int64_t n, const double *x0,
                                     const double *x1, double *out, void *stream)
{
    if (!V || !x0 || !out || p < 1 || n < 4 || (n & 3) != 0 || ldv < n || (ldv & 1) != 0)
        return IGS_EINVAL;
    if (((uintptr_t)V | (uintptr_t)x0 | (uintptr_t)(x1 ? x1 : x0)) & 15) return IGS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IGS_ECUDA;
    double *scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc != IGS_OK) return rc;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return IGS_ECUDA;
    igs::Workspace w;
    w.n = n;
    w.ld = ldv;
    w.num_sms = sms;
    w.V = const_cast<double *>(V);
    w.part = scratch;
    const int nq = x1 ? 2 : 1;
    // The multi-dot kernel gives each column group at most kDotsMaxGroupCols columns; the
    // plan caps the group count at 3 blocks per SM, so p beyond 3 * SMs * kDotsMaxGroupCols
    // (3648 on a 152-SM GPU) cannot be computed and is rejected before anything launches.
    if ((int64_t)p > max_columns(sms)) return IGS_EINVAL;
    const igs::DotsPlan pl = igs::plan_dots(w, p);
    if ((p + pl.groups - 1) / pl.groups > igs::kDotsMaxGroupCols) return IGS_EINVAL;
    if ((int64_t)nq * p * pl.rblocks > kStaticScratch) return IGS_EINVAL;  // beyond the fixed scratch
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    igs::DotsPlan used{};
    if (igs::launch_dots(w, p, x0, x1, false, s, &used) != cudaSuccess) return IGS_ECUDA;
    k_sum_partials<<<1, 256, 0, s>>>(scratch, nq * p, used.rblocks, out);
    if (cudaGetLastError() != cudaSuccess) return IGS_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return IGS_ECUDA;
    return IGS_OK;
}
