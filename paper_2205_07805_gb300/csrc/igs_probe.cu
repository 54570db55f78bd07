// Arithmetic-pipe probe (igs_probe_fma in include/igs.h): the FP64 and FP32 FMA throughput of
// the GPU, the best over a few launch shapes of independent FMA chains on every SM.  The FP64
// rate is the ceiling of this library's FP64 streaming kernels on GB300 (see igs_kernels.cu),
// so the benchmark reports it beside the unit-count peak it uses for the FP64 roofline.
#include "../../include/igs.h"

#include <cuda_runtime.h>

namespace {

constexpr int kProbeThreads = 256;

// CH independent FMA chains per thread, each a[c] = a[c] * m + k (one FMA), unrolled 4 times
// per loop trip so that loop control is a small share of the issue slots.
template <typename T, int CH>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T seed, T *sink)
{
    T a[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, k = (T)1e-7;
    for (int it = 0; it < iters; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) a[c] = a[c] * m + k;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += a[c];
    if (s == (T)-1) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

// FMAs per second of one launch configuration (a warm-up launch, then one timed launch).
template <typename T, int CH>
int probe_one(int blocks, int iters, cudaStream_t st, T *sink, double *fma_per_s)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return IGS_ECUDA;
    int rc = IGS_OK;
    k_fma_probe<T, CH><<<blocks, kProbeThreads, 0, st>>>(iters / 8, (T)1, sink);
    cudaEventRecord(e0, st);
    k_fma_probe<T, CH><<<blocks, kProbeThreads, 0, st>>>(iters, (T)1, sink);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
        rc = IGS_ECUDA;
    else
        *fma_per_s = (double)blocks * kProbeThreads * CH * (double)iters / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// The best of several occupancies (2, 4, 8 blocks of 256 threads per SM) and chain counts
// (4, 8, 16 per thread): the pipe's throughput, not one configuration's.
template <typename T>
int probe(int sms, int iters, cudaStream_t st, T *sink, double *fma_per_s)
{
    double best = 0.0;
    for (int bps : {2, 4, 8}) {
        double r4 = 0.0, r8 = 0.0, r16 = 0.0;
        int rc = probe_one<T, 4>(bps * sms, iters, st, sink, &r4);
        if (rc == IGS_OK) rc = probe_one<T, 8>(bps * sms, iters / 2, st, sink, &r8);
        if (rc == IGS_OK) rc = probe_one<T, 16>(bps * sms, iters / 4, st, sink, &r16);
        if (rc != IGS_OK) return rc;
        best = r4 > best ? r4 : best;
        best = r8 > best ? r8 : best;
        best = r16 > best ? r16 : best;
    }
    *fma_per_s = best;
    return IGS_OK;
}

}  // namespace

extern "C" int igs_probe_fma(int device, double *fp64_fma_per_s, double *fp32_fma_per_s)
{
    if (!fp64_fma_per_s || !fp32_fma_per_s) return IGS_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return IGS_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
        return IGS_ECUDA;
    cudaStream_t st = nullptr;
    double *sink = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return IGS_ECUDA;
    int rc = cudaMalloc(&sink, sizeof(double) * (size_t)(8 * sms)) == cudaSuccess ? IGS_OK : IGS_ENOMEM;
    // each FP64 launch about 30-120 ms at GB300's rate; FP32 with 16 times the iterations
    if (rc == IGS_OK) rc = probe<double>(sms, 1 << 14, st, sink, fp64_fma_per_s);
    if (rc == IGS_OK) rc = probe<float>(sms, 1 << 18, st, reinterpret_cast<float *>(sink), fp32_fma_per_s);
    cudaFree(sink);
    cudaStreamDestroy(st);
    return rc;
}
