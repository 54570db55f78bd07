// Arithmetic-pipe probe (igs_probe_fma in include/igs.h): the FP64 and FP32 FMA throughput of
// the GPU, measured with every SM full of independent FMA chains.  The FP64 rate is the
// ceiling of this library's FP64 streaming kernels on GB300 (see igs_kernels.cu), so the
// benchmark reports it beside the unit-count peak it uses for the FP64 roofline.
#include "../../include/igs.h"

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T seed, T *sink)
{
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, k = (T)1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] * m + k;  // one FMA each
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-1) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

template <typename T>
int probe(int blocks, int iters, cudaStream_t st, T *sink, double *fma_per_s)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return IGS_ECUDA;
    int rc = IGS_OK;
    k_fma_probe<T><<<blocks, kProbeThreads, 0, st>>>(iters / 8, (T)1, sink);  // warm-up
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, kProbeThreads, 0, st>>>(iters, (T)1, sink);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
        rc = IGS_ECUDA;
    else
        *fma_per_s = (double)blocks * kProbeThreads * kChains * (double)iters / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int igs_probe_fma(int device, double *fp64_fma_per_s, double *fp32_fma_per_s)
{
    if (!fp64_fma_per_s || !fp32_fma_per_s) return IGS_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return IGS_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
        return IGS_ECUDA;
    const int blocks = 8 * sms;  // 2048 threads per SM: every sub-partition full of warps
    cudaStream_t st = nullptr;
    double *sink = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return IGS_ECUDA;
    int rc = cudaMalloc(&sink, sizeof(double) * (size_t)blocks) == cudaSuccess ? IGS_OK : IGS_ENOMEM;
    // about 0.3 s of FP64 work at GB300's rate and the same instruction count in FP32
    if (rc == IGS_OK) rc = probe<double>(blocks, 1 << 15, st, sink, fp64_fma_per_s);
    if (rc == IGS_OK) rc = probe<float>(blocks, 1 << 19, st, reinterpret_cast<float *>(sink), fp32_fma_per_s);
    cudaFree(sink);
    cudaStreamDestroy(st);
    return rc;
}
