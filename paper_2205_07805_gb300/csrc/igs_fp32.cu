// FP32-basis kernels of the precision form (igs_solve with precision = IGS_PREC_FP32_IR):
// the Arnoldi cycle of Alg. 4.1 runs with the SpMV, the Krylov basis V and the vectors z, u
// in FP32, while the Gram reductions are accumulated in FP64, and the (I + L) solves, the
// Givens least squares, x and the residual r = b - A x stay in FP64.  Each restart is then
// one step of iterative refinement: r = b - A x in FP64, an FP32 cycle for A d = r,
// x = x + V y in FP64.  The paper names mixed precision only as future work (Sec. 6).
//
// Every kernel here mirrors an FP64 kernel of igs_kernels.cu and writes the same FP64
// per-block partial sums, so the single-block steps (igs_kernels.cu) serve both forms.
#include "igs_internal.h"

namespace igs {

namespace {

__device__ __forceinline__ bool halted32(const DevState *st) { return st->halt != 0; }

// Rows per FP32 partial sum of the reductions before it is promoted to FP64.
constexpr int kChunk4 = 8;  // float4 loads (32 rows)

}  // namespace

// y = A x in FP32 (A's values rounded to FP32 at create), thread per row.
__global__ void __launch_bounds__(kStreamThreads)
k_spmv32_rows(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ colind,
              const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y,
              const DevState *st)
{
    IGS_PDL_ENTER();
    if (halted32(st)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int lo = rowptr[i], hi = rowptr[i + 1];
        float s0 = 0.f, s1 = 0.f;
        int q = lo;
        for (; q + 1 < hi; q += 2) {
            s0 = fmaf(val[q], x[colind[q]], s0);
            s1 = fmaf(val[q + 1], x[colind[q + 1]], s1);
        }
        if (q < hi) s0 = fmaf(val[q], x[colind[q]], s0);
        y[i] = s0 + s1;
    }
}

// y = A x in FP32, warp per row (long rows).
__global__ void __launch_bounds__(kStreamThreads)
k_spmv32_warp(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ colind,
              const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y,
              const DevState *st)
{
    IGS_PDL_ENTER();
    if (halted32(st)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const int lo = rowptr[i], hi = rowptr[i + 1];
        float s = 0.f;
        for (int q = lo + lane; q < hi; q += 32) s = fmaf(val[q], x[colind[q]], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) y[i] = s;
    }
}

// Block multi-dot of the FP32 basis (Alg. 4.1 steps 5 and 14), same grid and partial layout
// as the FP64 k_dots: part[rb*(NQ*p) + q*p + c] = sum over row block rb of V[:,c] X_q.
// The block's cw columns are split over its warps: warp w takes column c_lo + w % cw and
// the (w / cw)-th of S = warps / cw contiguous sub-ranges of the block's rows, and streams it
// with coalesced 16-byte loads (a warp reads 512 contiguous bytes per load), so every column
// is read in long runs.  Each lane sums its products in FP32 over chunks of 32 of its rows
// and adds each chunk sum to an FP64 accumulator; the lanes are combined by a fixed FP64
// shuffle tree and the sub-ranges in order.
template <int NQ>
__global__ void __launch_bounds__(kStreamThreads, 2)
k_dots32(const float *__restrict__ V, int64_t ld, int p, int64_t n4, int64_t rows,
         const float *__restrict__ x0, const float *__restrict__ x1, double *__restrict__ part,
         const DevState *st, int check_halt)
{
    IGS_PDL_ENTER();
    if (check_halt && halted32(st)) return;
    constexpr int W = kStreamThreads / 32;
    __shared__ double red[NQ][W];
    const int rb = blockIdx.x, G = gridDim.y, cg = blockIdx.y;
    const int c_lo = (int)((int64_t)cg * p / G), c_hi = (int)((int64_t)(cg + 1) * p / G);
    const int cw = c_hi - c_lo;
    const int S = W / cw;  // sub-ranges per column (cw <= 4 <= W)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int cl = wid % cw, sr = wid / cw;
    const int64_t r_lo = (int64_t)rb * rows;
    const int64_t r_hi = r_lo + rows < n4 ? r_lo + rows : n4;
    double d0 = 0.0, d1 = 0.0;
    if (sr < S && r_lo < r_hi) {
        const int64_t nquad = (r_hi - r_lo) >> 2;
        const int64_t q0 = nquad * sr / S, q1 = nquad * (sr + 1) / S;
        const float4 *vc = reinterpret_cast<const float4 *>(V + (int64_t)(c_lo + cl) * ld + r_lo);
        const float4 *xa = reinterpret_cast<const float4 *>(x0 + r_lo);
        const float4 *xb = reinterpret_cast<const float4 *>((NQ == 2 ? x1 : x0) + r_lo);
        constexpr int U = NQ == 2 ? 4 : 8;  // loads per lane per batch; a chunk is 8 quads
        for (int64_t base = q0; base < q1; base += 32 * kChunk4) {
            float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
            for (int h = 0; h < kChunk4; h += U) {
                float4 v[U], x[U], y[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t q = base + (int64_t)(h + u) * 32 + lane;
                    const bool in = q < q1;
                    v[u] = in ? vc[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                    x[u] = in ? xa[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                    if (NQ == 2) y[u] = in ? xb[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    a0 = fmaf(v[u].x, x[u].x, a0);
                    a1 = fmaf(v[u].y, x[u].y, a1);
                    a0 = fmaf(v[u].z, x[u].z, a0);
                    a1 = fmaf(v[u].w, x[u].w, a1);
                    if (NQ == 2) {
                        b0 = fmaf(v[u].x, y[u].x, b0);
                        b1 = fmaf(v[u].y, y[u].y, b1);
                        b0 = fmaf(v[u].z, y[u].z, b0);
                        b1 = fmaf(v[u].w, y[u].w, b1);
                    }
                }
            }
            d0 += (double)(a0 + a1);
            if (NQ == 2) d1 += (double)(b0 + b1);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        if (NQ == 2) d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    }
    if (lane == 0) {
        red[0][wid] = d0;
        if (NQ == 2) red[NQ - 1][wid] = d1;
    }
    __syncthreads();
    if (threadIdx.x < cw * NQ) {
        const int c = threadIdx.x % cw, qq = threadIdx.x / cw;
        double acc = 0.0;
        for (int j = 0; j < S; ++j) acc += red[qq][j * cw + c];
        part[(int64_t)rb * NQ * p + (int64_t)qq * p + c_lo + c] = acc;
    }
}

// FP32 basis update (steps 7, 11, 13, 16): out[i] = a src[i] - sum_{c<p} V[i,c] coef[c],
// coef (FP64, from the single-block steps) rounded to FP32.  With norm_last, column p-1 is
// first scaled in place by 1/gamma and a = 1/gamma.  Four consecutive rows per thread
// (16-byte loads; a block reads 4 KB of each column), padding rows included (they stay 0).
__global__ void __launch_bounds__(kStreamThreads)
k_update32(float *V, int64_t ld, int p, int64_t n4, const double *__restrict__ coef, double alpha,
           const float *src, float *out, int norm_last, const DevState *st)
{
    IGS_PDL_ENTER();
    if (halted32(st)) return;
    extern __shared__ float scf[];
    const float a = norm_last ? (float)st->inv_gamma : (float)alpha;
    for (int c = threadIdx.x; c < p; c += blockDim.x) scf[c] = (float)coef[c];
    __syncthreads();
    const int pc = norm_last ? p - 1 : p;
    const int64_t nq = n4 >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
        const float4 *vq = reinterpret_cast<const float4 *>(V) + q;
        const int64_t ldq = ld >> 2;
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        int c = 0;
        for (; c + 7 < pc; c += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = vq[(int64_t)(c + u) * ldq];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                const float c0 = scf[c + u], c1 = scf[c + u + 1];
                acc0.x = fmaf(v[u].x, c0, acc0.x);
                acc0.y = fmaf(v[u].y, c0, acc0.y);
                acc0.z = fmaf(v[u].z, c0, acc0.z);
                acc0.w = fmaf(v[u].w, c0, acc0.w);
                acc1.x = fmaf(v[u + 1].x, c1, acc1.x);
                acc1.y = fmaf(v[u + 1].y, c1, acc1.y);
                acc1.z = fmaf(v[u + 1].z, c1, acc1.z);
                acc1.w = fmaf(v[u + 1].w, c1, acc1.w);
            }
        }
        for (; c < pc; ++c) {
            const float4 v = vq[(int64_t)c * ldq];
            const float cf = scf[c];
            acc0.x = fmaf(v.x, cf, acc0.x);
            acc0.y = fmaf(v.y, cf, acc0.y);
            acc0.z = fmaf(v.z, cf, acc0.z);
            acc0.w = fmaf(v.w, cf, acc0.w);
        }
        if (norm_last) {
            float4 *vl = reinterpret_cast<float4 *>(V) + (int64_t)(p - 1) * ldq + q;
            float4 v = *vl;
            v.x *= a;
            v.y *= a;
            v.z *= a;
            v.w *= a;
            *vl = v;
            const float cf = scf[p - 1];
            acc1.x = fmaf(v.x, cf, acc1.x);
            acc1.y = fmaf(v.y, cf, acc1.y);
            acc1.z = fmaf(v.z, cf, acc1.z);
            acc1.w = fmaf(v.w, cf, acc1.w);
        }
        const float4 sv = reinterpret_cast<const float4 *>(src)[q];
        float4 o;
        o.x = fmaf(a, sv.x, -(acc0.x + acc1.x));
        o.y = fmaf(a, sv.y, -(acc0.y + acc1.y));
        o.z = fmaf(a, sv.z, -(acc0.z + acc1.z));
        o.w = fmaf(a, sv.w, -(acc0.w + acc1.w));
        reinterpret_cast<float4 *>(out)[q] = o;
    }
}

// v_1 = r / rho (step 1): FP64 residual to the FP32 basis.
__global__ void __launch_bounds__(kStreamThreads)
k_scale_to32(int64_t n, const double *__restrict__ src, float *__restrict__ dst, const DevState *st)
{
    IGS_PDL_ENTER();
    if (halted32(st)) return;
    const double f = st->inv_rho;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = (float)(src[i] * f);
}

// v = w / gamma in place (the flush's normalisation of the last column).
__global__ void __launch_bounds__(kStreamThreads)
k_scale32(int64_t n, float *v, const DevState *st)
{
    IGS_PDL_ENTER();
    if (halted32(st)) return;
    const float f = (float)st->inv_gamma;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] *= f;
}

// x = x + V y in FP64 (the refinement step x_m = x_0 + V_m y_m), p = st->ncols columns of the
// FP32 basis; each product of an FP32 basis entry and an FP64 coefficient is formed in FP64.
__global__ void __launch_bounds__(kStreamThreads)
k_xupdate32(const float *__restrict__ V, int64_t ld, int64_t n, const double *__restrict__ y,
            double *__restrict__ x, const DevState *st)
{
    IGS_PDL_ENTER();
    extern __shared__ double sy[];
    const int p = st->ncols;
    for (int c = threadIdx.x; c < p; c += blockDim.x) sy[c] = y[c];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float *vi = V + i;
        double s0 = 0.0, s1 = 0.0;
        int c = 0;
        for (; c + 1 < p; c += 2) {
            s0 = fma((double)vi[(int64_t)c * ld], sy[c], s0);
            s1 = fma((double)vi[(int64_t)(c + 1) * ld], sy[c + 1], s1);
        }
        if (c < p) s0 = fma((double)vi[(int64_t)c * ld], sy[c], s0);
        x[i] = x[i] + (s0 + s1);
    }
}

// ---- launchers ----
cudaError_t launch_spmv32(const Workspace &w, const float *x, float *y, cudaStream_t s)
{
    // one thread (short rows) or one warp (long rows) per row, all rows in flight at once
    const int64_t per_block = w.spmv_warp_rows ? kStreamThreads / 32 : kStreamThreads;
    const int64_t want = (w.n + per_block - 1) / per_block;
    const int grid = (int)(want < (int64_t)1 << 30 ? want : (int64_t)1 << 30);
    if (w.spmv_warp_rows)
        launch_k(false, k_spmv32_warp, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.rowptr, w.colind, w.val32,
                 x, y, (const DevState *)w.st);
    else
        launch_k(false, k_spmv32_rows, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.rowptr, w.colind, w.val32,
                 x, y, (const DevState *)w.st);
    return cudaGetLastError();
}

cudaError_t launch_dots32(const Workspace &w, int p, const float *x0, const float *x1, cudaStream_t s,
                          DotsPlan *plan_out)
{
    // one wave: two resident blocks per SM (register budget of k_dots32), never more row
    // blocks than the FP64 plan (whose partial-sum capacity the workspace holds)
    const DotsPlan pl = plan_dots_slots(w, p, 2 * w.num_sms);
    if (plan_out) *plan_out = pl;
    const int64_t n4 = (w.n + 3) / 4 * 4;
    dim3 grid(pl.rblocks, pl.groups);
    if (x1)
        launch_k(false, k_dots32<2>, grid, dim3(kStreamThreads), 0, s, (const float *)w.V32, w.ld, p, n4, pl.rows,
                 x0, x1, w.part, (const DevState *)w.st, 1);
    else
        launch_k(false, k_dots32<1>, grid, dim3(kStreamThreads), 0, s, (const float *)w.V32, w.ld, p, n4, pl.rows,
                 x0, (const float *)nullptr, w.part, (const DevState *)w.st, 1);
    return cudaGetLastError();
}

cudaError_t launch_update32(const Workspace &w, int p, const double *coef, double alpha, const float *src,
                            float *out, bool norm_last, cudaStream_t s)
{
    const size_t smem = sizeof(float) * (size_t)(p > 0 ? p : 1);
    const int64_t n4 = (w.n + 3) & ~int64_t(3);
    const int grid = (int)((n4 / 4 + kStreamThreads - 1) / kStreamThreads);
    launch_k(false, k_update32, dim3(grid), dim3(kStreamThreads), smem, s, w.V32, w.ld, p, n4, coef, alpha, src,
             out, norm_last ? 1 : 0, (const DevState *)w.st);
    return cudaGetLastError();
}

cudaError_t launch_scale_to32(const Workspace &w, const double *src, float *dst, cudaStream_t s)
{
    const int grid = w.num_sms * kBlocksPerSM;
    launch_k(false, k_scale_to32, dim3(grid), dim3(kStreamThreads), 0, s, w.n, src, dst, (const DevState *)w.st);
    return cudaGetLastError();
}

cudaError_t launch_scale32(const Workspace &w, float *v, cudaStream_t s)
{
    const int grid = w.num_sms * kBlocksPerSM;
    launch_k(false, k_scale32, dim3(grid), dim3(kStreamThreads), 0, s, w.n, v, (const DevState *)w.st);
    return cudaGetLastError();
}

cudaError_t launch_xupdate32(const Workspace &w, cudaStream_t s)
{
    const size_t smem = sizeof(double) * (size_t)(w.mmax + 1);
    const int grid = (int)((w.n + kStreamThreads - 1) / kStreamThreads);
    launch_k(false, k_xupdate32, dim3(grid), dim3(kStreamThreads), smem, s, (const float *)w.V32, w.ld, w.n,
             (const double *)w.y, w.x, (const DevState *)w.st);
    return cudaGetLastError();
}

}  // namespace igs
