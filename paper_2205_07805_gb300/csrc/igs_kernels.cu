// CUDA kernels of the GB300 (sm_103a) IGS-GMRES library.
//
// Method: Alg. 4.1 of Thomas, Carson, Rozloznik, Carr, Swirydowicz, "Iterated Gauss-Seidel
// GMRES" (arXiv 2205.07805), FP64 throughout.
//
// Hardware facts that shape every kernel here (measured on GB300): the FP64 pipe retires
// 2 FMAs per clock per SM, and each FP64 warp instruction holds its sub-partition's pipe
// for 64 clocks whatever its active-lane mask.  The streaming kernels are therefore
// FP64-issue-bound, not HBM-bound: every FP64 instruction must be a useful FMA on all 32
// lanes, reductions are laid out so that few additions are spent outside the products, and
// serial work (Givens rotations, the (I+L) solve) is reformulated to be lane-parallel.
#include "igs_internal.h"

#include <cmath>
#include <cstdio>

namespace igs {

namespace {

__device__ __forceinline__ bool halted(const DevState *st) { return st->halt != 0; }

// -------------------------------------------------------------------------------------
// Deterministic block-wide sum of the values held by each thread (fixed tree).
// `sh` must hold blockDim.x doubles.  Result valid in every thread.
// -------------------------------------------------------------------------------------
__device__ double block_sum(double v, double *sh)
{
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double s = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[0] = s;
    }
    __syncthreads();
    double r = sh[0];
    __syncthreads();
    return r;
}

// out[v] = sum_{rb < nrb} part[rb * nv + v] for v < nv (fixed order; block-wide, ends with
// a barrier).  The layout is row-block major, so consecutive threads read consecutive
// partials.  Each value is split over tpv threads (a power of two) so that no thread has
// more than kRedRegs partials; a thread issues all of its loads before its first add (one
// memory round trip), and the tpv sums are combined by a fixed shuffle tree.
constexpr int kRedRegs = 24;
__device__ void reduce_partials(const double *__restrict__ part, int nv, int nrb, double *out)
{
    const int T = blockDim.x, t = threadIdx.x;
    int tpv = 1;
    while (tpv < 32 && (nrb + tpv - 1) / tpv > kRedRegs) tpv <<= 1;
    const int vpr = T / tpv;
    for (int v0 = 0; v0 < nv; v0 += vpr) {
        const int v = v0 + t / tpv, sub = t % tpv;
        if (v0 + (t & ~31) / tpv >= nv) continue;  // whole warp idle: no FP64 issue slots spent
        double s = 0.0;
        if (v < nv) {
            double a[kRedRegs];
            double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
            // one pass unless nrb > kRedRegs * 32; the adds stop at the warp-uniform count
            // jmax of loaded partials (every FP64 add costs the warp's sub-partition dearly)
            for (int pass0 = 0; pass0 < nrb; pass0 += kRedRegs * tpv) {
                const int rb0 = pass0 + sub;
                const int jmax = min(kRedRegs, (nrb - pass0 + tpv - 1) / tpv);
#pragma unroll
                for (int j = 0; j < kRedRegs; ++j) {
                    const int rb = rb0 + j * tpv;
                    a[j] = (j < jmax && rb < nrb) ? part[(int64_t)rb * nv + v] : 0.0;
                }
#pragma unroll
                for (int j = 0; j < kRedRegs; j += 4) {
                    if (j >= jmax) break;
                    acc0 += a[j];
                    acc1 += a[j + 1];
                    acc2 += a[j + 2];
                    acc3 += a[j + 3];
                }
            }
            s = (acc0 + acc1) + (acc2 + acc3);
        }
        for (int o = tpv >> 1; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, tpv);
        if (sub == 0 && v < nv) out[v] = s;
    }
    __syncthreads();
}

// FP64 -> FP32 of v * 2^-e, rounded to nearest even, in integer arithmetic only (on this
// GPU one FP64-pipe instruction, a conversion included, holds a sub-partition for 64
// cycles).  Requires |v| 2^-e < 2^127; results below the FP32 normal range become +-0.
__device__ __forceinline__ float f64_scaled_to_f32(double v, int e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int be = (int)((b >> 52) & 0x7ff);
    const int fe = be - 1023 - e + 127;
    if (be == 0 || fe <= 0) return __int_as_float((int)sign);
    const unsigned long long m = b & 0xfffffffffffffull;
    unsigned int r = ((unsigned int)fe << 23) | (unsigned int)(m >> 29);
    const unsigned int rem = (unsigned int)(m & 0x1fffffffu);
    if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) r += 1u;
    return __int_as_float((int)(sign | r));
}

// FP32 -> FP64 of y * 2^e, exact, in integer arithmetic only.  FP32 zeros and subnormals,
// and results below the FP64 normal range, give +-0; requires y 2^e < 2^1024.
__device__ __forceinline__ double f32_scaled_to_f64(float y, int e)
{
    const unsigned int b = (unsigned int)__float_as_int(y);
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const int fe = (int)((b >> 23) & 0xff);
    const int dei = fe - 127 + 1023 + e;
    if (fe == 0 || dei <= 0) return __longlong_as_double((long long)sign);
    const unsigned long long de = (unsigned long long)dei;
    return __longlong_as_double((long long)(sign | (de << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// Row-packed strictly-lower triangle of L: row i (columns 0..i-1) starts at i(i-1)/2.  The
// step kernels keep a global copy in this layout beside the column-major L, so that staging
// rows 0..r-1 into shared memory is one contiguous copy.
__device__ __forceinline__ int packed_row(int i) { return i * (i - 1) / 2; }

// Start the copy of rows 0..rows-1 of the row-packed L (global, 16-byte aligned) into Lsm
// (shared, 16-byte aligned) with 16-byte cp.async chunks; an odd last double is copied by a
// plain load.  Nothing of Lsm beyond the rows is written.  lower_wait() completes it.
__device__ void lower_prefetch(const double *__restrict__ Lrow, int rows, double *Lsm)
{
    const int total = rows * (rows - 1) / 2;
    const int chunks = total >> 1;
    for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(Lsm + 2 * q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(Lrow + 2 * q) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if ((total & 1) && threadIdx.x == blockDim.x - 1) Lsm[total - 1] = Lrow[total - 1];
}

// Wait for this thread's cp.async copies (before a return that skips lower_wait).
__device__ __forceinline__ void lower_drain() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Wait for this thread's cp.async copies, then for the block.
__device__ __forceinline__ void lower_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
}

// x = (I + L_p)^{-1} rhs for the unit lower-triangular I + L (Alg. 4.1 steps 12 and 15).
// Lsm is the row-packed shared copy of L_p (lower_prefetch).  rhs and x live in shared memory (x
// must not alias rhs; `tmp` is scratch of p entries).  Block-wide.
//
// When ||L||_F is small the solve is evaluated as the truncated Neumann series
// sum_{i<t} (-L)^i rhs (Horner form), whose truncation error ||L||^t ||rhs|| / (1-||L||) is
// kept below 2^-60 ||rhs|| -- far under the FP64 rounding of the substitution itself.  Each
// term is one lane-parallel matrix-vector product instead of p dependent steps.  With two
// Gauss-Seidel iterations ||L||_F is O(eps) and t = 2.  Otherwise the classical
// column-oriented forward substitution runs (terms = 0; see neumann_terms).
//
// With f32 set (terms == 2 and (p+2) ||L||_F <= 2^-36, see neumann_fp32) the one correction
// term L rhs is evaluated in FP32: rhs is scaled by a power of two to [-2, 2), L's entries are
// rounded to FP32 as they are read, and x = rhs - 2^e (L rhs)_32.  Rounding L, rhs and the length-p sums to FP32 errs
// by at most (p+2) 2^-24 ||L||_F ||rhs|| <= 2^-60 ||rhs||, the bound the truncation already
// meets (entries flushed below the FP32 normal range add at most p 2^-125 max|rhs|), while
// the FP64 pipe of the one SM running this block would take microseconds for the p^2/2
// products.  Scaling and conversions are integer operations; the FP64 pipe does only the p
// final subtractions.
__device__ void unit_lower_solve(const double *Lsm, int p, const double *rhs, double *x,
                                 double *tmp, int terms, bool f32)
{
    const int T = blockDim.x, t = threadIdx.x;
    if (f32) {
        __shared__ int s_wmax[kSmallThreads / 32];
        const int lane = t & 31, wid = t >> 5;
        // e = largest binary exponent of rhs (biased exponent field; a subnormal counts as
        // -1022, above its true exponent, which keeps |rhs| 2^-e < 2)
        int e = -1022;
        for (int i = t; i < p; i += T) {
            const int be = (int)((__double_as_longlong(rhs[i]) >> 52) & 0x7ff);
            e = max(e, be - 1023);
        }
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0) s_wmax[wid] = e;
        __syncthreads();
        int emax = s_wmax[0];
        for (int q = 1; q < T / 32; ++q) emax = max(emax, s_wmax[q]);
        emax = min(emax, 1000);  // a non-finite rhs stays non-finite below
        float *xf = reinterpret_cast<float *>(tmp);
        float *yf = xf + p;  // tmp holds 2p floats
        for (int i = t; i < p; i += T) xf[i] = f64_scaled_to_f32(rhs[i], emax);
        __syncthreads();
        // Rows a and p-1-a (equal total length) form pair a; tpp threads share a pair and
        // take every tpp-th column, then combine by a fixed shuffle tree.
        const int npair = (p + 1) >> 1;
        int tpp = 32;
        while (tpp > 1 && npair * tpp > T) tpp >>= 1;
        for (int base = 0; base < npair * tpp; base += T) {
            const int q = base + t, a = q / tpp, h = q % tpp;
            const bool act = a < npair;
            const int r0 = a, r1 = p - 1 - a;
            float s0 = 0.0f, s1 = 0.0f;
            if (act) {
                const double *l0 = Lsm + packed_row(r0), *l1 = Lsm + packed_row(r1);
                for (int c = h; c < r0; c += tpp) s0 = fmaf(f64_scaled_to_f32(l0[c], 0), xf[c], s0);
                if (r1 != r0)
                    for (int c = h; c < r1; c += tpp) s1 = fmaf(f64_scaled_to_f32(l1[c], 0), xf[c], s1);
            }
            for (int o = tpp >> 1; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (act && h == 0) {
                yf[r0] = s0;
                if (r1 != r0) yf[r1] = s1;
            }
        }
        __syncthreads();
        for (int i = t; i < p; i += T) x[i] = rhs[i] - f32_scaled_to_f64(yf[i], emax);
        __syncthreads();
        return;
    }
    if (terms >= 1) {
        for (int i = t; i < p; i += T) x[i] = rhs[i];
        __syncthreads();
        // tmp = rhs - L x.  Rows a and p-1-a (equal total length) form pair a; tpp threads
        // share a pair and take every tpp-th column (two independent FMA chains each), then
        // combine by a fixed shuffle tree.  tpp spreads the pairs over the whole block (two
        // rounds when that doubles tpp from 2): the FP64 instructions of the single SM are the
        // cost, so every warp should carry its share.
        const int npair = (p + 1) >> 1;
        int tpp = 32;
        while (tpp > 1 && npair * tpp > T) tpp >>= 1;
        if (tpp <= 2 && npair * 2 * tpp <= 2 * T) tpp *= 2;
        for (int it = 1; it < terms; ++it) {
            for (int base = 0; base < npair * tpp; base += T) {
                const int q = base + t, a = q / tpp, h = q % tpp;
                const bool act = a < npair;
                const int r0 = a, r1 = p - 1 - a;
                double s0 = 0.0, s1 = 0.0;
                if (act) {
                    const double *l0 = Lsm + packed_row(r0), *l1 = Lsm + packed_row(r1);
                    for (int c = h; c < r0; c += tpp) s0 = fma(l0[c], x[c], s0);
                    if (r1 != r0)
                        for (int c = h; c < r1; c += tpp) s1 = fma(l1[c], x[c], s1);
                }
                for (int o = tpp >> 1; o > 0; o >>= 1) {
                    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                }
                if (act && h == 0) {
                    tmp[r0] = rhs[r0] - s0;
                    if (r1 != r0) tmp[r1] = rhs[r1] - s1;
                }
            }
            __syncthreads();
            for (int i = t; i < p; i += T) x[i] = tmp[i];
            __syncthreads();
        }
        return;
    }
    // Forward substitution, column oriented: after x[c] is final, every later row subtracts
    // L(i,c) x[c].  Rows are owned by threads (i = t + T*q, q < 4 covers p <= 4T).
    double xi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = t + T * q;
        xi[q] = i < p ? rhs[i] : 0.0;
    }
    for (int c = 0; c < p; ++c) {
        if ((c % T) == t) x[c] = xi[c / T];
        __syncthreads();
        const double xc = x[c];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = t + T * q;
            if (i > c && i < p) xi[q] = fma(-Lsm[packed_row(i) + c], xc, xi[q]);
        }
    }
    __syncthreads();
}

// Number of Neumann terms t for (I+L)^{-1}: the smallest t with ||L||_F^t <= 2^-60, from the
// binary exponent of ||L||_F^2 (integer arithmetic only); 1 when L = 0; 0 (substitution)
// when ||L||_F >= 2^-15 or the value is not finite.
__device__ __forceinline__ int neumann_terms(double lfro2)
{
    const long long b = __double_as_longlong(lfro2);
    if (b == 0) return 1;
    const int ex = (int)((b >> 52) & 0x7ff) - 1023;  // lfro2 in [2^ex, 2^(ex+1))
    if (b < 0 || ex >= -30) return 0;
    const int d = -(ex + 1);                          // ||L||_F < 2^(-d/2), d >= 30
    const int terms = (120 + d - 1) / d;
    return terms < 2 ? 2 : terms;
}

// Whether unit_lower_solve may evaluate the Neumann correction in FP32: two terms, and
// (p+2) ||L||_F <= 2^-36 (lfro2 = ||L||_F^2; false for a non-finite value).
__device__ __forceinline__ bool neumann_fp32(double lfro2, int p, int terms)
{
    const double q = (double)(p + 2);
    return terms == 2 && q * q * lfro2 <= 0x1p-72;
}

// ||col[0:len]||^2 by the block's last warp (fixed shuffle tree), stored in *out.  Called
// before a block-wide step that ends with a barrier, so that it overlaps that step.
__device__ void last_warp_sumsq(const double *__restrict__ col, int len, double *out)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid != ((int)blockDim.x >> 5) - 1) return;
    double a0 = 0.0, a1 = 0.0;
    int i = lane;
    for (; i + 32 < len; i += 64) {
        a0 = fma(col[i], col[i], a0);
        a1 = fma(col[i + 32], col[i + 32], a1);
    }
    if (i < len) a0 = fma(col[i], col[i], a0);
    double v = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) *out = v;
}

}  // namespace

// =====================================================================================
// SpMV (Alg. 4.1 step 4; also r = b - A x for steps 1 and the end-of-cycle residual).
// =====================================================================================
// Thread per row: short rows (stencil matrices).  Two accumulation chains per row.
__global__ void __launch_bounds__(kStreamThreads)
k_spmv_rows(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ colind,
            const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
            const double *__restrict__ b, const DevState *st, int check_halt, float2 *__restrict__ ydf)
{
    IGS_PDL_ENTER();
    if (check_halt && halted(st)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int lo = rowptr[i], hi = rowptr[i + 1];
        double s0 = 0.0, s1 = 0.0;
        int q = lo;
        for (; q + 1 < hi; q += 2) {
            s0 = fma(val[q], x[colind[q]], s0);
            s1 = fma(val[q + 1], x[colind[q + 1]], s1);
        }
        if (q < hi) s0 = fma(val[q], x[colind[q]], s0);
        const double s = s0 + s1;
        const double o = b ? b[i] - s : s;
        y[i] = o;
        if (ydf) {
            float h, l;
            df_split(o, h, l);
            ydf[i] = make_float2(h, l);
        }
    }
}

// Thread per row over the SELL-32 copy (short rows): a warp is one 32-row slice, so every
// column-index and value load of the warp is one contiguous 128- or 256-byte segment.  The
// entries of a row are visited in CSR order with the same two chains as k_spmv_rows (even
// and odd positions), so the results are bitwise those of the CSR kernel.
__global__ void __launch_bounds__(kStreamThreads)
k_spmv_sell(int64_t n, const int64_t *__restrict__ sell_off, const int *__restrict__ sell_col,
            const double *__restrict__ sell_val, const double *__restrict__ x, double *__restrict__ y,
            const double *__restrict__ b, const DevState *st, int check_halt, float2 *__restrict__ ydf)
{
    IGS_PDL_ENTER();
    if (check_halt && halted(st)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // the grid covers n
    if (i >= n) return;
    const int64_t off = sell_off[i >> 5];
    const int wd = (int)((sell_off[(i >> 5) + 1] - off) >> 5);
    const int *cs = sell_col + off + (i & 31);
    const double *vs = sell_val + off + (i & 31);
    double s0 = 0.0, s1 = 0.0;
    int k = 0;
    for (; k + 1 < wd; k += 2) {
        const int c0 = cs[32 * k], c1 = cs[32 * (k + 1)];
        const double v0 = vs[32 * k], v1 = vs[32 * (k + 1)];
        if (c0 >= 0) s0 = fma(v0, x[c0], s0);
        if (c1 >= 0) s1 = fma(v1, x[c1], s1);
    }
    if (k < wd) {
        const int c0 = cs[32 * k];
        if (c0 >= 0) s0 = fma(vs[32 * k], x[c0], s0);
    }
    const double s = s0 + s1;
    const double o = b ? b[i] - s : s;
    y[i] = o;
    if (ydf) {  // the split copy the double-float form's multi-dot reads
        float h, l;
        df_split(o, h, l);
        ydf[i] = make_float2(h, l);
    }
}

// Thread per row over the ELL form of the SELL-32 copy (every slice W entries wide, padding
// column -1): the slice offset is arithmetic, so a thread issues all W column-index and value
// loads at once, then all its gathers of x, instead of waiting on the offset first.  The two
// chains take the entries in the same order as k_spmv_rows / k_spmv_sell (bitwise the same sums).
template <int W>
__global__ void __launch_bounds__(kStreamThreads)
k_spmv_ell(int64_t n, const int *__restrict__ col, const double *__restrict__ val, const double *__restrict__ x,
           double *__restrict__ y, const double *__restrict__ b, const DevState *st, int check_halt,
           float2 *__restrict__ ydf)
{
    IGS_PDL_ENTER();
    if (check_halt && halted(st)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // the grid covers n
    if (i >= n) return;
    const int64_t base = (i >> 5) * (32 * W) + (i & 31);
    int c[W];
    double v[W], xv[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        c[k] = col[base + 32 * k];
        v[k] = val[base + 32 * k];
    }
#pragma unroll
    for (int k = 0; k < W; ++k) xv[k] = c[k] >= 0 ? x[c[k]] : 0.0;
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        if (c[k] >= 0) {
            if (k & 1)
                s1 = fma(v[k], xv[k], s1);
            else
                s0 = fma(v[k], xv[k], s0);
        }
    }
    const double s = s0 + s1;
    const double o = b ? b[i] - s : s;
    y[i] = o;
    if (ydf) {
        float h, l;
        df_split(o, h, l);
        ydf[i] = make_float2(h, l);
    }
}

// Warp per row: long rows (dense or wide-band matrices).
__global__ void __launch_bounds__(kStreamThreads)
k_spmv_warp(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ colind,
            const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
            const double *__restrict__ b, const DevState *st, int check_halt, float2 *__restrict__ ydf)
{
    IGS_PDL_ENTER();
    if (check_halt && halted(st)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const int lo = rowptr[i], hi = rowptr[i + 1];
        double s0 = 0.0, s1 = 0.0;
        int q = lo + lane;
        for (; q + 32 < hi; q += 64) {
            s0 = fma(val[q], x[colind[q]], s0);
            s1 = fma(val[q + 32], x[colind[q + 32]], s1);
        }
        if (q < hi) s0 = fma(val[q], x[colind[q]], s0);
        double s = s0 + s1;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double o = b ? b[i] - s : s;
            y[i] = o;
            if (ydf) {
                float h, l;
                df_split(o, h, l);
                ydf[i] = make_float2(h, l);
            }
        }
    }
}

// =====================================================================================
// Block multi-dot (Alg. 4.1 step 5, the one global reduction per iteration; step 14).
// part[rb*(NQ*p) + q*p + c] = sum over the rows of row block rb of V[:,c] * X_q.
// Grid: x = row blocks (rows on multiples of 64), y = column groups (p columns split
// evenly, at most 4 per group).  Warp w of a block streams column c_lo + w % cwp over its
// row sub-slice w / cwp in 64-row segments: each lane loads two consecutive rows, so one
// warp instruction reads 512 contiguous bytes of the column (HBM row locality; scattered
// 16-byte lane loads ran 7 % slower).  No lane spends an FP64 add on other lanes' products
// until the fixed-order tree over the column's lane partials at the end.  With NQ = 2 each
// V element feeds two FMAs ([V, w]^T [w, z]).
// =====================================================================================
template <int NQ>
__global__ void __launch_bounds__(kStreamThreads, kDotsBlocksPerSM)
k_dots(const double *__restrict__ V, int64_t ld, int p, int64_t n4, int64_t rows,
       const double *__restrict__ x0, const double *__restrict__ x1, double *__restrict__ part,
       const DevState *st, int check_halt)
{
    IGS_PDL_ENTER();
    if (check_halt && halted(st)) return;
    constexpr int W = kStreamThreads / 32;
    __shared__ double red[NQ][kStreamThreads];
    const int rb = blockIdx.x, G = gridDim.y, cg = blockIdx.y;
    const int c_lo = (int)((int64_t)cg * p / G), c_hi = (int)((int64_t)(cg + 1) * p / G);
    const int cw = c_hi - c_lo;
    const int cwp = cw <= 1 ? 1 : cw <= 2 ? 2 : cw <= 4 ? 4 : 8;
    const int S = W / cwp;          // warps (row sub-slices) per column
    const int K = S * 32;           // lane partials per column
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int cl = wid % cwp, s = wid / cwp;
    const int64_t r_lo = (int64_t)rb * rows;
    const int64_t r_hi = r_lo + rows < n4 ? r_lo + rows : n4;
    double a0 = 0.0, a1 = 0.0;
    if (cl < cw && r_lo < r_hi) {
        const int64_t nseg = (r_hi - r_lo + 63) >> 6;  // 64-row segments: 512 bytes per column
        const int64_t g0 = nseg * s / S, g1 = nseg * (s + 1) / S;
        const double *__restrict__ vc = V + (int64_t)(c_lo + cl) * ld;
#pragma unroll 4
        for (int64_t g = g0; g < g1; ++g) {
            const int64_t i = r_lo + (g << 6) + 2 * lane;
            if (i < r_hi) {
                const double2 v = *reinterpret_cast<const double2 *>(vc + i);
                const double2 xa = *reinterpret_cast<const double2 *>(x0 + i);
                if (NQ == 2) {
                    const double2 ya = *reinterpret_cast<const double2 *>(x1 + i);
                    a0 = fma(v.x, xa.x, a0);
                    a1 = fma(v.x, ya.x, a1);
                    a0 = fma(v.y, xa.y, a0);
                    a1 = fma(v.y, ya.y, a1);
                } else {
                    a0 = fma(v.x, xa.x, a0);
                    a1 = fma(v.y, xa.y, a1);
                }
            }
        }
    }
    // lane partials of column cl at red[q][cl * K + s * 32 + lane]; fixed-order tree per column
    if (cl < cw) {
        const int k = s * 32 + lane;
        if (NQ == 1) {
            red[0][cl * K + k] = a0 + a1;
        } else {
            red[0][cl * K + k] = a0;
            red[NQ - 1][cl * K + k] = a1;
        }
    }
    for (int h = K >> 1; h >= 1; h >>= 1) {
        __syncthreads();
        if (t < cwp * h) {
            const int c = t / h, k = t % h;
            if (c < cw) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) red[q][c * K + k] += red[q][c * K + k + h];
            }
        }
    }
    __syncthreads();
    if (t < cw) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) part[(int64_t)rb * NQ * p + (int64_t)q * p + c_lo + t] = red[q][t * K];
    }
}

// =====================================================================================
// Basis update (Alg. 4.1 steps 7, 11, 13 and 16; x_m = x_0 + V_m y_m at cycle end):
//   out[i] = a * src[i] - sum_{c<p} V[i,c] coef[c]
// Two rows per thread (16-byte loads), coalesced over rows for each column.  With
// norm_last, column p-1 (the lagged w_{k-1}) is first normalised in place,
// v = w * inv_gamma (step 7), and a = inv_gamma (step 11).
// Each row's sum starts from a * src[i] (src itself when a = 1) and adds the products with
// the negated coefficients in column order, so the result needs no closing additions: every
// FP64 instruction but the scaling is one of the update's multiply-adds (the kernel is bound
// by the FP64 pipe).
// =====================================================================================
__global__ void __launch_bounds__(kStreamThreads, kUpdateBlocksPerSM)
k_update(double *V, int64_t ld, int p, int64_t n, const double *__restrict__ coef, int neg_coef,
         double alpha, const double *src, double *out, int norm_last, int p_from_state,
         DevState *st, int check_halt)
{
    IGS_PDL_ENTER();
    if (check_halt && halted(st)) return;
    extern __shared__ double sc[];  // -coef (the products are added)
    if (p_from_state) p = st->ncols;
    const double a = norm_last ? st->inv_gamma : alpha;
    const bool unit = a == 1.0;
    for (int c = threadIdx.x; c < p; c += blockDim.x) sc[c] = neg_coef ? coef[c] : -coef[c];
    __syncthreads();
    const int pc = norm_last ? p - 1 : p;
    // Two rows per thread (16-byte loads; ld is even and the pad rows stay zero).
    // Block b owns the contiguous pair range [b ppb, (b+1) ppb): with a grid of a whole
    // number of blocks per SM every SM gets the same share of the FP64 work.
    const int64_t npairs = (n + 1) >> 1;
    const int64_t ppb = (npairs + gridDim.x - 1) / gridDim.x;
    const int64_t pr_lo = (int64_t)blockIdx.x * ppb;
    const int64_t pr_hi = pr_lo + ppb < npairs ? pr_lo + ppb : npairs;
    for (int64_t pr = pr_lo + threadIdx.x; pr < pr_hi; pr += blockDim.x) {
        const int64_t i = 2 * pr;
        const double *vi = V + i;
        const double2 sv = *reinterpret_cast<const double2 *>(src + i);
        double x = unit ? sv.x : a * sv.x, y = unit ? sv.y : a * sv.y;
        int c = 0;
        if (pc >= 4) {
            // software pipeline: the next 4 columns load while these 4 are used
            double2 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = *reinterpret_cast<const double2 *>(vi + (int64_t)q * ld);
            for (; c + 7 < pc; c += 4) {
                double2 nv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) nv[q] = *reinterpret_cast<const double2 *>(vi + (int64_t)(c + 4 + q) * ld);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x = fma(v[q].x, sc[c + q], x);
                    y = fma(v[q].y, sc[c + q], y);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = nv[q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                x = fma(v[q].x, sc[c + q], x);
                y = fma(v[q].y, sc[c + q], y);
            }
            c += 4;
        }
        for (; c < pc; ++c) {
            const double2 v = *reinterpret_cast<const double2 *>(vi + (int64_t)c * ld);
            x = fma(v.x, sc[c], x);
            y = fma(v.y, sc[c], y);
        }
        if (norm_last) {
            double2 *vl = reinterpret_cast<double2 *>(V + (int64_t)(p - 1) * ld + i);
            double2 v = *vl;
            v.x *= a;
            v.y *= a;
            *vl = v;
            x = fma(v.x, sc[p - 1], x);
            y = fma(v.y, sc[p - 1], y);
        }
        *reinterpret_cast<double2 *>(out + i) = make_double2(x, y);
    }
}

// Partial sums of squares of up to three vectors: part[blockIdx.x * nvec + q].
__global__ void __launch_bounds__(kStreamThreads)
k_norms(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
        const double *__restrict__ c, double *__restrict__ part, int nvec)
{
    IGS_PDL_ENTER();
    __shared__ double sh[kStreamThreads];
    const double *vs[3] = {a, b, c};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int q = 0; q < 3; ++q) {
        if (!vs[q]) break;
        const double *v = vs[q];
        double s0 = 0.0, s1 = 0.0;
        int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + stride < n; i += 2 * stride) {
            s0 = fma(v[i], v[i], s0);
            s1 = fma(v[i + stride], v[i + stride], s1);
        }
        if (i < n) s0 = fma(v[i], v[i], s0);
        const double tot = block_sum(s0 + s1, sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * nvec + q] = tot;
    }
}

// dst = src * scale, scale = st->inv_rho (which = 0) or st->inv_gamma (which = 1).
__global__ void __launch_bounds__(kStreamThreads)
k_scale(int64_t n, const double *src, double *dst, int which, const DevState *st, int check_halt)
{
    IGS_PDL_ENTER();
    if (check_halt && halted(st)) return;
    const double f = which == 0 ? st->inv_rho : st->inv_gamma;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = src[i] * f;
}

// =====================================================================================
// Small single-block steps.
// =====================================================================================
struct SmallArgs {
    double *H, *L, *Lrow, *R, *cs, *sn, *g, *lfro2, *r1v, *r2v, *r3v, *y, *hist_res, *hist_lfro;
    const double *part;
    DevState *st;
    int ldh, ldl;
};

static SmallArgs small_args(const Workspace &w)
{
    SmallArgs a;
    a.H = w.H; a.L = w.L; a.Lrow = w.Lrow; a.R = w.R; a.cs = w.cs; a.sn = w.sn; a.g = w.g; a.lfro2 = w.lfro2;
    a.r1v = w.r1v; a.r2v = w.r2v; a.r3v = w.r3v; a.y = w.y;
    a.hist_res = w.hist_res; a.hist_lfro = w.hist_lfro; a.part = w.part; a.st = w.st;
    a.ldh = w.ldh(); a.ldl = w.ldl();
    return a;
}

// Solve-level initialisation of the device state.
__global__ void k_init_state(DevState *st, double tol, double normA, double inner_tol)
{
    IGS_PDL_ENTER();
    if (threadIdx.x == 0) {
        DevState s = {};
        s.tol = tol;
        s.normA = normA;
        s.inner_tol = inner_tol;
        *st = s;
    }
}

// ||b|| from its partial sums of squares.
__global__ void __launch_bounds__(kSmallThreads) k_bnorm(const double *part, int nblk, DevState *st)
{
    IGS_PDL_ENTER();
    __shared__ double out[1];
    reduce_partials(part, 1, nblk, out);
    if (threadIdx.x == 0) st->bnorm = sqrt(out[0]);
}

// End of a cycle (and start of a solve): r = b - A x is in place; from the partial sums of
// squares of r and x compute ||r||, ||x|| and beta(x) = ||r|| / (||b|| + ||A||_2 ||x||)
// (eq. "nrbe").
__global__ void __launch_bounds__(kSmallThreads) k_beta(const double *part, int nblk, DevState *st)
{
    IGS_PDL_ENTER();
    __shared__ double out[2];
    reduce_partials(part, 2, nblk, out);
    if (threadIdx.x == 0) {
        const double rn = sqrt(out[0]), xn = sqrt(out[1]);
        st->rnorm = rn;
        st->xnorm = xn;
        st->beta = rn == 0.0 ? 0.0 : rn / (st->bnorm + st->normA * xn);
    }
}

// Cycle start (Alg. 4.1 step 1): rho = ||r0||, g = rho e1, stop-test denominator, flags.
__global__ void __launch_bounds__(kSmallThreads) k_cycle_start(SmallArgs a, int mmax)
{
    IGS_PDL_ENTER();
    DevState *st = a.st;
    for (int i = threadIdx.x; i <= mmax; i += blockDim.x) a.g[i] = 0.0;
    if (threadIdx.x == 0) {
        const double rho = st->rnorm;
        st->rho = rho;
        st->inv_rho = 1.0 / rho;
        a.g[0] = rho;
        a.lfro2[0] = 0.0;
        st->stop_den = st->bnorm + st->normA * st->xnorm;
        st->stop_floor = st->inner_tol * rho;
        st->halt = 0;
        st->stop_cols = 0;
        st->stop_reason = 0;
        st->ncols = 0;
        if (!(rho > 0.0) || !isfinite(rho)) {
            st->halt = 1;
            st->stop_cols = 0;
            st->stop_reason = rho == 0.0 ? 2 : -4;
        }
    }
}

// Step 2 (priming): H_{1,1} = v_1^T w_2; the update w_2 -= H_{1,1} v_1 follows.
__global__ void __launch_bounds__(kSmallThreads) k_prime(SmallArgs a, int nrb)
{
    IGS_PDL_ENTER();
    if (halted(a.st)) return;
    __shared__ double out[1];
    reduce_partials(a.part, 1, nrb, out);
    if (threadIdx.x == 0) {
        a.H[0] = out[0];
        a.r1v[0] = out[0];
    }
}

// Steps 5 (combine) to 12 of iteration k (p = k-1 columns in V_{k-1}):
//   gamma = ||w_{k-1}||, H_{k-1,k-2} = gamma, r^(0) /= gamma (twice for its last entry),
//   new L row = (V_{k-2}^T w_{k-1}) / gamma, r^(1) = (I + L_{k-1})^{-1} r^(0);
//   with one Gauss-Seidel iteration also H_{1:k-1,k-1} = r^(1).
// Partials: value c < p-1 is V[:,c].w, value p-1 is w.w, value p+c is V[:,c].z.
__global__ void __launch_bounds__(kSmallThreads) k_step_a(SmallArgs a, int k, int gs, int nrb)
{
    extern __shared__ __align__(16) double dsm[];
    const int pp = k - 1;
    double *buf = dsm;              // 2p combined partials
    double *r0s = buf + 2 * pp;     // r^(0)
    double *r1s = r0s + pp;         // r^(1)
    double *tmp = r1s + pp;         // solve scratch
    double *Lsm = dsm + ((5 * pp + 1) & ~1);  // row-packed L_p (16-byte aligned)
    __shared__ double s_inv_gamma;
    __shared__ int s_stop, s_terms, s_f32;
    __shared__ double s_hn2;
    const int p = k - 1, t = threadIdx.x;
    // Rows 0..p-2 of L, ||L_{p-1}||_F^2 and H column p-2 (the breakdown test needs its
    // squared norm) come from earlier steps, which completed before the multi-dot this kernel
    // follows was launched: they are staged before the programmatic wait, overlapping the
    // multi-dot's tail.  Row p-1 of L is formed below and written to shared memory directly.
    lower_prefetch(a.Lrow, p - 1, Lsm);
    const double lf2_prev = t == 0 ? a.lfro2[p - 2] : 0.0;
    last_warp_sumsq(a.H + (int64_t)(p - 2) * a.ldh, p - 1, &s_hn2);
    IGS_PDL_ENTER();
    DevState *st = a.st;
    if (halted(st)) {
        lower_drain();
        return;
    }
    if (st->stop_reason != 0) {  // the previous column met the stop test
        if (t == 0) st->halt = 1;
        lower_drain();
        return;
    }
    reduce_partials(a.part, 2 * p, nrb, buf);
    const double hn2 = s_hn2;
    if (t == 0) {
        const double ww = buf[p - 1];
        int stop = 0;
        double gam = 0.0, ig = 0.0;
        if (!(ww >= 0.0) || isinf(ww)) {
            stop = -4;
        } else {
            if (ww > 0.0) {
                ig = rsqrt(ww);
                gam = ww * ig;
            }
            a.H[(int64_t)(p - 2) * a.ldh + (p - 1)] = gam;
            if (ww == 0.0 || ww <= kBreakdownFactor * kBreakdownFactor * hn2) stop = 2;
        }
        if (stop != 0) {
            st->halt = 1;
            st->stop_reason = stop;
            st->stop_cols = p - 1;
        }
        st->inv_gamma = ig;
        s_inv_gamma = ig;
        s_stop = stop;
    }
    __syncthreads();
    if (s_stop != 0) {
        lower_drain();
        return;
    }
    const double ig = s_inv_gamma;
    if (t < 32) {
        // step 10 (warp 0): the new L row, its squared norm and the Neumann term count
        double rowsq = 0.0;
        for (int c = t; c < p - 1; c += 32) {
            const double l = buf[c] * ig;
            a.L[(int64_t)c * a.ldl + (p - 1)] = l;
            a.Lrow[packed_row(p - 1) + c] = l;
            Lsm[packed_row(p - 1) + c] = l;
            rowsq = fma(l, l, rowsq);
        }
        for (int o = 16; o > 0; o >>= 1) rowsq += __shfl_down_sync(0xffffffffu, rowsq, o);
        if (t == 0) {
            const double lf2 = lf2_prev + rowsq;
            a.lfro2[p - 1] = lf2;
            s_terms = neumann_terms(lf2);
            s_f32 = neumann_fp32(lf2, p, s_terms);
        }
    } else {
        // steps 8-9 (other warps): r^(0) / gamma, its last entry once more
        for (int c = t - 32; c < p; c += blockDim.x - 32) {
            double r = buf[p + c] * ig;
            if (c == p - 1) r *= ig;
            r0s[c] = r;
        }
    }
    __syncthreads();
    // step 12
    const int terms = s_terms;
    const bool f32 = s_f32 != 0;
    lower_wait();
    unit_lower_solve(Lsm, p, r0s, r1s, tmp, terms, f32);
    for (int c = t; c < p; c += blockDim.x) {
        a.r1v[c] = r1s[c];
        if (gs == 1) a.H[(int64_t)(p - 1) * a.ldh + c] = r1s[c];
    }
    if (t == 0) st->neumann_terms = terms;
}

// Steps 14 (combine) to 17 with two Gauss-Seidel iterations:
//   r^(3) = (I + L_{k-1})^{-1} r^(2),  H_{1:k-1,k-1} = r^(1) + r^(3).
__global__ void __launch_bounds__(kSmallThreads) k_step_b(SmallArgs a, int k, int nrb)
{
    extern __shared__ __align__(16) double dsm[];
    const int p = k - 1, t = threadIdx.x;
    double *r2s = dsm, *r3s = r2s + p, *tmp = r3s + p;
    double *Lsm = dsm + ((3 * p + 1) & ~1);  // row-packed L_p (16-byte aligned)
    // L_{k-1} and ||L||_F were written by k_step_a, which completed before the multi-dot this
    // kernel follows was launched: they are staged before waiting for that multi-dot.
    const int terms = neumann_terms(a.lfro2[p - 1]);
    const bool f32 = neumann_fp32(a.lfro2[p - 1], p, terms);
    lower_prefetch(a.Lrow, p, Lsm);
    IGS_PDL_ENTER();
    DevState *st = a.st;
    if (halted(st)) {
        lower_drain();
        return;
    }
    reduce_partials(a.part, p, nrb, r2s);
    lower_wait();
    unit_lower_solve(Lsm, p, r2s, r3s, tmp, terms, f32);
    for (int c = t; c < p; c += blockDim.x) {
        a.r3v[c] = r3s[c];
        a.H[(int64_t)(p - 1) * a.ldh + c] = a.r1v[c] + r3s[c];
    }
}

// End of the k-loop (k = m+1 done): gamma_{m+1} = ||w_{m+1}||, H_{m+1,m} = gamma_{m+1}, the
// last row of L; the scaling v_{m+1} = w_{m+1} / gamma_{m+1} follows.  Partials: value
// c < m is V[:,c].w, value m is w.w.
__global__ void __launch_bounds__(kSmallThreads) k_flush(SmallArgs a, int m, int nrb)
{
    IGS_PDL_ENTER();
    DevState *st = a.st;
    if (halted(st)) return;
    if (st->stop_reason != 0) {
        if (threadIdx.x == 0) st->halt = 1;
        return;
    }
    __shared__ double buf[kMaxRestart + 1];
    __shared__ double sh[kSmallThreads];
    __shared__ double s_ig;
    __shared__ int s_stop;
    __shared__ double s_hn2;
    const int t = threadIdx.x;
    last_warp_sumsq(a.H + (int64_t)(m - 1) * a.ldh, m, &s_hn2);
    reduce_partials(a.part, m + 1, nrb, buf);
    const double hn2 = s_hn2;
    if (t == 0) {
        const double ww = buf[m];
        int stop = 0;
        double ig = 0.0;
        if (!(ww >= 0.0) || isinf(ww)) {
            stop = -4;
        } else {
            double gam = 0.0;
            if (ww > 0.0) {
                ig = rsqrt(ww);
                gam = ww * ig;
            }
            a.H[(int64_t)(m - 1) * a.ldh + m] = gam;
            if (ww == 0.0 || ww <= kBreakdownFactor * kBreakdownFactor * hn2) stop = 2;
        }
        if (stop != 0) {
            st->halt = 1;
            st->stop_reason = stop;
            st->stop_cols = m;
        }
        st->inv_gamma = ig;
        s_ig = ig;
        s_stop = stop;
    }
    __syncthreads();
    if (s_stop != 0) return;
    double rowsq = 0.0;
    for (int c = t; c < m; c += blockDim.x) {
        const double l = buf[c] * s_ig;
        a.L[(int64_t)c * a.ldl + m] = l;
        a.Lrow[packed_row(m) + c] = l;
        rowsq = fma(l, l, rowsq);
    }
    const double rs = block_sum(rowsq, sh);
    if (t == 0) a.lfro2[m] = a.lfro2[m - 1] + rs;
}

// =====================================================================================
// Alg. 4.2 (one-reduce hybrid MGS-CGS GMRES).  V[:, nb] holds u_{k-1}, the output of the
// previous iteration's single projection (nb = k-2 normalised columns before it); the one
// reduction gives (partials of the step-5 multi-dot over p = nb+1 columns with x0 = u,
// x1 = A u): value c < nb is r^(2)_c = V[:,c].u, value nb is ||u||^2, value nb+1+c is
// V[:,c].(A u), value 2nb+1 is u.(A u).
//
// Of an iteration's small steps, the fused basis update that follows needs only r^(2), gamma
// and r^(1).  The rest -- r^(3) = (I + L)^{-1} r^(2), the completed Hessenberg column, its
// breakdown test, the new row of L and the next first-projection coefficients q -- depends
// only on what the iteration stores (r2v, r1v, 1/gamma, gamma^2), so the next launch does it
// in its prologue, before its programmatic wait: on an SM the multi-dot has already left,
// while the multi-dot's last blocks still run.  Hence the launch for nb (k = nb+2) first
// completes column nb-2 (the previous launch's), then forms this iteration's r^(2), gamma and
// r^(1).  The Givens rotation of column nb-2 follows it on the side branch.  The cycle's end
// (flush) completes columns m-2 and m-1.
// =====================================================================================
// Steps 5, 9, 14 and 15 of the previous iteration (nbp = nb-1 columns before its u), from its
// r2v, r1v, st->inv_gamma, st->lag_g2 and q (r3v; H_11 in H[0] when nbp = 1), with
// L_{nbp} staged in Lsm: r^(3) = (I + L_{nbp})^{-1} r^(2) (into r3s), H_{0:nbp-1, nbp-1} =
// q + r^(3) (into hcol and H), the breakdown test gamma^2 <= (64 eps)^2 ||column||^2, then
// (no stop) L row nbp = r^(2) / gamma (global, and into Lsm) with ||L_{nbp+1}||_F^2 (*lf2),
// and the next q = r^(1) - H_{0:nbp, 0:nbp-1} r^(3) / gamma (into qs and r3v).  Returns the
// stop reason the column ends with (0: none).  Block-wide.
__device__ int complete_column_1r(const SmallArgs &a, int nbp, double *Lsm, double *r2s, double *r3s, double *qs,
                                  double *hcol, double *tmp, double *lf2)
{
    __shared__ double s_hn2;
    __shared__ int s_stop;
    DevState *st = a.st;
    const int t = threadIdx.x;
    const double ig = st->inv_gamma, g2 = st->lag_g2, lf2_prev = a.lfro2[nbp - 1];
    for (int c = t; c < nbp; c += blockDim.x) {
        r2s[c] = a.r2v[c];
        qs[c] = nbp == 1 ? a.H[0] : a.r3v[c];
    }
    const int terms = neumann_terms(lf2_prev);
    const bool f32 = neumann_fp32(lf2_prev, nbp, terms);
    lower_wait();  // also orders the loads above before their use
    unit_lower_solve(Lsm, nbp, r2s, r3s, tmp, terms, f32);
    for (int c = t; c < nbp; c += blockDim.x) {
        const double h = qs[c] + r3s[c];
        a.H[(int64_t)(nbp - 1) * a.ldh + c] = h;
        hcol[c] = h;
    }
    __syncthreads();
    if (t < 32) {
        double hn2 = 0.0;
        for (int c = t; c < nbp; c += 32) hn2 = fma(hcol[c], hcol[c], hn2);
        for (int o = 16; o > 0; o >>= 1) hn2 += __shfl_down_sync(0xffffffffu, hn2, o);
        if (t == 0) {
            int stop = st->stop_reason;  // the previous launch's own stop (this column still completes)
            if (stop == 0 && g2 <= kBreakdownFactor * kBreakdownFactor * hn2) {
                stop = 2;
                st->halt = 1;
                st->stop_reason = 2;
                st->stop_cols = nbp;
            }
            s_stop = stop;
        }
    }
    __syncthreads();
    if (s_stop != 0) return s_stop;
    // step 9: L row nbp = r^(2) / gamma
    if (t < 32) {
        double rowsq = 0.0;
        for (int c = t; c < nbp; c += 32) {
            const double l = r2s[c] * ig;
            a.L[(int64_t)c * a.ldl + nbp] = l;
            a.Lrow[packed_row(nbp) + c] = l;
            Lsm[packed_row(nbp) + c] = l;
            rowsq = fma(l, l, rowsq);
        }
        for (int o = 16; o > 0; o >>= 1) rowsq += __shfl_down_sync(0xffffffffu, rowsq, o);
        if (t == 0) {
            a.lfro2[nbp] = lf2_prev + rowsq;
            *lf2 = lf2_prev + rowsq;
        }
    }
    // step 15: q_i = r^(1)_i - sum_c H(i, c) r^(3)_c / gamma over the columns c < nbp
    // (H(i, c) = 0 for i > c+1; column nbp-1 is hcol with H_{nbp, nbp-1} = gamma)
    for (int c = t; c < nbp; c += blockDim.x) r3s[c] *= ig;
    __syncthreads();
    for (int i = t; i <= nbp; i += blockDim.x) {
        double hs = 0.0;
        for (int c = i > 0 ? i - 1 : 0; c < nbp - 1; ++c) hs = fma(a.H[(int64_t)c * a.ldh + i], r3s[c], hs);
        hs = fma(i < nbp ? hcol[i] : a.H[(int64_t)(nbp - 1) * a.ldh + nbp], r3s[nbp - 1], hs);
        const double q = a.r1v[i] - hs;
        a.r3v[i] = q;
        qs[i] = q;
    }
    __syncthreads();
    return 0;
}

// Iteration k = nb+2 of Alg. 4.2, steps 6-8 and 12 (what the fused update needs), after the
// previous iteration's column has been completed in the prologue (complete_column_1r):
//   gamma^2 = ||u||^2 - ||r^(2)||^2 (lagged norm), 1/gamma, H_{nb, nb-1} = gamma,
//   r^(1) = [V^T A u / gamma; u.A u / gamma^2 - r^(2).(V^T A u) / gamma^2] (Stephen's trick:
//   the last entry is r^(0)_nb - L_nb . r^(0)_{0:nb-1} with L_nb = r^(2) / gamma).
// Stops the cycle where gamma^2 is not finite (IGS_ENUMERIC) or gamma = 0 (breakdown).
// Outputs: r2v = r^(2), r1v = r^(1), st->inv_gamma, st->lag_g2 = gamma^2.
// With flush (nb = m, the reduction of u_{m+1}: value c < m is V[:,c].u, value m is ||u||^2)
// the column m-1 is completed here as well (steps 5, 9 and 14; no r^(1)), for the last
// v_{m+1} = (u - V_m r^(2)) / gamma.
__global__ void __launch_bounds__(kSmallThreads) k_step_1r(SmallArgs a, int nb, int flush, int nrb)
{
    extern __shared__ __align__(16) double dsm[];
    double *buf = dsm;              // r^(2) of the previous iteration, then the combined partials
    double *r3s = buf + (nb + 1);   // (with buf: 2 nb + 2 partials)
    double *qs = r3s + (nb + 1);    // q of the column being completed
    double *hcol = qs + nb;         // that column
    double *tmp = hcol + nb;        // solve scratch (nb + 1)
    double *Lsm = dsm + ((5 * nb + 4) & ~1);  // row-packed L (16-byte aligned)
    __shared__ double s_ig, s_g2, s_r1last, s_lf2, s_hn2;
    __shared__ int s_stop, s_pro;
    DevState *st = a.st;
    const int t = threadIdx.x;
    const int nbp = nb - 1;
    // ---- prologue: everything read here was written by launches that completed before the
    // multi-dot this kernel follows was launched
    lower_prefetch(a.Lrow, nbp, Lsm);  // rows 0..nb-2
    if (nb >= 2) {
        // completes column nb-2 unless an earlier column already ended the cycle
        const bool skip = st->stop_reason != 0 && st->stop_cols < nbp;
        int pro = skip ? 1 : complete_column_1r(a, nbp, Lsm, buf, r3s, qs, hcol, tmp, &s_lf2);
        if (t == 0) s_pro = pro;
    } else {
        if (t == 0) {
            qs[0] = a.H[0];
            s_lf2 = a.lfro2[0];
            s_pro = 0;
        }
    }
    lower_drain();
    __syncthreads();
    IGS_PDL_ENTER();
    if (s_pro != 0 || halted(st)) return;
    if (st->stop_reason != 0) {  // the previous column met the stop test
        if (t == 0) st->halt = 1;
        return;
    }
    const int nv = flush ? nb + 1 : 2 * (nb + 1);
    reduce_partials(a.part, nv, nrb, buf);
    if (t < 32) {
        // ||r^(2)||^2 and r^(2).(V^T A u) (fixed shuffle trees), then the scalars on lane 0
        // (1/gamma by rsqrt: no DSQRT or DDIV)
        double rr = 0.0, dr = 0.0;
        for (int c = t; c < nb; c += 32) {
            rr = fma(buf[c], buf[c], rr);
            if (!flush) dr = fma(buf[c], buf[nb + 1 + c], dr);
        }
        for (int o = 16; o > 0; o >>= 1) {
            rr += __shfl_down_sync(0xffffffffu, rr, o);
            dr += __shfl_down_sync(0xffffffffu, dr, o);
        }
        if (t == 0) {
            const double g2 = buf[nb] - rr;
            int stop = 0;
            double ig = 0.0;
            if (g2 != g2 || isinf(g2)) {
                stop = -4;
            } else {
                double gam = 0.0;
                if (g2 > 0.0) {
                    ig = rsqrt(g2);
                    gam = g2 * ig;
                }
                a.H[(int64_t)(nb - 1) * a.ldh + nb] = gam;
                if (gam == 0.0) stop = 2;
            }
            if (stop != 0 && !(flush && stop == 2)) {  // the flush decides breakdown below
                st->halt = 1;
                st->stop_reason = stop;
                st->stop_cols = nb;
            }
            st->inv_gamma = ig;
            st->lag_g2 = g2;
            s_ig = ig;
            s_g2 = g2;
            s_r1last = flush ? 0.0 : (buf[2 * nb + 1] - dr) * (ig * ig);
            s_stop = stop;
        }
    }
    __syncthreads();
    if (s_stop < 0) return;
    const double ig = s_ig;
    if (!flush) {
        // r^(2) also where gamma = 0 ended the cycle: the next launch completes this column
        for (int c = t; c < nb; c += blockDim.x) a.r2v[c] = buf[c];
        if (s_stop != 0) return;
        for (int c = t; c < nb; c += blockDim.x) a.r1v[c] = buf[nb + 1 + c] * ig;
        if (t == 0) a.r1v[nb] = s_r1last;
        return;
    }
    // ---- the flush: column m-1 (q in qs, L_m in Lsm with row m-1 from the prologue)
    const int terms = neumann_terms(s_lf2);
    const bool f32 = neumann_fp32(s_lf2, nb, terms);
    unit_lower_solve(Lsm, nb, buf, r3s, tmp, terms, f32);
    for (int c = t; c < nb; c += blockDim.x) {
        const double h = qs[c] + r3s[c];
        a.H[(int64_t)(nb - 1) * a.ldh + c] = h;
        hcol[c] = h;
    }
    __syncthreads();
    if (t < 32) {
        double hn2 = 0.0;
        for (int c = t; c < nb; c += 32) hn2 = fma(hcol[c], hcol[c], hn2);
        for (int o = 16; o > 0; o >>= 1) hn2 += __shfl_down_sync(0xffffffffu, hn2, o);
        if (t == 0) {
            s_hn2 = hn2;
            if (s_stop != 0 || s_g2 <= kBreakdownFactor * kBreakdownFactor * hn2) {
                st->halt = 1;
                st->stop_reason = 2;
                st->stop_cols = nb;
                s_stop = 2;
            }
        }
    }
    __syncthreads();
    if (s_stop != 0) return;
    if (t < 32) {
        double rowsq = 0.0;
        for (int c = t; c < nb; c += 32) {
            const double l = buf[c] * ig;
            a.L[(int64_t)c * a.ldl + nb] = l;
            a.Lrow[packed_row(nb) + c] = l;
            rowsq = fma(l, l, rowsq);
        }
        for (int o = 16; o > 0; o >>= 1) rowsq += __shfl_down_sync(0xffffffffu, rowsq, o);
        if (t == 0) a.lfro2[nb] = s_lf2 + rowsq;
    }
    for (int c = t; c < nb; c += blockDim.x) a.r2v[c] = buf[c];
}

// Steps 10-11 and 13 in one pass over V_nb (two FMAs per basis element):
//   v = (u - V_nb r^(2)) / gamma into V[:, nb] (in place of u),
//   u_new = z / gamma - V_nb r^(1)_{0:nb-1} - v r^(1)_nb into V[:, nb+1] (when vonly == 0).
__global__ void __launch_bounds__(kStreamThreads)
k_update_1r(double *V, int64_t ld, int nb, int64_t n, const double *__restrict__ r2,
            const double *__restrict__ r1, const double *__restrict__ z, int vonly, const DevState *st)
{
    IGS_PDL_ENTER();
    if (halted(st)) return;
    extern __shared__ double sc[];  // r2 (nb), r1 (nb + 1)
    double *s2 = sc, *s1 = sc + nb;
    for (int c = threadIdx.x; c < nb; c += blockDim.x) s2[c] = r2[c];
    if (!vonly)
        for (int c = threadIdx.x; c <= nb; c += blockDim.x) s1[c] = r1[c];
    __syncthreads();
    const double ig = st->inv_gamma;
    // block b owns rows [b rpb, (b+1) rpb) (one row per thread with the launcher's grid; this
    // form measured 7 % faster than the equivalent grid-stride loop)
    const int64_t rpb = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i_lo = (int64_t)blockIdx.x * rpb;
    const int64_t i_hi = i_lo + rpb < n ? i_lo + rpb : n;
    for (int64_t i = i_lo + threadIdx.x; i < i_hi; i += blockDim.x) {
        const double *vi = V + i;
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
        int c = 0;
        if (nb >= 4) {
            // software pipeline: the next 4 columns load while these 4 are used
            double v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = vi[(int64_t)q * ld];
            for (;; c += 4) {
                const bool more = c + 7 < nb;
                double nv[4];
                if (more) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) nv[q] = vi[(int64_t)(c + 4 + q) * ld];
                }
                a0 = fma(v[0], s2[c], a0);
                a1 = fma(v[1], s2[c + 1], a1);
                a0 = fma(v[2], s2[c + 2], a0);
                a1 = fma(v[3], s2[c + 3], a1);
                if (!vonly) {
                    b0 = fma(v[0], s1[c], b0);
                    b1 = fma(v[1], s1[c + 1], b1);
                    b0 = fma(v[2], s1[c + 2], b0);
                    b1 = fma(v[3], s1[c + 3], b1);
                }
                if (!more) break;
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = nv[q];
            }
            c += 4;
        }
        for (; c < nb; ++c) {
            const double v = vi[(int64_t)c * ld];
            a0 = fma(v, s2[c], a0);
            if (!vonly) b0 = fma(v, s1[c], b0);
        }
        double *un = V + (int64_t)nb * ld + i;
        const double vnew = (*un - (a0 + a1)) * ig;
        *un = vnew;
        if (!vonly) V[(int64_t)(nb + 1) * ld + i] = fma(z[i], ig, -((b0 + b1) + vnew * s1[nb]));
    }
}

// Givens least squares for column j (Sec. 1 eq. "llse"; the paper names no method).
// The j earlier rotations are applied to the new column as a parallel scan: rotation i maps
// the running entry a_i to a_{i+1} = -s_i a_i + c_i h_{i+1} and emits c_i a_i + s_i h_{i+1};
// the affine maps a -> alpha a + beta compose associatively, so a block-wide scan replaces
// the j-long dependent chain.  Then the new rotation, the rotated right-hand side g, the
// Arnoldi residual |g_{j+1}|, the history, and the in-cycle stop test
// |g_{j+1}| <= tol (||b|| + ||A|| ||x0||).
__global__ void __launch_bounds__(kGivensThreads) k_givens(SmallArgs a, int j)
{
    IGS_PDL_ENTER();
    DevState *st = a.st;
    const int stop_cols = st->stop_cols;
    if (st->stop_reason < 0) return;
    if (stop_cols > 0 && j >= stop_cols) return;
    constexpr int T = kGivensThreads;
    constexpr int E = (kMaxRestart + T - 1) / T;  // maps per thread (upper bound)
    __shared__ double h[kMaxRestart + 2];
    __shared__ double wA[T / 32], wB[T / 32];
    __shared__ double s_last;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const double *col = a.H + (int64_t)j * a.ldh;
    for (int i = t; i <= j + 1; i += T) h[i] = col[i];
    __syncthreads();
    // thread t owns maps [t*e, min(j, (t+1)*e)) with e = ceil(j / T)
    const int e = (j + T - 1) / T;
    const int m0 = t * e, m1 = min(j, m0 + e);
    double cA = 1.0, cB = 0.0;  // composition of the owned maps: a -> cA a + cB
    double cc[E], ss[E];
    for (int q = 0; q < e && m0 + q < m1; ++q) {
        cc[q] = a.cs[m0 + q];
        ss[q] = a.sn[m0 + q];
        const double al = -ss[q], be = cc[q] * h[m0 + q + 1];
        cB = fma(al, cB, be);
        cA = al * cA;
    }
    // inclusive warp scan of (cA, cB) under "later o earlier"
    for (int o = 1; o < 32; o <<= 1) {
        const double pA = __shfl_up_sync(0xffffffffu, cA, o);
        const double pB = __shfl_up_sync(0xffffffffu, cB, o);
        if (lane >= o) {
            cB = fma(cA, pB, cB);
            cA = cA * pA;
        }
    }
    if (lane == 31) { wA[wid] = cA; wB[wid] = cB; }
    __syncthreads();
    // exclusive prefix for this thread = (prefix of earlier warps) then earlier lanes
    double eA = 1.0, eB = 0.0;
    for (int q = 0; q < wid; ++q) {
        eB = fma(wA[q], eB, wB[q]);
        eA = wA[q] * eA;
    }
    {
        double pA = __shfl_up_sync(0xffffffffu, cA, 1);
        double pB = __shfl_up_sync(0xffffffffu, cB, 1);
        if (lane == 0) { pA = 1.0; pB = 0.0; }
        // compose: first the earlier warps (eA,eB), then lanes < lane of this warp (pA,pB)
        eB = fma(pA, eB, pB);
        eA = pA * eA;
    }
    double av = fma(eA, h[0], eB);  // running entry entering map m0
    for (int q = 0; q < e && m0 + q < m1; ++q) {
        const int i = m0 + q;
        const double hi1 = h[i + 1];
        a.R[(int64_t)j * a.ldh + i] = fma(cc[q], av, ss[q] * hi1);
        av = fma(-ss[q], av, cc[q] * hi1);
    }
    // the thread owning the last map (or thread 0 when j == 0) holds a_j
    const int owner = j == 0 ? 0 : (j - 1) / e;
    if (t == owner) s_last = j == 0 ? h[0] : av;
    __syncthreads();
    if (t == 0) {
        const double aj = s_last, hj1 = h[j + 1];
        const double r = hypot(aj, hj1);
        double c = 1.0, s = 0.0;
        if (r != 0.0) {
            const double ir = 1.0 / r;
            c = aj * ir;
            s = hj1 * ir;
        }
        a.cs[j] = c;
        a.sn[j] = s;
        a.R[(int64_t)j * a.ldh + j] = r;
        const double gj = a.g[j];
        a.g[j + 1] = -s * gj;
        a.g[j] = c * gj;
        const double res = fabs(s * gj);
        a.hist_res[j] = res;
        a.hist_lfro[j] = sqrt(a.lfro2[j]);
        // in-cycle stop: the estimated backward error meets tol, or (FP32 cycles of the
        // precision form) the cycle reduced its residual by inner_tol
        if (st->stop_reason == 0 &&
            ((st->stop_den > 0.0 && res <= st->tol * st->stop_den) || res <= st->stop_floor)) {
            st->stop_reason = 1;
            st->stop_cols = j + 1;
        }
    }
}

// y = R^{-1} g for the p = (stop_cols or m) columns of the cycle (back substitution,
// column oriented over the block), st->ncols = p.
__global__ void __launch_bounds__(kSmallThreads) k_lsq(SmallArgs a, int m)
{
    IGS_PDL_ENTER();
    DevState *st = a.st;
    __shared__ double ys[kMaxRestart + 1];
    __shared__ int s_p;
    const int T = blockDim.x, t = threadIdx.x;
    if (t == 0) {
        int p = st->stop_reason != 0 ? st->stop_cols : m;
        if (st->stop_reason < 0) p = 0;
        st->ncols = p;
        s_p = p;
    }
    __syncthreads();
    const int p = s_p;
    double gi[4], rinv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = t + T * q;
        gi[q] = i < p ? a.g[i] : 0.0;
        rinv[q] = i < p ? 1.0 / a.R[(int64_t)i * a.ldh + i] : 0.0;
    }
    for (int c = p - 1; c >= 0; --c) {
        if ((c % T) == t) ys[c] = gi[c / T] * rinv[c / T];
        __syncthreads();
        const double yc = ys[c];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = t + T * q;
            if (i < c) gi[q] = fma(-a.R[(int64_t)c * a.ldh + i], yc, gi[q]);
        }
    }
    __syncthreads();
    for (int i = t; i < p; i += T) a.y[i] = ys[i];
}

// Column-major -> row-major copy of a small matrix (the L factor handed to the caller).
__global__ void k_transpose(const double *__restrict__ src, int ld_src, int rows, int cols,
                            double *__restrict__ dst, int ld_dst)
{
    IGS_PDL_ENTER();
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / cols), c = (int)(e % cols);
        dst[(int64_t)i * ld_dst + c] = src[(int64_t)c * ld_src + i];
    }
}

// -------------------------------------------------------------------------------------
// Power iteration for ||A||_2 (create time): x <- A^T A x / ||A^T A x||.
// -------------------------------------------------------------------------------------
__global__ void k_power_init(int64_t n, double *x)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double s = 1.0 / sqrt((double)n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t hsh = (uint64_t)i * 0x9E3779B97F4A7C15ull;
        hsh ^= hsh >> 29;
        x[i] = s * (0.5 + (double)(hsh >> 11) * 0x1p-53);
    }
}

__global__ void __launch_bounds__(kSmallThreads) k_power_norm(const double *part, int nblk, double *lam)
{
    __shared__ double out[1];
    reduce_partials(part, 1, nblk, out);
    if (threadIdx.x == 0) lam[0] = sqrt(out[0]);
}

__global__ void k_power_scale(int64_t n, double *x, const double *lam)
{
    const double f = lam[0] > 0.0 ? 1.0 / lam[0] : 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] *= f;
}

// =====================================================================================
// Host-side launchers.
// =====================================================================================
static int stream_grid(const Workspace &w)
{
    return w.num_sms * kBlocksPerSM;
}

static int dots_slots(const Workspace &w)
{
    return w.num_sms * kDotsBlocksPerSM;
}

DotsPlan plan_dots(const Workspace &w, int p) { return plan_dots_slots(w, p, dots_slots(w)); }

DotsPlan plan_dots_slots(const Workspace &w, int p, int slots)
{
    DotsPlan pl;
    int groups = (p + kDotsColsPerBlock - 1) / kDotsColsPerBlock;
    if (groups > slots) groups = slots;
    if (groups < 1) groups = 1;
    int rblocks = slots / groups;
    const int64_t n4 = (w.n + 3) & ~int64_t(3);
    // at least 64 rows per block
    const int64_t maxrb = (n4 + 63) / 64;
    if (rblocks > maxrb) rblocks = (int)maxrb;
    if (rblocks < 1) rblocks = 1;
    int64_t rows = (n4 + rblocks - 1) / rblocks;
    rows = (rows + 63) & ~int64_t(63);  // 64-row (512-byte) segments of the multi-dot
    rblocks = (int)((n4 + rows - 1) / rows);
    pl.groups = groups;
    pl.rblocks = rblocks;
    pl.rows = rows;
    return pl;
}

cudaError_t launch_spmv(const Workspace &w, const double *x, double *y, const double *b,
                        bool check_halt, cudaStream_t s, float2 *y_df)
{
    // one thread (short rows) or one warp (long rows) per row, so that every row's three
    // dependent loads (row pointer, column index, x) are in flight at once
    const int64_t per_block = w.spmv_warp_rows ? kStreamThreads / 32 : kStreamThreads;
    const int64_t want = (w.n + per_block - 1) / per_block;
    const int grid = (int)(want < (int64_t)1 << 30 ? want : (int64_t)1 << 30);
    if (w.spmv_warp_rows)
        launch_k(false, k_spmv_warp, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.rowptr, w.colind, w.val, x, y, b, w.st,
                 check_halt, y_df);
    else if (w.ell_width > 0) {
        const dim3 g(grid), bl(kStreamThreads);
        const DevState *st = w.st;
        const int ch = check_halt ? 1 : 0;
        switch (w.ell_width) {
        case 1: launch_k(false, k_spmv_ell<1>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        case 2: launch_k(false, k_spmv_ell<2>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        case 3: launch_k(false, k_spmv_ell<3>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        case 4: launch_k(false, k_spmv_ell<4>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        case 5: launch_k(false, k_spmv_ell<5>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        case 6: launch_k(false, k_spmv_ell<6>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        case 7: launch_k(false, k_spmv_ell<7>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        default: launch_k(false, k_spmv_ell<8>, g, bl, 0, s, w.n, w.sell_col, w.sell_val, x, y, b, st, ch, y_df); break;
        }
    } else if (w.sell_col)
        launch_k(false, k_spmv_sell, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.sell_off, w.sell_col, w.sell_val, x, y,
                 b, (const DevState *)w.st, check_halt ? 1 : 0, y_df);
    else
        launch_k(false, k_spmv_rows, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.rowptr, w.colind, w.val, x, y, b, w.st,
                 check_halt, y_df);
    return cudaGetLastError();
}

cudaError_t launch_dots(const Workspace &w, int p, const double *x0, const double *x1,
                        bool check_halt, cudaStream_t s, DotsPlan *plan_out)
{
    const DotsPlan pl = plan_dots(w, p);
    if (plan_out) *plan_out = pl;
    const int64_t n4 = (w.n + 3) & ~int64_t(3);
    dim3 grid(pl.rblocks, pl.groups);
    if (x1)
        launch_k(false, k_dots<2>, dim3(grid), dim3(kStreamThreads), 0, s, w.V, w.ld, p, n4, pl.rows, x0, x1, w.part, w.st,
                                                  check_halt);
    else
        launch_k(false, k_dots<1>, dim3(grid), dim3(kStreamThreads), 0, s, w.V, w.ld, p, n4, pl.rows, x0, nullptr, w.part,
                                                  w.st, check_halt);
    return cudaGetLastError();
}

cudaError_t launch_update(const Workspace &w, int p, const double *coef, bool neg_coef,
                          double alpha, const double *src, double *out, bool norm_last,
                          bool p_from_state, bool check_halt, cudaStream_t s)
{
    const int pmax = p_from_state ? w.mmax + 1 : p;
    const size_t smem = sizeof(double) * (size_t)(pmax > 0 ? pmax : 1);
    // one row per thread: the whole vector is resident at once (occupancy, not a grid-stride
    // loop, hides the loads' latency)
    const int grid = w.num_sms * kUpdateBlocksPerSM;
    launch_k(w.pdl, k_update, dim3(grid), dim3(kStreamThreads), smem, s, w.V, w.ld, p, w.n, coef, neg_coef ? 1 : 0,
                                                          alpha, src, out, norm_last ? 1 : 0,
                                                          p_from_state ? 1 : 0, w.st,
                                                          check_halt ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_norms(const Workspace &w, const double *a, const double *b, const double *c,
                         int *blocks_out, cudaStream_t s)
{
    const int grid = w.num_sms;
    const int nvec = !a ? 0 : !b ? 1 : !c ? 2 : 3;
    launch_k(false, k_norms, dim3(grid), dim3(kStreamThreads), 0, s, w.n, a, b, c, w.part, nvec);
    if (blocks_out) *blocks_out = grid;
    return cudaGetLastError();
}

cudaError_t launch_scale(const Workspace &w, const double *src, double *dst, int which,
                         bool check_halt, cudaStream_t s)
{
    launch_k(false, k_scale, dim3(stream_grid(w)), dim3(kStreamThreads), 0, s, w.n, src, dst, which, w.st, check_halt ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const Workspace &w, double tol, double normA, double inner_tol,
                              cudaStream_t s)
{
    launch_k(w.pdl, k_init_state, dim3(1), dim3(32), 0, s, w.st, tol, normA, inner_tol);
    return cudaGetLastError();
}

cudaError_t launch_bnorm(const Workspace &w, int nblk, cudaStream_t s)
{
    launch_k(w.pdl, k_bnorm, dim3(1), dim3(kSmallThreads), 0, s, w.part, nblk, w.st);
    return cudaGetLastError();
}

cudaError_t launch_beta(const Workspace &w, int nblk, cudaStream_t s)
{
    launch_k(w.pdl, k_beta, dim3(1), dim3(kSmallThreads), 0, s, w.part, nblk, w.st);
    return cudaGetLastError();
}

cudaError_t launch_cycle_start(const Workspace &w, int, cudaStream_t s)
{
    launch_k(w.pdl, k_cycle_start, dim3(1), dim3(kSmallThreads), 0, s, small_args(w), w.mmax);
    return cudaGetLastError();
}

cudaError_t launch_prime(const Workspace &w, const DotsPlan &pl, cudaStream_t s)
{
    launch_k(w.pdl, k_prime, dim3(1), dim3(kSmallThreads), 0, s, small_args(w), pl.rblocks);
    return cudaGetLastError();
}

size_t small_solve_smem(int p, int vecs)
{
    return sizeof(double) * ((size_t)vecs * p + 2 + (size_t)p * (p - 1) / 2);  // + alignment of L
}

cudaError_t configure_kernels(const Workspace &w)
{
    // Dynamic shared-memory limits are raised (never lowered: they are per function, not per
    // context) once per context, before any graph capture, to what the context's largest
    // restart length needs.
    cudaError_t e = raise_smem_limit((const void *)k_step_a, small_solve_smem(w.mmax, 5));
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_step_b, small_solve_smem(w.mmax, 3));
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_step_1r, small_solve_smem(w.mmax + 1, 6));
    return e;
}

cudaError_t launch_step_a(const Workspace &w, int k, int gs, const DotsPlan &pl, cudaStream_t s)
{
    const size_t smem = small_solve_smem(k - 1, 5);
    launch_k(w.pdl, k_step_a, dim3(1), dim3(kSmallThreads), smem, s, small_args(w), k, gs, pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_step_b(const Workspace &w, int k, const DotsPlan &pl, cudaStream_t s)
{
    const size_t smem = small_solve_smem(k - 1, 3);
    launch_k(w.pdl, k_step_b, dim3(1), dim3(kSmallThreads), smem, s, small_args(w), k, pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_flush(const Workspace &w, int m, const DotsPlan &pl, cudaStream_t s)
{
    launch_k(w.pdl, k_flush, dim3(1), dim3(kSmallThreads), 0, s, small_args(w), m, pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_step_1r(const Workspace &w, int nb, bool flush, const DotsPlan &pl, cudaStream_t s)
{
    const size_t smem = small_solve_smem(nb + 1, 6);
    launch_k(w.pdl, k_step_1r, dim3(1), dim3(kSmallThreads), smem, s, small_args(w), nb, flush ? 1 : 0, pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_update_1r(const Workspace &w, int nb, const double *z, bool vonly, cudaStream_t s)
{
    const size_t smem = sizeof(double) * (size_t)(2 * nb + 2);
    const int grid = (int)((w.n + kStreamThreads - 1) / kStreamThreads);
    launch_k(w.pdl, k_update_1r, dim3(grid), dim3(kStreamThreads), smem, s, w.V, w.ld, nb, w.n,
             (const double *)w.r2v, (const double *)w.r1v, z, vonly ? 1 : 0, (const DevState *)w.st);
    return cudaGetLastError();
}

cudaError_t launch_givens(const Workspace &w, int j, cudaStream_t s)
{
    launch_k(w.pdl, k_givens, dim3(1), dim3(kGivensThreads), 0, s, small_args(w), j);
    return cudaGetLastError();
}

cudaError_t launch_lsq(const Workspace &w, int m, cudaStream_t s)
{
    launch_k(w.pdl, k_lsq, dim3(1), dim3(kSmallThreads), 0, s, small_args(w), m);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const double *src, int ld_src, int rows, int cols, double *dst,
                             int ld_dst, cudaStream_t s)
{
    const int64_t total = (int64_t)rows * cols;
    int grid = (int)((total + 255) / 256);
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    launch_k(false, k_transpose, dim3(grid), dim3(256), 0, s, src, ld_src, rows, cols, dst, ld_dst);
    return cudaGetLastError();
}

cudaError_t estimate_norm2(const Workspace &w, const int *at_rowptr, const int *at_colind,
                           const double *at_val, int iters, double *out, cudaStream_t s)
{
    // x: w.t, A x: w.z, A^T (A x): w.u; lambda in w.y[0]
    const int grid = stream_grid(w);
    launch_k(false, k_power_init, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.t);
    for (int it = 0; it < iters; ++it) {
        if (w.spmv_warp_rows) {
            launch_k(false, k_spmv_warp, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.rowptr, w.colind, w.val, w.t, w.z,
                                                        nullptr, w.st, 0, (float2 *)nullptr);
            launch_k(false, k_spmv_warp, dim3(grid), dim3(kStreamThreads), 0, s, w.n, at_rowptr, at_colind, at_val, w.z, w.u,
                                                        nullptr, w.st, 0, (float2 *)nullptr);
        } else {
            launch_k(false, k_spmv_rows, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.rowptr, w.colind, w.val, w.t, w.z,
                                                        nullptr, w.st, 0, (float2 *)nullptr);
            launch_k(false, k_spmv_rows, dim3(grid), dim3(kStreamThreads), 0, s, w.n, at_rowptr, at_colind, at_val, w.z, w.u,
                                                        nullptr, w.st, 0, (float2 *)nullptr);
        }
        launch_k(false, k_norms, dim3(w.num_sms), dim3(kStreamThreads), 0, s, w.n, w.u, nullptr, nullptr, w.part, 1);
        launch_k(false, k_power_norm, dim3(1), dim3(kSmallThreads), 0, s, w.part, w.num_sms, w.y);
        launch_k(false, k_power_scale, dim3(grid), dim3(kStreamThreads), 0, s, w.n, w.u, w.y);
        cudaMemcpyAsync(w.t, w.u, sizeof(double) * (size_t)w.n, cudaMemcpyDeviceToDevice, s);
    }
    double lam = 0.0;
    cudaMemcpyAsync(&lam, w.y, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *out = sqrt(lam);
    return cudaGetLastError();
}

}  // namespace igs
