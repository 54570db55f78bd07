// Device code that solves ONE sparse system by restarted IGS-GMRES(m) (Alg. 4.1) inside a
// kernel, with a gang of G >= 1 CTAs: the batched solver (igs_batch.cu, one CTA per system)
// and the request server (igs_serve.cu, one cooperative launch of G CTAs per request).
//
// Steps (as in the single-system library path): cycle start r = b - A x and the backward
// error of eq. "nrbe"; step 1 (v_1 = r / rho); step 2 (the prime, one projection); the
// k = 3..m+1 loop (step 4 SpMV, step 5 fused reduction, steps 6-11 lagged normalisation,
// steps 12-16 one or two Gauss-Seidel corrections with (I + L), step 17 H column); the Givens
// least squares of eq. "llse" with the in-cycle stop test; the flush that sets H_{m+1,m};
// x_m = x_0 + V_m y_m; breakdown and restart rules.
//
// Basis type T: double (everything FP64), or float (the precision form: FP32 SpMV, basis and
// basis updates; FP64 Gram accumulation over FP32 chunks of at most 32 rows, FP64 (I + L),
// Givens, x and residual r = b - A x; each restart is one step of iterative refinement, and
// an FP32 cycle also stops when its residual estimate fell by inner_tol).
//
// Gang: CTA g of G owns rows [lo, hi) of the system (multiples of 32 except the end).  A dot
// product is summed over fixed slices of the CTA's rows (slice count a function of the
// CTA's row count and the column count), each slice in row order, then over the slices in
// order, then over the gang's CTAs in rank order through a global exchange buffer; every CTA
// then holds the same sums and repeats the small steps (gamma, the L row, the (I + L) solves,
// Givens, back substitution) itself, bit for bit identically.  So a system's result depends
// only on the system, the options and G, and G depends only on the system's size.  The gang
// synchronises twice per step for the reductions and once after the basis update (the next
// SpMV reads other CTAs' rows); every wait is bounded: a CTA that waits too long (or sees
// another CTA's abort) stops the solve with IGS_ETIMEOUT.
#pragma once

#include "../../include/igs.h"
#include "igs_internal.h"

#include <type_traits>

namespace igs {
namespace sysdev {

constexpr int kMaxM = 128;          // largest restart length (four rows per lane in warp solves)
constexpr int kMaxSlices = 16;      // dot products over at most this many slices per CTA
constexpr int kRowAlign = 32;       // gang row ranges start on multiples of 32 rows
constexpr long long kSpinLimit = 1ll << 22;  // bounded gang waits: a few seconds (3.2 s measured)

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

__host__ __device__ inline int slices_hi(int nl)
{
    const int s = (nl >> 1) / 4;  // at least four row pairs per slice
    return s < 1 ? 1 : (s > kMaxSlices ? kMaxSlices : s);
}
__host__ __device__ inline int slices_lo(int nl) { return slices_hi(nl) < 8 ? slices_hi(nl) : 8; }

// Slice count in [slices_lo, slices_hi] whose nsl * pc items leave the fewest idle lanes.
__host__ __device__ inline int pick_slices(int nl, int pc)
{
    int best = slices_lo(nl), best_idle = 0, best_tot = 1;
    for (int s = slices_lo(nl); s <= slices_hi(nl); ++s) {
        const int items = s * pc;
        const int tot = (items + 31) / 32 * 32;
        const int idle = tot - items;
        if (s == slices_lo(nl) || idle * best_tot < best_idle * tot) {
            best = s;
            best_idle = idle;
            best_tot = tot;
        }
    }
    return best;
}

// Shared-memory index of local row i of the Krylov vector z/u: two elements of padding every
// 128 rows put different slices' starts in different banks.
__host__ __device__ inline int pad_idx(int i) { return i + 2 * (i >> 7); }

// Packed strictly-lower L of order m+1, column-major: column c holds rows c+1..m.
__host__ __device__ inline int lower_base(int c, int m) { return c * m - c * (c - 1) / 2 - c - 1; }
// Packed upper R (order m), column-major: column j holds rows 0..j.
__host__ __device__ inline int upper_base(int j) { return j * (j + 1) / 2; }

// Dynamic shared memory (in doubles) for a CTA with at most nl local rows and restart m.
struct SmemLayout {
    int zu, part, L, red, r0, r1, r3, hcol, cs, sn, g, y, total;
};

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int nl, int m)
{
    SmemLayout s;
    int o = 0;
    const int zu_elems = round_up(pad_idx(round_up(nl, 2)) + 2, 2);
    s.zu = o;   o += round_up((int)((zu_elems * sizeof(T) + 7) / 8), 2);
    s.part = o; o += round_up(kMaxSlices * (m + 1) * 2, 2);
    s.L = o;    o += round_up((m + 1) * m / 2 + 1, 2);
    s.red = o;  o += round_up(2 * (m + 1) + 2, 2);
    s.r0 = o;   o += round_up(m + 1, 2);
    s.r1 = o;   o += round_up(m + 1, 2);
    s.r3 = o;   o += round_up(m + 1, 2);
    s.hcol = o; o += round_up(m + 2, 2);
    s.cs = o;   o += round_up(m + 1, 2);
    s.sn = o;   o += round_up(m + 1, 2);
    s.g = o;    o += round_up(m + 2, 2);
    s.y = o;    o += round_up(m + 1, 2);
    s.total = o;
    return s;
}

// Gang synchronisation words (zeroed before the launch).
struct GangSync {
    unsigned int count;
    unsigned int gen;
    int abort;
    int pad;
};

// Everything one system's solve needs (device pointers; vectors system-local).
template <typename T>
struct SysArgs {
    int n, m, gs, max_cycles;
    int ldv;                      // leading dimension of V (multiple of 4)
    double tol, inner_tol, normA;
    const int64_t *sell_off;      // the system's SELL-32 slice offsets (slice k at sell_off[k])
    const int *sell_col;          // system-local column, -1 = padding
    const double *sell_val;       // FP64 values (residual; the SpMV when T = double)
    const float *sell_val32;      // FP32 values (the SpMV when T = float)
    const double *b;
    const double *x0;             // nullable
    double *x;
    T *V;                         // ldv x (m+1)
    double *r64;                  // FP64 residual (T = float; length >= n)
    double *beta_out;
    int *status_out;
    int64_t *steps_out;
    int *cycles_out;
};

// This CTA's place in its gang.
struct Gang {
    int G, g, lo, hi;             // rank, and rows [lo, hi) of the system
    GangSync *sync;               // null when G == 1
    double *gpart;                // 2 x G x gld exchange buffer (G > 1)
    int gld;
    double *R;                    // this CTA's Givens factor (packed upper, m(m+1)/2)
};

// Block-uniform state.
struct Shared {
    double nb, rho, inv, stop_den, stop_floor, beta;
    int status, cst, done, stop, cycles, ok, swarp;
    unsigned int gen;             // this CTA's gang barrier generation
    int xbuf;                     // exchange buffer parity
    long long steps;
};

static __device__ __forceinline__ double2 ld2(const double *p) { return *reinterpret_cast<const double2 *>(p); }
static __device__ __forceinline__ void st2(double *p, double2 v) { *reinterpret_cast<double2 *>(p) = v; }
static __device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
static __device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

// ---- gang synchronisation -------------------------------------------------------------
// Barrier over the gang's CTAs (all co-resident: cooperative launch).  Returns false (on
// every thread of the CTA) when the wait gave up or another CTA aborted.
static __device__ bool gang_barrier(const Gang &gg, Shared &sh)
{
    __syncthreads();
    if (gg.G <= 1) return sh.ok != 0;
    if (threadIdx.x == 0) {
        GangSync *gs = gg.sync;
        const unsigned target = sh.gen + 1;
        int ok = sh.ok;
        if (ok) {
            __threadfence();
            const unsigned arrived = atomicAdd(&gs->count, 1u) + 1u;
            if (arrived == (unsigned)gg.G) {
                atomicExch(&gs->count, 0u);
                __threadfence();
                atomicExch(&gs->gen, target);
            } else {
                long long spins = 0;
                while (atomicAdd(&gs->gen, 0u) != target) {
                    if (atomicAdd(&gs->abort, 0) != 0) {
                        ok = 0;
                        break;
                    }
                    if (++spins > kSpinLimit) {
                        atomicExch(&gs->abort, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
        }
        sh.gen = target;
        sh.ok = ok;
    }
    __syncthreads();
    return sh.ok != 0;
}

// red[0..nv) (this CTA's sums) becomes the gang's sums (rank order).  False on abort.
static __device__ bool gang_combine(const Gang &gg, Shared &sh, double *red, int nv)
{
    if (gg.G <= 1) return sh.ok != 0;
    double *buf = gg.gpart + (size_t)sh.xbuf * gg.G * gg.gld;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) buf[(size_t)gg.g * gg.gld + v] = red[v];
    const bool ok = gang_barrier(gg, sh);
    if (ok) {
        for (int v = threadIdx.x; v < nv; v += blockDim.x) {
            double acc = 0.0;
            for (int h = 0; h < gg.G; ++h) acc += __ldcg(buf + (size_t)h * gg.gld + v);
            red[v] = acc;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) sh.xbuf ^= 1;
    __syncthreads();
    return ok;
}

// ---- streaming steps over this CTA's rows ----------------------------------------------
// Loads of vector entries that other CTAs of the gang write (the SpMV's gathers): through L2
// (L1 is not coherent across SMs) when the gang has more than one CTA.
template <typename T>
__device__ __forceinline__ T ld_shared_vec(const T *p, bool cg)
{
    return cg ? __ldcg(p) : *p;
}

// y[i] = (A x)_i or b_i - (A x)_i for rows i in [lo, hi) (rows >= n give 0); each row summed
// in its CSR order, eight entries in flight.  Y: shared (local index, padded) or global.
template <typename TV, typename TA, typename TX, typename TY, bool OUT_SMEM>
__device__ void d_spmv(const SysArgs<TV> &a, const Gang &gg, const TA *val, const TX *x, const double *b,
                       TY *y)
{
    for (int i = gg.lo + threadIdx.x; i < gg.hi; i += blockDim.x) {
        TY out = 0;
        if (i < a.n) {
            int64_t e = a.sell_off[i >> 5] + (i & 31);
            const int64_t e1 = a.sell_off[(i >> 5) + 1];
            TA acc = 0;
            for (; e < e1; e += 256) {
                int c[8];
                TA v[8], xv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const bool in = e + 32 * u < e1;
                    c[u] = in ? a.sell_col[e + 32 * u] : -1;
                    v[u] = in ? val[e + 32 * u] : (TA)0;
                }
                const bool cg = gg.G > 1;
#pragma unroll
                for (int u = 0; u < 8; ++u) xv[u] = c[u] >= 0 ? (TA)ld_shared_vec(x + c[u], cg) : (TA)0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
            }
            out = b ? (TY)(b[i] - (double)acc) : (TY)acc;
        }
        if (OUT_SMEM) y[pad_idx(i - gg.lo)] = out;
        else y[i] = out;
    }
}

// Products of a slice [i0, i1) (even bounds).  FP64: two interleaved chains per vector over
// the whole slice.  FP32: sums of at most 32 rows (16 pairs) in FP32, each added to the FP64
// accumulator.
template <typename T, int NQ, bool X0SMEM>
__device__ void slice_dot(const T *vc, const T *x0, const T *x1, int lo, int i0, int i1, double &d0,
                          double &d1)
{
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    if constexpr (sizeof(T) == 8) {
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
        int i = i0;
        for (; i + 8 <= i1; i += 8) {
            T2 v[4], xa[4], xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = ld2(vc + i + 2 * u);
                xa[u] = ld2(x0 + (X0SMEM ? pad_idx(i + 2 * u - lo) : i + 2 * u));
                if (NQ == 2) xb[u] = ld2(x1 + pad_idx(i + 2 * u - lo));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a0 = fma(v[u].x, xa[u].x, a0);
                a1 = fma(v[u].y, xa[u].y, a1);
                if (NQ == 2) {
                    b0 = fma(v[u].x, xb[u].x, b0);
                    b1 = fma(v[u].y, xb[u].y, b1);
                }
            }
        }
        for (; i < i1; i += 2) {
            const T2 v = ld2(vc + i);
            const T2 xa = ld2(x0 + (X0SMEM ? pad_idx(i - lo) : i));
            a0 = fma(v.x, xa.x, a0);
            a1 = fma(v.y, xa.y, a1);
            if (NQ == 2) {
                const T2 xb = ld2(x1 + pad_idx(i - lo));
                b0 = fma(v.x, xb.x, b0);
                b1 = fma(v.y, xb.y, b1);
            }
        }
        d0 = a0 + a1;
        d1 = b0 + b1;
    } else {
        double a = 0.0, b = 0.0;
        for (int c0 = i0; c0 < i1; c0 += 32) {
            const int c1 = c0 + 32 < i1 ? c0 + 32 : i1;
            float p0 = 0.f, p1 = 0.f, q0 = 0.f, q1 = 0.f;
            int i = c0;
            for (; i + 8 <= c1; i += 8) {
                T2 v[4], xa[4], xb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v[u] = ld2(vc + i + 2 * u);
                    xa[u] = ld2(x0 + (X0SMEM ? pad_idx(i + 2 * u - lo) : i + 2 * u));
                    if (NQ == 2) xb[u] = ld2(x1 + pad_idx(i + 2 * u - lo));
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    p0 = fmaf(v[u].x, xa[u].x, p0);
                    p1 = fmaf(v[u].y, xa[u].y, p1);
                    if (NQ == 2) {
                        q0 = fmaf(v[u].x, xb[u].x, q0);
                        q1 = fmaf(v[u].y, xb[u].y, q1);
                    }
                }
            }
            for (; i < c1; i += 2) {
                const T2 v = ld2(vc + i);
                const T2 xa = ld2(x0 + (X0SMEM ? pad_idx(i - lo) : i));
                p0 = fmaf(v.x, xa.x, p0);
                p1 = fmaf(v.y, xa.y, p1);
                if (NQ == 2) {
                    const T2 xb = ld2(x1 + pad_idx(i - lo));
                    q0 = fmaf(v.x, xb.x, q0);
                    q1 = fmaf(v.y, xb.y, q1);
                }
            }
            a += (double)(p0 + p1);
            b += (double)(q0 + q1);
        }
        d0 = a;
        d1 = b;
    }
}

// red[c*NQ + q] = V[:, c]^T X_q over the gang's rows for c < pc (X_0 = x0, global or the
// padded shared vector; X_1 = x1, shared), then over the gang.  FP64 basis: (column, slice)
// items, one thread each, slices summed in order.  FP32 basis: whole columns per warp (see
// below).  False on a gang abort.
template <typename T, int NQ, bool X0SMEM>
__device__ bool d_dots(const Gang &gg, Shared &sh, int ldv, const T *V, int pc, const T *x0, const T *x1,
                       double *part, double *red)
{
    const int nl = gg.hi - gg.lo;
    if constexpr (sizeof(T) == 4) {
        // FP32 basis (bandwidth-bound): a warp streams whole columns over the CTA's rows with
        // coalesced loads; lane l takes row pairs l, l + 32, ...; its products are summed in
        // FP32 over chunks of 16 pairs and each chunk is added to the lane's FP64 sum; a fixed
        // FP64 shuffle tree then combines the lanes.  Independent of the block size.
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int npairs = nl >> 1;
        for (int c = wid; c < pc; c += nw) {
            const T *vc = V + (int64_t)c * ldv + gg.lo;
            double s0 = 0.0, s1 = 0.0;
            for (int base = 0; base < npairs; base += 32 * 16) {
                float p0 = 0.f, q0 = 0.f;
#pragma unroll 4
                for (int k = 0; k < 16; ++k) {
                    const int pr = base + 32 * k + lane;
                    if (pr < npairs) {
                        const float2 v = ld2(vc + 2 * pr);
                        const float2 xa = ld2(x0 + (X0SMEM ? pad_idx(2 * pr) : gg.lo + 2 * pr));
                        p0 = fmaf(v.x, xa.x, p0);
                        p0 = fmaf(v.y, xa.y, p0);
                        if (NQ == 2) {
                            const float2 xb = ld2(x1 + pad_idx(2 * pr));
                            q0 = fmaf(v.x, xb.x, q0);
                            q0 = fmaf(v.y, xb.y, q0);
                        }
                    }
                }
                s0 += (double)p0;
                s1 += (double)q0;
            }
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                if (NQ == 2) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (lane == 0) {
                red[c * NQ] = s0;
                if (NQ == 2) red[c * NQ + 1] = s1;
            }
        }
        __syncthreads();
    } else {
        const int nsl = pick_slices(nl, pc);
        const int npairs = nl >> 1;
        const int nitems = pc * nsl;
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int c = it % pc, s = it / pc;
            const int i0 = gg.lo + 2 * (s * npairs / nsl);
            const int i1 = gg.lo + 2 * ((s + 1) * npairs / nsl);
            double d0, d1;
            slice_dot<T, NQ, X0SMEM>(V + (int64_t)c * ldv, x0, x1, gg.lo, i0, i1, d0, d1);
            part[(s * pc + c) * NQ] = d0;
            if (NQ == 2) part[(s * pc + c) * NQ + 1] = d1;
        }
        __syncthreads();
        for (int v = threadIdx.x; v < pc * NQ; v += blockDim.x) {
            double acc = 0.0;
            for (int s = 0; s < nsl; ++s) acc += part[s * pc * NQ + v];
            red[v] = acc;
        }
        __syncthreads();
    }
    return gang_combine(gg, sh, red, pc * NQ);
}

// red[q] = ||v_q||^2 over the gang's rows for up to two FP64 or T vectors (any alignment).
template <typename A0, typename A1>
__device__ bool d_sumsq(const Gang &gg, Shared &sh, int n, const A0 *v0, const A1 *v1, int nv, double *part,
                        double *red)
{
    const int lo = gg.lo, hi = gg.hi < n ? gg.hi : n;
    const int nl = hi > lo ? hi - lo : 0;
    const int nsl = slices_hi(gg.hi - gg.lo);
    const int nitems = nv * nsl;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
        const int q = it % nv, s = it / nv;
        const int i0 = lo + s * nl / nsl, i1 = lo + (s + 1) * nl / nsl;
        double a0 = 0.0, a1 = 0.0;
        int i = i0;
        for (; i + 1 < i1; i += 2) {
            const double u0 = q == 0 ? (double)v0[i] : (double)v1[i];
            const double u1 = q == 0 ? (double)v0[i + 1] : (double)v1[i + 1];
            a0 = fma(u0, u0, a0);
            a1 = fma(u1, u1, a1);
        }
        if (i < i1) {
            const double u0 = q == 0 ? (double)v0[i] : (double)v1[i];
            a0 = fma(u0, u0, a0);
        }
        part[s * nv + q] = a0 + a1;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < nsl; ++s) acc += part[s * nv + q];
        red[q] = acc;
    }
    __syncthreads();
    return gang_combine(gg, sh, red, nv);
}

// out[i] = alpha * src[i] - sum_{c < pc} V[i, c] coef[c] for rows [lo, hi) (two per thread).
// When nc >= 0 (then nc = pc - 1) column nc is first scaled in place by scale_nc (step 7) and
// enters the sum last; its store precedes the other columns' loads.  SRC/OUT: shared (local,
// padded) or global.
template <typename T, bool SRC_SMEM, bool OUT_SMEM>
__device__ void d_update(const Gang &gg, int ldv, T *V, int pc, const double *coef, double alpha, const T *src,
                         T *out, int nc, double scale_nc)
{
    const int lo = gg.lo, npairs = (gg.hi - gg.lo) >> 1;
    const int ps = nc >= 0 ? nc : pc;
    const T a = (T)alpha, sn = (T)scale_nc;
    for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
        const int i = lo + 2 * pr;
        typename std::conditional<sizeof(T) == 8, double2, float2>::type vn;
        vn.x = 0;
        vn.y = 0;
        if (nc >= 0) {
            vn = ld2(V + (int64_t)nc * ldv + i);
            vn.x *= sn;
            vn.y *= sn;
            st2(V + (int64_t)nc * ldv + i, vn);
        }
        T sx = 0, sy = 0;
        int c = 0;
        for (; c + 4 <= ps; c += 4) {
            typename std::conditional<sizeof(T) == 8, double2, float2>::type v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ld2(V + (int64_t)(c + u) * ldv + i);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T cf = (T)coef[c + u];
                sx = fma(v[u].x, cf, sx);
                sy = fma(v[u].y, cf, sy);
            }
        }
        for (; c < ps; ++c) {
            const auto v = ld2(V + (int64_t)c * ldv + i);
            const T cf = (T)coef[c];
            sx = fma(v.x, cf, sx);
            sy = fma(v.y, cf, sy);
        }
        if (nc >= 0) {
            const T cf = (T)coef[nc];
            sx = fma(vn.x, cf, sx);
            sy = fma(vn.y, cf, sy);
        }
        const auto sv = ld2(src + (SRC_SMEM ? pad_idx(i - lo) : i));
        decltype(vn) o;
        o.x = a * sv.x - sx;
        o.y = a * sv.y - sy;
        st2(out + (OUT_SMEM ? pad_idx(i - lo) : i), o);
    }
}

// x[i] = x[i] + sum_{c < p} V[i, c] y[c] in FP64 for the gang's rows i < n.
template <typename T>
__device__ void d_xupdate(const Gang &gg, int n, int ldv, const T *V, int p, const double *y, double *x)
{
    const int hi = gg.hi < n ? gg.hi : n;
    for (int i = gg.lo + threadIdx.x; i < hi; i += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < p; ++c) s = fma((double)V[(int64_t)c * ldv + i], y[c], s);
        x[i] = x[i] + s;
    }
}

// ---- single-warp steps -----------------------------------------------------------------
// The warp steps hold RL rows (or Givens maps) per lane: RL = 2 for m <= 64, 4 for m <= 128.
template <int RL>
static __device__ __forceinline__ double pick(const double (&x)[RL], int k)
{
    double r = x[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
        if (k == q) r = x[q];
    return r;
}

// out = (I + L_p)^{-1} rhs by forward substitution (steps 12, 15); lane l owns rows l + 32k.
template <int RL>
static __device__ void w_lower_solve(int p, const double *L, int m, const double *rhs, double *out)
{
    const int lane = threadIdx.x & 31;
    double x[RL];
#pragma unroll
    for (int k = 0; k < RL; ++k) x[k] = lane + 32 * k < p ? rhs[lane + 32 * k] : 0.0;
    for (int c = 0; c + 1 < p; ++c) {
        const double xc = __shfl_sync(0xffffffffu, pick<RL>(x, c >> 5), c & 31);
        const int base = lower_base(c, m);
#pragma unroll
        for (int k = 0; k < RL; ++k) {
            if (32 * k + 31 <= c || 32 * k >= p) continue;  // no row of this group below c
            const int i = lane + 32 * k;
            if (i > c && i < p) x[k] = fma(-L[base + i], xc, x[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < RL; ++k)
        if (lane + 32 * k < p) out[lane + 32 * k] = x[k];
}

// y = R_p^{-1} g by back substitution (R packed upper).
template <int RL>
static __device__ void w_upper_solve(int p, const double *R, const double *g, double *y)
{
    const int lane = threadIdx.x & 31;
    double a[RL];
#pragma unroll
    for (int k = 0; k < RL; ++k) a[k] = lane + 32 * k < p ? g[lane + 32 * k] : 0.0;
    for (int c = p - 1; c >= 0; --c) {
        const int ol = c & 31;
        const int base = upper_base(c);
        double yc = 0.0;
        if (lane == ol) yc = pick<RL>(a, c >> 5) / R[base + c];
        yc = __shfl_sync(0xffffffffu, yc, ol);
        if (lane == 0) y[c] = yc;
#pragma unroll
        for (int k = 0; k < RL; ++k) {
            if (32 * k >= c) continue;
            const int i = lane + 32 * k;
            if (i < c) a[k] = fma(-R[base + i], yc, a[k]);
        }
    }
}

// Bring Hessenberg column j (h[0..j], subdiagonal hsub) into the Givens QR (eq. "llse"): the
// j earlier rotations as a warp scan of the affine maps a -> -s_i a + c_i h_{i+1} (lane l owns
// maps RL*l ..), then the new rotation.  Returns |g_{j+1}| on every lane.
template <int RL>
static __device__ double w_givens(int j, const double *h, double hsub, double *cs, double *sn, double *g, double *R)
{
    const int lane = threadIdx.x & 31;
    const int m0 = RL * lane;
    double cA = 1.0, cB = 0.0;
#pragma unroll
    for (int q = 0; q < RL; ++q) {
        const int i = m0 + q;
        if (i < j) {
            const double al = -sn[i], be = cs[i] * h[i + 1];
            cB = fma(al, cB, be);
            cA = al * cA;
        }
    }
    for (int o = 1; o < 32; o <<= 1) {
        const double pA = __shfl_up_sync(0xffffffffu, cA, o);
        const double pB = __shfl_up_sync(0xffffffffu, cB, o);
        if (lane >= o) {
            cB = fma(cA, pB, cB);
            cA = cA * pA;
        }
    }
    double eA = __shfl_up_sync(0xffffffffu, cA, 1);
    double eB = __shfl_up_sync(0xffffffffu, cB, 1);
    if (lane == 0) {
        eA = 1.0;
        eB = 0.0;
    }
    double av = fma(eA, h[0], eB);
    const int rb = upper_base(j);
#pragma unroll
    for (int q = 0; q < RL; ++q) {
        const int i = m0 + q;
        if (i < j) {
            const double hi1 = h[i + 1];
            R[rb + i] = fma(cs[i], av, sn[i] * hi1);
            av = fma(-sn[i], av, cs[i] * hi1);
        }
    }
    const double aj = j == 0 ? h[0] : __shfl_sync(0xffffffffu, av, (j - 1) / RL);
    const double r = hypot(aj, hsub);
    double c = 1.0, s = 0.0;
    if (r != 0.0) {
        c = aj / r;
        s = hsub / r;
    }
    const double gj = g[j];
    __syncwarp();
    if (lane == 0) {
        cs[j] = c;
        sn[j] = s;
        R[rb + j] = r;
        g[j + 1] = -s * gj;
        g[j] = c * gj;
    }
    __syncwarp();
    return fabs(s * gj);
}

static __device__ double w_sumsq(const double *h, int len)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < len; i += 32) s = fma(h[i], h[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Complete Hessenberg column j (pending entries hcol[0..j]) with subdiagonal gamma: numeric
// check, Givens, breakdown test, in-cycle stop test.  Returns 1 to stop.
template <int RL>
static __device__ int w_complete_column(int j, double gamma, double *sm, const SmemLayout &L, double *R, Shared &sh,
                                 double tol)
{
    const int lane = threadIdx.x & 31;
    if (!isfinite(gamma)) {
        if (lane == 0) sh.cst = IGS_ENUMERIC;
        return 1;
    }
    const double hn2 = w_sumsq(sm + L.hcol, j + 1);
    const double res = w_givens<RL>(j, sm + L.hcol, gamma, sm + L.cs, sm + L.sn, sm + L.g, R);
    int stop = 0;
    if (gamma == 0.0 || gamma <= kBreakdownFactor * sqrt(hn2)) {
        if (lane == 0) sh.cst = IGS_BREAKDOWN;
        stop = 1;
    } else if ((sh.stop_den > 0.0 && res <= tol * sh.stop_den) || res <= sh.stop_floor) {
        stop = 1;
    }
    if (lane == 0) sh.done = j + 1;
    return stop;
}

// ---- one cycle and the whole solve ------------------------------------------------------
// One Arnoldi cycle on the residual: T = double, r in V[:, 0]; T = float, r in a.r64.
template <typename T, int RL>
__device__ void d_cycle(const SysArgs<T> &a, const Gang &gg, double *sm, const SmemLayout &L, Shared &sh)
{
    const int m = a.m, gs = a.gs, ldv = a.ldv;
    const bool sw = (int)(threadIdx.x >> 5) == sh.swarp;
    const int lane = threadIdx.x & 31;
    T *V = a.V;
    T *zu = reinterpret_cast<T *>(sm + L.zu);
    double *part = sm + L.part, *red = sm + L.red;
    const bool f32 = sizeof(T) == 4;
    if (threadIdx.x == 0) {
        sh.cst = IGS_OK;
        sh.done = 0;
        sh.stop = 0;
        sm[L.g] = sh.rho;
    }
    // Step 1: v_1 = r_0 / rho.
    {
        const double ir = 1.0 / sh.rho;
        const int hi = gg.hi;
        for (int i = gg.lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double r = f32 ? (i < a.n ? a.r64[i] : 0.0) : (double)V[i];
            V[i] = (T)(r * ir);
        }
    }
    if (!gang_barrier(gg, sh)) return;
    // Step 2: w_2 = A v_1, H_11 = v_1^T w_2, w_2 = w_2 - H_11 v_1.
    if (f32) d_spmv<T, float, T, T, false>(a, gg, a.sell_val32, V, nullptr, V + ldv);
    else d_spmv<T, double, T, T, false>(a, gg, a.sell_val, V, nullptr, V + ldv);
    __syncthreads();
    if (!d_dots<T, 1, false>(gg, sh, ldv, V, 1, V + ldv, nullptr, part, red)) return;
    if (threadIdx.x == 0) {
        sm[L.hcol] = red[0];
        sm[L.r1] = red[0];
    }
    __syncthreads();
    d_update<T, false, false>(gg, ldv, V, 1, sm + L.r1, 1.0, V + ldv, V + ldv, -1, 0.0);
    if (!gang_barrier(gg, sh)) return;

    for (int k = 3; k <= m + 1; ++k) {
        const int p = k - 1;
        T *w = V + (int64_t)(p - 1) * ldv;
        // Step 4: z = A w_{k-1} (this CTA's rows, into shared memory).
        if (f32) d_spmv<T, float, T, T, true>(a, gg, a.sell_val32, w, nullptr, zu);
        else d_spmv<T, double, T, T, true>(a, gg, a.sell_val, w, nullptr, zu);
        __syncthreads();
        // Step 5: [V_{k-2}, w]^T [w, z] and ||w||^2 in one pass over V.
        if (!d_dots<T, 2, false>(gg, sh, ldv, V, p, w, zu, part, red)) return;
        if (sw) {
            // Step 6: gamma = ||w||, the subdiagonal of column p-2, now complete.
            const double gamma = sqrt(red[2 * (p - 1)]);
            const int stop = w_complete_column<RL>(p - 2, gamma, sm, L, gg.R, sh, a.tol);
            if (!stop) {
                const double inv = 1.0 / gamma;
                // Steps 8-9: r^(0) / gamma, its last entry once more; step 10: L row / gamma.
                for (int c = lane; c < p; c += 32) {
                    double v = red[2 * c + 1] * inv;
                    if (c == p - 1) v *= inv;
                    sm[L.r0 + c] = v;
                }
                for (int c = lane; c < p - 1; c += 32) sm[L.L + lower_base(c, m) + (p - 1)] = red[2 * c] * inv;
                __syncwarp();
                // Step 12: r^(1) = (I + L)^{-1} r^(0).
                w_lower_solve<RL>(p, sm + L.L, m, sm + L.r0, sm + L.r1);
                if (gs == 1) {
                    __syncwarp();
                    for (int c = lane; c < p; c += 32) sm[L.hcol + c] = sm[L.r1 + c];
                }
                if (lane == 0) sh.inv = inv;
            }
            if (lane == 0) sh.stop = stop;
        }
        __syncthreads();
        if (sh.stop) break;
        const double inv = sh.inv;
        T *wk = V + (int64_t)p * ldv;
        if (gs == 2) {
            // Steps 7, 11, 13: v_{k-1} = w / gamma in place; u = z / gamma - V_{k-1} r^(1).
            d_update<T, true, true>(gg, ldv, V, p, sm + L.r1, inv, zu, zu, p - 1, inv);
            __syncthreads();
            // Step 14: r^(2) = V_{k-1}^T u.
            if (!d_dots<T, 1, true>(gg, sh, ldv, V, p, zu, nullptr, part, red)) return;
            if (sw) {
                // Step 15: r^(3) = (I + L)^{-1} r^(2); step 17: H column = r^(1) + r^(3).
                w_lower_solve<RL>(p, sm + L.L, m, red, sm + L.r3);
                __syncwarp();
                for (int c = lane; c < p; c += 32) sm[L.hcol + c] = sm[L.r1 + c] + sm[L.r3 + c];
            }
            __syncthreads();
            // Step 16: w_k = u - V_{k-1} r^(3).
            d_update<T, true, false>(gg, ldv, V, p, sm + L.r3, 1.0, zu, wk, -1, 0.0);
        } else {
            d_update<T, true, false>(gg, ldv, V, p, sm + L.r1, inv, zu, wk, p - 1, inv);
        }
        if (!gang_barrier(gg, sh)) return;
    }
    // Flush: gamma_{m+1} = ||w_{m+1}|| completes column m-1.
    if (!sh.stop && sh.cst == IGS_OK && sh.done == m - 1) {
        if (!d_sumsq<T, T>(gg, sh, a.n, V + (int64_t)m * ldv, (const T *)nullptr, 1, part, red)) return;
        if (sw) w_complete_column<RL>(m - 1, sqrt(red[0]), sm, L, gg.R, sh, a.tol);
        __syncthreads();
    }
}

// Restarted IGS-GMRES(m) on one system (the single-system solver's control flow).  Writes
// x (the gang's rows) and, from rank 0, beta / status / steps / cycles.
template <typename T>
__device__ void d_solve(const SysArgs<T> &a, const Gang &gg, double *sm, const SmemLayout &L, Shared &sh)
{
    double *part = sm + L.part, *red = sm + L.red;
    const bool f32 = sizeof(T) == 4;
    const int hi_n = gg.hi < a.n ? gg.hi : a.n;
    // the residual lives in V[:, 0] (FP64 basis) or in r64 (FP32 basis)
    double *rv = f32 ? a.r64 : reinterpret_cast<double *>(a.V);
    for (int i = gg.lo + threadIdx.x; i < hi_n; i += blockDim.x) a.x[i] = a.x0 ? a.x0[i] : 0.0;
    if (threadIdx.x == 0) {
        sh.cycles = 0;
        sh.steps = 0;
        sh.status = IGS_NOT_CONVERGED;
        sh.beta = nan("");
    }
    bool ok = d_sumsq<double, double>(gg, sh, a.n, a.b, (const double *)nullptr, 1, part, red);
    if (threadIdx.x == 0) sh.nb = sqrt(red[0]);
    __syncthreads();
    // the first residual reads other CTAs' x rows
    if (ok) ok = gang_barrier(gg, sh);
    while (ok) {
        // r = b - A x (FP64); beta(x) per eq. "nrbe" (zero residual: beta = 0).
        d_spmv<T, double, double, double, false>(a, gg, a.sell_val, a.x, a.b, rv);
        __syncthreads();
        if (!d_sumsq<double, double>(gg, sh, a.n, rv, a.x, 2, part, red)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0) {
            const double rn = sqrt(red[0]), xn = sqrt(red[1]);
            const double beta = rn == 0.0 ? 0.0 : rn / (sh.nb + a.normA * xn);
            sh.beta = beta;
            int brk = 0;
            if (!isfinite(beta)) {
                sh.status = IGS_ENUMERIC;
                brk = 1;
            } else if (beta <= a.tol || rn == 0.0) {
                sh.status = IGS_OK;
                brk = 1;
            } else if (sh.cycles >= a.max_cycles) {
                sh.status = IGS_NOT_CONVERGED;
                brk = 1;
            }
            sh.rho = rn;
            sh.stop_den = sh.nb + a.normA * xn;
            sh.stop_floor = a.inner_tol * rn;
            sh.stop = brk;
        }
        __syncthreads();
        if (sh.stop) break;
        if (a.m <= 64) d_cycle<T, 2>(a, gg, sm, L, sh);
        else d_cycle<T, 4>(a, gg, sm, L, sh);
        if (!sh.ok) {
            ok = false;
            break;
        }
        const int done = sh.done, cst = sh.cst;
        __syncthreads();
        if (threadIdx.x == 0) {
            sh.steps += done;
            sh.cycles += 1;
        }
        if (cst == IGS_ENUMERIC) {
            if (threadIdx.x == 0) sh.status = IGS_ENUMERIC;
            __syncthreads();
            break;
        }
        // x_m = x_0 + V_m y_m (y by back substitution on this CTA's copy of the Givens factor).
        if (done > 0) {
            if ((int)(threadIdx.x >> 5) == sh.swarp) {
                if (a.m <= 64) w_upper_solve<2>(done, gg.R, sm + L.g, sm + L.y);
                else w_upper_solve<4>(done, gg.R, sm + L.g, sm + L.y);
            }
            __syncthreads();
            d_xupdate<T>(gg, a.n, a.ldv, a.V, done, sm + L.y, a.x);
        }
        // the next residual reads other CTAs' x rows
        if (!gang_barrier(gg, sh)) {
            ok = false;
            break;
        }
        if (cst == IGS_BREAKDOWN) {
            d_spmv<T, double, double, double, false>(a, gg, a.sell_val, a.x, a.b, rv);
            __syncthreads();
            if (!d_sumsq<double, double>(gg, sh, a.n, rv, a.x, 2, part, red)) {
                ok = false;
                break;
            }
            if (threadIdx.x == 0) {
                const double rn = sqrt(red[0]), xn = sqrt(red[1]);
                const double beta = rn == 0.0 ? 0.0 : rn / (sh.nb + a.normA * xn);
                sh.beta = beta;
                sh.status = (isfinite(beta) && beta <= a.tol) ? IGS_OK : IGS_BREAKDOWN;
            }
            __syncthreads();
            break;
        }
    }
    if (threadIdx.x == 0 && gg.g == 0) {
        const int status = ok ? sh.status : IGS_ETIMEOUT;
        if (a.beta_out) *a.beta_out = sh.beta;
        if (a.status_out) *a.status_out = status;
        if (a.steps_out) *a.steps_out = sh.steps;
        if (a.cycles_out) *a.cycles_out = sh.cycles;
    }
    __syncthreads();
}

// Initialise the block-uniform state of a CTA (thread 0; a barrier must follow).
__device__ inline void init_shared(Shared &sh)
{
    unsigned wid;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid));
    // single-warp steps on warp (hardware warp slot / 4) mod warps: co-resident CTAs put them
    // on different SM sub-partitions; any choice gives the same results
    sh.swarp = (int)((wid >> 2) % (blockDim.x >> 5));
    sh.ok = 1;
    sh.gen = 0;
    sh.xbuf = 0;
}

}  // namespace sysdev
}  // namespace igs
