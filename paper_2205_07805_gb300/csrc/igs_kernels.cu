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

// out[v] = sum_{rb < nrb} part[v * nrb + rb] for v < nv (fixed order; block-wide).
// Threads per value grow with fewer values so that long partial lists are split.
__device__ void reduce_partials(const double *__restrict__ part, int nv, int nrb, double *out)
{
    const int T = blockDim.x, t = threadIdx.x;
    int tpv = 1;
    while (tpv < 32 && tpv * 2 * nv <= T) tpv *= 2;
    const int vpr = T / tpv;
    for (int v0 = 0; v0 < nv; v0 += vpr) {
        const int v = v0 + t / tpv, sub = t % tpv;
        double a0 = 0.0, a1 = 0.0;
        if (v < nv) {
            const double *pv = part + (int64_t)v * nrb;
            int rb = sub;
            for (; rb + tpv < nrb; rb += 2 * tpv) {
                a0 += pv[rb];
                a1 += pv[rb + tpv];
            }
            if (rb < nrb) a0 += pv[rb];
        }
        double s = a0 + a1;
        for (int o = tpv >> 1; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, tpv);
        if (sub == 0 && v < nv) out[v] = s;
    }
    __syncthreads();
}

// x = (I + L_p)^{-1} rhs for the unit lower-triangular I + L (Alg. 4.1 steps 12 and 15).
// L is row-major (leading dimension ldl), rows 0..p-1.  rhs and x live in shared memory
// (x must not alias rhs; `tmp` is scratch of p entries).  Block-wide.
//
// When ||L||_F is small the solve is evaluated as the truncated Neumann series
// sum_{i<t} (-L)^i rhs (Horner form), whose truncation error ||L||^t ||rhs|| / (1-||L||) is
// kept below 2^-60 ||rhs|| -- far under the FP64 rounding of the substitution itself.  Each
// term is one lane-parallel matrix-vector product, instead of p dependent steps.  With
// two Gauss-Seidel iterations ||L||_F is O(eps) and t = 2.  Otherwise the classical
// column-oriented forward substitution runs.  Returns the number of terms (0 =
// substitution).
__device__ int unit_lower_solve(const double *__restrict__ L, int ldl, int p,
                                const double *rhs, double *x, double *tmp, double lfro2)
{
    const int T = blockDim.x, t = threadIdx.x;
    int terms = 0;
    if (lfro2 <= 0.0) {
        terms = 1;
    } else if (lfro2 < 0x1p-30) {  // ||L||_F < 2^-15
        // need ||L||^terms <= 2^-60:  terms >= 120 / (-log2 lfro2)
        const double bits = -log2(lfro2);  // > 30
        terms = (int)ceil(120.0 / bits);
        if (terms < 2) terms = 2;
    }
    if (terms >= 1 && terms <= 4) {
        for (int i = t; i < p; i += T) x[i] = rhs[i];
        __syncthreads();
        for (int it = 1; it < terms; ++it) {
            // tmp = rhs - L x, rows paired (i, p-1-i) to balance the triangle over threads
            for (int i = t; i < (p + 1) / 2; i += T) {
                for (int h = 0; h < 2; ++h) {
                    const int row = h == 0 ? i : p - 1 - i;
                    if (h == 1 && row == i) break;
                    const double *Lr = L + (int64_t)row * ldl;
                    double a0 = 0.0, a1 = 0.0;
                    int c = 0;
                    for (; c + 1 < row; c += 2) {
                        a0 = fma(Lr[c], x[c], a0);
                        a1 = fma(Lr[c + 1], x[c + 1], a1);
                    }
                    if (c < row) a0 = fma(Lr[c], x[c], a0);
                    tmp[row] = rhs[row] - (a0 + a1);
                }
            }
            __syncthreads();
            for (int i = t; i < p; i += T) x[i] = tmp[i];
            __syncthreads();
        }
        return terms;
    }
    // Forward substitution, column oriented: after x[c] is final, every later row subtracts
    // L[i][c] x[c].  Rows are owned by threads (i = t + T*q, q < 4 covers p <= 4T).
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
            if (i > c && i < p) xi[q] = fma(-L[(int64_t)i * ldl + c], xc, xi[q]);
        }
    }
    __syncthreads();
    return 0;
}

}  // namespace

// =====================================================================================
// SpMV (Alg. 4.1 step 4; also r = b - A x for steps 1 and the end-of-cycle residual).
// =====================================================================================
// Thread per row: short rows (stencil matrices).  Two accumulation chains per row.
__global__ void __launch_bounds__(kStreamThreads)
k_spmv_rows(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ colind,
            const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
            const double *__restrict__ b, const DevState *st, int check_halt)
{
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
        y[i] = b ? b[i] - s : s;
    }
}

// Warp per row: long rows (dense or wide-band matrices).
__global__ void __launch_bounds__(kStreamThreads)
k_spmv_warp(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ colind,
            const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
            const double *__restrict__ b, const DevState *st, int check_halt)
{
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
        if (lane == 0) y[i] = b ? b[i] - s : s;
    }
}

// =====================================================================================
// Block multi-dot (Alg. 4.1 step 5, the one global reduction per iteration; step 14).
// part[(q*p + c)*gridDim.x + rb] = sum over rows of row block rb of V[:,c] * X_q.
// Grid: x = row blocks, y = column groups (p columns split evenly).  Thread t of a block
// owns column c_lo + t % cw and streams its own contiguous row slice t / cw: no lane ever
// spends an FP64 add on combining other lanes' products until the slice tree at the end.
// With NQ = 2 each V element feeds two FMAs ([V, w]^T [w, z]); with NQ = 1 two chains over
// alternate rows keep two independent FMAs in flight.
// =====================================================================================
template <int NQ>
__global__ void __launch_bounds__(kStreamThreads, kBlocksPerSM)
k_dots(const double *__restrict__ V, int64_t ld, int p, int64_t n4, int64_t rows,
       const double *__restrict__ x0, const double *__restrict__ x1, double *__restrict__ part,
       const DevState *st, int check_halt)
{
    if (check_halt && halted(st)) return;
    __shared__ double red[NQ][kStreamThreads];
    const int rb = blockIdx.x, G = gridDim.y, cg = blockIdx.y;
    const int c_lo = (int)((int64_t)cg * p / G), c_hi = (int)((int64_t)(cg + 1) * p / G);
    const int cw = c_hi - c_lo;
    const int S = blockDim.x / cw;
    const int t = threadIdx.x, cl = t % cw, s = t / cw;
    const int64_t r_lo = (int64_t)rb * rows;
    const int64_t r_hi = r_lo + rows < n4 ? r_lo + rows : n4;
    double a0 = 0.0, a1 = 0.0;
    if (s < S && r_lo < r_hi) {
        // slice boundaries on multiples of 4 rows (n4 and rows are multiples of 4)
        const int64_t nquad = (r_hi - r_lo) >> 2;
        const int64_t i0 = r_lo + 4 * (nquad * s / S), i1 = r_lo + 4 * (nquad * (s + 1) / S);
        const double *__restrict__ vc = V + (int64_t)(c_lo + cl) * ld;
        for (int64_t i = i0; i < i1; i += 4) {
            const double2 va = *reinterpret_cast<const double2 *>(vc + i);
            const double2 vb = *reinterpret_cast<const double2 *>(vc + i + 2);
            const double2 xa = *reinterpret_cast<const double2 *>(x0 + i);
            const double2 xb = *reinterpret_cast<const double2 *>(x0 + i + 2);
            if (NQ == 2) {
                const double2 ya = *reinterpret_cast<const double2 *>(x1 + i);
                const double2 yb = *reinterpret_cast<const double2 *>(x1 + i + 2);
                a0 = fma(va.x, xa.x, a0); a1 = fma(va.x, ya.x, a1);
                a0 = fma(va.y, xa.y, a0); a1 = fma(va.y, ya.y, a1);
                a0 = fma(vb.x, xb.x, a0); a1 = fma(vb.x, yb.x, a1);
                a0 = fma(vb.y, xb.y, a0); a1 = fma(vb.y, yb.y, a1);
            } else {
                a0 = fma(va.x, xa.x, a0); a1 = fma(va.y, xa.y, a1);
                a0 = fma(vb.x, xb.x, a0); a1 = fma(vb.y, xb.y, a1);
            }
        }
    }
    if (NQ == 1) {
        red[0][t] = a0 + a1;
    } else {
        red[0][t] = a0;
        red[NQ - 1][t] = a1;
    }
    // fixed-order tree over the S slices of each column
    int Sp = S;
    while (Sp > 1) {
        const int h = (Sp + 1) >> 1;
        __syncthreads();
        if (s < Sp - h) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) red[q][t] += red[q][t + h * cw];
        }
        Sp = h;
    }
    __syncthreads();
    if (s == 0) {
        const int nrb = gridDim.x;
#pragma unroll
        for (int q = 0; q < NQ; ++q) part[((int64_t)q * p + c_lo + cl) * nrb + rb] = red[q][t];
    }
}

// =====================================================================================
// Basis update (Alg. 4.1 steps 7, 11, 13 and 16; x_m = x_0 + V_m y_m at cycle end):
//   out[i] = a * src[i] - sum_{c<p} V[i,c] coef[c]
// Thread per row, coalesced over rows for each column.  With norm_last, column p-1 (the
// lagged w_{k-1}) is first normalised in place, v = w * inv_gamma (step 7), and
// a = inv_gamma (step 11).
// =====================================================================================
__global__ void __launch_bounds__(kStreamThreads)
k_update(double *V, int64_t ld, int p, int64_t n, const double *__restrict__ coef, int neg_coef,
         double alpha, const double *src, double *out, int norm_last, int p_from_state,
         DevState *st, int check_halt)
{
    if (check_halt && halted(st)) return;
    extern __shared__ double sc[];
    if (p_from_state) p = st->ncols;
    const double a = norm_last ? st->inv_gamma : alpha;
    for (int c = threadIdx.x; c < p; c += blockDim.x) sc[c] = neg_coef ? -coef[c] : coef[c];
    __syncthreads();
    const int pc = norm_last ? p - 1 : p;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double *vi = V + i;
        double acc0 = 0.0, acc1 = 0.0;
        int c = 0;
        for (; c + 3 < pc; c += 4) {
            const double v0 = vi[(int64_t)c * ld], v1 = vi[(int64_t)(c + 1) * ld];
            const double v2 = vi[(int64_t)(c + 2) * ld], v3 = vi[(int64_t)(c + 3) * ld];
            acc0 = fma(v0, sc[c], acc0);
            acc1 = fma(v1, sc[c + 1], acc1);
            acc0 = fma(v2, sc[c + 2], acc0);
            acc1 = fma(v3, sc[c + 3], acc1);
        }
        for (; c < pc; ++c) acc0 = fma(vi[(int64_t)c * ld], sc[c], acc0);
        if (norm_last) {
            double *vl = V + (int64_t)(p - 1) * ld + i;
            const double v = *vl * a;
            *vl = v;
            acc1 = fma(v, sc[p - 1], acc1);
        }
        out[i] = fma(a, src[i], -(acc0 + acc1));
    }
}

// Partial sums of squares of up to three vectors: part[q * gridDim.x + blockIdx.x].
__global__ void __launch_bounds__(kStreamThreads)
k_norms(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
        const double *__restrict__ c, double *__restrict__ part)
{
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
        if (threadIdx.x == 0) part[q * gridDim.x + blockIdx.x] = tot;
    }
}

// dst = src * scale, scale = st->inv_rho (which = 0) or st->inv_gamma (which = 1).
__global__ void __launch_bounds__(kStreamThreads)
k_scale(int64_t n, const double *src, double *dst, int which, const DevState *st, int check_halt)
{
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
    double *H, *L, *R, *cs, *sn, *g, *lfro2, *r0v, *r1v, *r2v, *r3v, *y, *hist_res, *hist_lfro;
    const double *part;
    DevState *st;
    int ldh, ldl;
};

static SmallArgs small_args(const Workspace &w)
{
    SmallArgs a;
    a.H = w.H; a.L = w.L; a.R = w.R; a.cs = w.cs; a.sn = w.sn; a.g = w.g; a.lfro2 = w.lfro2;
    a.r0v = w.r0v; a.r1v = w.r1v; a.r2v = w.r2v; a.r3v = w.r3v; a.y = w.y;
    a.hist_res = w.hist_res; a.hist_lfro = w.hist_lfro; a.part = w.part; a.st = w.st;
    a.ldh = w.ldh(); a.ldl = w.ldl();
    return a;
}

// Solve-level initialisation of the device state.
__global__ void k_init_state(DevState *st, double tol, double normA)
{
    if (threadIdx.x == 0) {
        DevState s = {};
        s.tol = tol;
        s.normA = normA;
        *st = s;
    }
}

// ||b|| from its partial sums of squares.
__global__ void __launch_bounds__(kSmallThreads) k_bnorm(const double *part, int nblk, DevState *st)
{
    __shared__ double out[1];
    reduce_partials(part, 1, nblk, out);
    if (threadIdx.x == 0) st->bnorm = sqrt(out[0]);
}

// End of a cycle (and start of a solve): r = b - A x is in place; from the partial sums of
// squares of r and x compute ||r||, ||x|| and beta(x) = ||r|| / (||b|| + ||A||_2 ||x||)
// (eq. "nrbe").
__global__ void __launch_bounds__(kSmallThreads) k_beta(const double *part, int nblk, DevState *st)
{
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
    DevState *st = a.st;
    for (int i = threadIdx.x; i <= mmax; i += blockDim.x) a.g[i] = 0.0;
    if (threadIdx.x == 0) {
        const double rho = st->rnorm;
        st->rho = rho;
        st->inv_rho = 1.0 / rho;
        a.g[0] = rho;
        a.lfro2[0] = 0.0;
        st->stop_den = st->bnorm + st->normA * st->xnorm;
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
    DevState *st = a.st;
    if (halted(st)) return;
    if (st->stop_reason != 0) {  // the previous column met the stop test
        if (threadIdx.x == 0) st->halt = 1;
        return;
    }
    __shared__ double buf[2 * (kMaxRestart + 1)];
    __shared__ double r0s[kMaxRestart + 1], r1s[kMaxRestart + 1], tmp[kMaxRestart + 1];
    __shared__ double sh[kSmallThreads];
    __shared__ double s_inv_gamma;
    __shared__ int s_stop;
    const int p = k - 1, t = threadIdx.x;
    reduce_partials(a.part, 2 * p, nrb, buf);
    // breakdown test needs ||H(0:p-2, p-2)||^2
    double hv = 0.0;
    for (int i = t; i <= p - 2; i += blockDim.x) {
        const double h = a.H[(int64_t)(p - 2) * a.ldh + i];
        hv = fma(h, h, hv);
    }
    const double hn2 = block_sum(hv, sh);
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
    if (s_stop != 0) return;
    const double ig = s_inv_gamma;
    // steps 8-10
    double rowsq = 0.0;
    for (int c = t; c < p; c += blockDim.x) {
        double r = buf[p + c] * ig;
        if (c == p - 1) r *= ig;
        r0s[c] = r;
        if (c < p - 1) {
            const double l = buf[c] * ig;
            a.L[(int64_t)(p - 1) * a.ldl + c] = l;
            rowsq = fma(l, l, rowsq);
        }
    }
    const double rs = block_sum(rowsq, sh);  // also a barrier for r0s
    const double lf2 = a.lfro2[p - 2] + rs;
    if (t == 0) a.lfro2[p - 1] = lf2;
    // step 12
    const int terms = unit_lower_solve(a.L, a.ldl, p, r0s, r1s, tmp, lf2);
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
    DevState *st = a.st;
    if (halted(st)) return;
    __shared__ double r2s[kMaxRestart + 1], r3s[kMaxRestart + 1], tmp[kMaxRestart + 1];
    const int p = k - 1, t = threadIdx.x;
    reduce_partials(a.part, p, nrb, r2s);
    unit_lower_solve(a.L, a.ldl, p, r2s, r3s, tmp, a.lfro2[p - 1]);
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
    const int t = threadIdx.x;
    reduce_partials(a.part, m + 1, nrb, buf);
    double hv = 0.0;
    for (int i = t; i <= m - 1; i += blockDim.x) {
        const double h = a.H[(int64_t)(m - 1) * a.ldh + i];
        hv = fma(h, h, hv);
    }
    const double hn2 = block_sum(hv, sh);
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
        a.L[(int64_t)m * a.ldl + c] = l;
        rowsq = fma(l, l, rowsq);
    }
    const double rs = block_sum(rowsq, sh);
    if (t == 0) a.lfro2[m] = a.lfro2[m - 1] + rs;
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
        if (st->stop_reason == 0 && st->stop_den > 0.0 && res <= st->tol * st->stop_den) {
            st->stop_reason = 1;
            st->stop_cols = j + 1;
        }
    }
}

// y = R^{-1} g for the p = (stop_cols or m) columns of the cycle (back substitution,
// column oriented over the block), st->ncols = p.
__global__ void __launch_bounds__(kSmallThreads) k_lsq(SmallArgs a, int m)
{
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

DotsPlan plan_dots(const Workspace &w, int p)
{
    DotsPlan pl;
    const int slots = stream_grid(w);
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
    rows = (rows + 3) & ~int64_t(3);
    rblocks = (int)((n4 + rows - 1) / rows);
    pl.groups = groups;
    pl.rblocks = rblocks;
    pl.rows = rows;
    return pl;
}

cudaError_t launch_spmv(const Workspace &w, const double *x, double *y, const double *b,
                        bool check_halt, cudaStream_t s)
{
    const int grid = stream_grid(w);
    if (w.spmv_warp_rows)
        k_spmv_warp<<<grid, kStreamThreads, 0, s>>>(w.n, w.rowptr, w.colind, w.val, x, y, b, w.st,
                                                    check_halt);
    else
        k_spmv_rows<<<grid, kStreamThreads, 0, s>>>(w.n, w.rowptr, w.colind, w.val, x, y, b, w.st,
                                                    check_halt);
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
        k_dots<2><<<grid, kStreamThreads, 0, s>>>(w.V, w.ld, p, n4, pl.rows, x0, x1, w.part, w.st,
                                                  check_halt);
    else
        k_dots<1><<<grid, kStreamThreads, 0, s>>>(w.V, w.ld, p, n4, pl.rows, x0, nullptr, w.part,
                                                  w.st, check_halt);
    return cudaGetLastError();
}

cudaError_t launch_update(const Workspace &w, int p, const double *coef, bool neg_coef,
                          double alpha, const double *src, double *out, bool norm_last,
                          bool p_from_state, bool check_halt, cudaStream_t s)
{
    const int pmax = p_from_state ? w.mmax + 1 : p;
    const size_t smem = sizeof(double) * (size_t)(pmax > 0 ? pmax : 1);
    k_update<<<stream_grid(w), kStreamThreads, smem, s>>>(w.V, w.ld, p, w.n, coef, neg_coef ? 1 : 0,
                                                          alpha, src, out, norm_last ? 1 : 0,
                                                          p_from_state ? 1 : 0, w.st,
                                                          check_halt ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_norms(const Workspace &w, const double *a, const double *b, const double *c,
                         int *blocks_out, cudaStream_t s)
{
    const int grid = w.num_sms;
    k_norms<<<grid, kStreamThreads, 0, s>>>(w.n, a, b, c, w.part);
    if (blocks_out) *blocks_out = grid;
    return cudaGetLastError();
}

cudaError_t launch_scale(const Workspace &w, const double *src, double *dst, int which,
                         bool check_halt, cudaStream_t s)
{
    k_scale<<<stream_grid(w), kStreamThreads, 0, s>>>(w.n, src, dst, which, w.st, check_halt ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const Workspace &w, double tol, double normA, cudaStream_t s)
{
    k_init_state<<<1, 32, 0, s>>>(w.st, tol, normA);
    return cudaGetLastError();
}

cudaError_t launch_bnorm(const Workspace &w, int nblk, cudaStream_t s)
{
    k_bnorm<<<1, kSmallThreads, 0, s>>>(w.part, nblk, w.st);
    return cudaGetLastError();
}

cudaError_t launch_beta(const Workspace &w, int nblk, cudaStream_t s)
{
    k_beta<<<1, kSmallThreads, 0, s>>>(w.part, nblk, w.st);
    return cudaGetLastError();
}

cudaError_t launch_cycle_start(const Workspace &w, int, cudaStream_t s)
{
    k_cycle_start<<<1, kSmallThreads, 0, s>>>(small_args(w), w.mmax);
    return cudaGetLastError();
}

cudaError_t launch_prime(const Workspace &w, const DotsPlan &pl, cudaStream_t s)
{
    k_prime<<<1, kSmallThreads, 0, s>>>(small_args(w), pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_step_a(const Workspace &w, int k, int gs, const DotsPlan &pl, cudaStream_t s)
{
    k_step_a<<<1, kSmallThreads, 0, s>>>(small_args(w), k, gs, pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_step_b(const Workspace &w, int k, const DotsPlan &pl, cudaStream_t s)
{
    k_step_b<<<1, kSmallThreads, 0, s>>>(small_args(w), k, pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_flush(const Workspace &w, int m, const DotsPlan &pl, cudaStream_t s)
{
    k_flush<<<1, kSmallThreads, 0, s>>>(small_args(w), m, pl.rblocks);
    return cudaGetLastError();
}

cudaError_t launch_givens(const Workspace &w, int j, cudaStream_t s)
{
    k_givens<<<1, kGivensThreads, 0, s>>>(small_args(w), j);
    return cudaGetLastError();
}

cudaError_t launch_lsq(const Workspace &w, int m, cudaStream_t s)
{
    k_lsq<<<1, kSmallThreads, 0, s>>>(small_args(w), m);
    return cudaGetLastError();
}

cudaError_t estimate_norm2(const Workspace &w, const int *at_rowptr, const int *at_colind,
                           const double *at_val, int iters, double *out, cudaStream_t s)
{
    // x: w.t, A x: w.z, A^T (A x): w.u; lambda in w.y[0]
    const int grid = stream_grid(w);
    k_power_init<<<grid, kStreamThreads, 0, s>>>(w.n, w.t);
    for (int it = 0; it < iters; ++it) {
        if (w.spmv_warp_rows) {
            k_spmv_warp<<<grid, kStreamThreads, 0, s>>>(w.n, w.rowptr, w.colind, w.val, w.t, w.z,
                                                        nullptr, w.st, 0);
            k_spmv_warp<<<grid, kStreamThreads, 0, s>>>(w.n, at_rowptr, at_colind, at_val, w.z, w.u,
                                                        nullptr, w.st, 0);
        } else {
            k_spmv_rows<<<grid, kStreamThreads, 0, s>>>(w.n, w.rowptr, w.colind, w.val, w.t, w.z,
                                                        nullptr, w.st, 0);
            k_spmv_rows<<<grid, kStreamThreads, 0, s>>>(w.n, at_rowptr, at_colind, at_val, w.z, w.u,
                                                        nullptr, w.st, 0);
        }
        k_norms<<<w.num_sms, kStreamThreads, 0, s>>>(w.n, w.u, nullptr, nullptr, w.part);
        k_power_norm<<<1, kSmallThreads, 0, s>>>(w.part, w.num_sms, w.y);
        k_power_scale<<<grid, kStreamThreads, 0, s>>>(w.n, w.u, w.y);
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
