// Batched IGS-GMRES (include/igs_batch.h): many independent sparse systems solved by one
// persistent kernel launch.
//
// Each CTA takes systems from a device work queue (largest first) and runs the whole
// restarted IGS-GMRES(m) of Alg. 4.1 on one system at a time: cycle start r = b - A x and
// the backward error of eq. "nrbe", step 1 (v_1 = r / rho), step 2 (the single-projection
// prime), the k = 3..m+1 loop (steps 4-18: SpMV, the fused reduction of step 5, the lagged
// normalisation of steps 6-11, one or two Gauss-Seidel corrections with the unit lower
// triangular (I + L), the Hessenberg column of step 17), the Givens least squares beside
// it with the in-cycle stop test, the flush that sets H_{m+1,m}, and x_m = x_0 + V_m y_m.
// The control flow (stop, breakdown and restart rules) is the same as the single-system
// path's.  Every per-step scalar lives in shared memory, so a step costs no kernel launch
// and no host round trip.
//
// Determinism: the arithmetic of a system depends only on that system (its n, its CSR rows
// and the solve options), never on the CTA, the block size, the number of resident CTAs or
// the other systems of the batch:
//   - a dot product is summed over row slices whose number depends on n and the column count
//     only (pick_slices), each slice in row order with two interleaved chains, then over
//     the slices in order;
//   - every row of an update or SpMV is one thread's fixed-order chain;
//   - the triangular solves, the Givens scan and the back substitution run on warp 0 with
//     fixed lane roles.
// So a system's x, beta and step count are bitwise the same whether it is solved alone or
// in a batch, and under every launch configuration the tuner may pick.
//
// Memory: each CTA (slot) owns a basis V of (m+1) columns with leading dimension
// round_up(n, 4) and the Givens factor R (packed upper, column-major) in HBM (re-read from
// L2 when the working set fits); the Krylov vector z/u, the slice partial sums, L (packed
// strictly-lower, column-major) and the small vectors are in shared memory.
#include "../../include/igs.h"
#include "../../include/igs_batch.h"
#include "igs_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace igs {
namespace batch {

constexpr int kMaxM = IGS_BATCH_MAX_M;  // largest restart length (two rows per lane in warp solves)
constexpr int kMaxN = IGS_BATCH_MAX_N;  // largest system (the Krylov vector is kept in shared memory)
constexpr int kMaxSlices = 16;      // dot products are split into at most this many row slices
constexpr int kMaxSlotsPerSM = 8;   // largest resident CTAs per SM any configuration uses

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Row slices of the dot products.  A system of n2 (even) rows is cut into nsl slices of
// whole row pairs, slice s holding pairs [s*P/nsl, (s+1)*P/nsl) (P = n2/2).  For a product
// over pc columns, nsl is chosen in [slices_lo(n2), slices_hi(n2)] so that the nsl*pc
// (slice, column) items leave the fewest idle lanes in the last warp; the choice depends
// on n and pc only.
__host__ __device__ inline int slices_hi(int n2)
{
    const int s = (n2 >> 1) / 4;  // at least four row pairs per slice
    return s < 1 ? 1 : (s > kMaxSlices ? kMaxSlices : s);
}
__host__ __device__ inline int slices_lo(int n2) { return slices_hi(n2) < 8 ? slices_hi(n2) : 8; }

__host__ __device__ inline int pick_slices(int n2, int pc)
{
    int best = slices_lo(n2), best_idle = 0, best_tot = 1;
    for (int s = slices_lo(n2); s <= slices_hi(n2); ++s) {
        const int items = s * pc;
        const int tot = (items + 31) / 32 * 32;
        const int idle = tot - items;
        if (s == slices_lo(n2) || idle * best_tot < best_idle * tot) {
            best = s;
            best_idle = idle;
            best_tot = tot;
        }
    }
    return best;
}

// Shared-memory index of row i of the Krylov vector: two doubles of padding every 128 rows
// put the starts of different slices in different banks.
__host__ __device__ inline int pad_idx(int i) { return i + 2 * (i >> 7); }

// Packed strictly-lower L of order m+1, column-major: column c holds rows c+1..m.
__host__ __device__ inline int lower_base(int c, int m) { return c * m - c * (c - 1) / 2 - c - 1; }
// Packed upper R (order m), column-major: column j holds rows 0..j.
__host__ __device__ inline int upper_base(int j) { return j * (j + 1) / 2; }

// Offsets (in doubles) of the dynamic shared-memory arrays for a batch with largest system
// nmax and restart m.
struct SmemLayout {
    int zu, part, L, red, r0, r1, r3, hcol, cs, sn, g, y, total;
};

__host__ __device__ inline SmemLayout smem_layout(int nmax, int m)
{
    SmemLayout s;
    int o = 0;
    const int n2 = round_up(nmax, 2);
    s.zu = o;   o += round_up(pad_idx(n2) + 2, 2);
    s.part = o; o += round_up(kMaxSlices * (m + 1) * 2, 2);
    s.L = o;    o += round_up((m + 1) * m / 2 + 1, 2);
    s.red = o;  o += round_up(2 * (m + 1), 2);
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
    unsigned long long *summary;  // [0] total steps, [1+k] systems with status code k+4
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

// Block-uniform state of the system being solved.
struct Shared {
    double nb, normA, rho, inv, stop_den, beta, rn, xn;
    int status, cst, done, stop, cycles;
    int swarp;  // warp of this CTA that runs the single-warp steps
    long long steps;
};

struct Sys {
    int n, n2, ldv, slice0;
    int64_t row0;
};

__device__ __forceinline__ double2 ld2(const double *p) { return *reinterpret_cast<const double2 *>(p); }
__device__ __forceinline__ void st2(double *p, double2 v) { *reinterpret_cast<double2 *>(p) = v; }

// y = A x, or y = b - A x when b != null (rows >= n of y are set to 0).  x, b: system-local.
// Each row is summed in its CSR order; lanes of a warp read consecutive SELL entries.
template <bool OUT_PAD>
__device__ void b_spmv(const Args &a, const Sys &S, const double *x, const double *b, double *y)
{
    const int64_t *so = a.sell_off + S.slice0;
    for (int i = threadIdx.x; i < S.n2; i += blockDim.x) {
        double acc = 0.0;
        if (i < S.n) {
            const int k = i >> 5;
            int64_t e = so[k] + (i & 31);
            const int64_t e1 = so[k + 1];
            // eight entries per batch (all loads of a batch in flight together)
            for (; e < e1; e += 256) {
                int c[8];
                double v[8], xv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const bool in = e + 32 * u < e1;
                    c[u] = in ? a.sell_col[e + 32 * u] : -1;
                    v[u] = in ? a.sell_val[e + 32 * u] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) xv[u] = c[u] >= 0 ? x[c[u]] : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
            }
            if (b) acc = b[i] - acc;
        }
        y[OUT_PAD ? pad_idx(i) : i] = acc;
    }
}

// red[c*NQ + q] = V[:, c]^T X_q for c < pc (X_0 = x0, X_1 = x1; x1 is the padded shared
// vector).  Fixed slices, fixed order (see the file comment).
template <int NQ, bool X0PAD>
__device__ void b_dots(const Sys &S, const double *V, int pc, const double *x0, const double *x1,
                       double *part, double *red)
{
    const int nsl = pick_slices(S.n2, pc);
    const int npairs = S.n2 >> 1;
    const int nitems = pc * nsl;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
        const int c = it % pc, s = it / pc;
        const int i0 = 2 * (s * npairs / nsl);
        const int i1 = 2 * ((s + 1) * npairs / nsl);
        const double *vc = V + (int64_t)c * S.ldv;
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
        int i = i0;
        for (; i + 8 <= i1; i += 8) {
            double2 v[4], xa[4], xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = ld2(vc + i + 2 * u);
                xa[u] = ld2(x0 + (X0PAD ? pad_idx(i + 2 * u) : i + 2 * u));
                if (NQ == 2) xb[u] = ld2(x1 + pad_idx(i + 2 * u));
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
            const double2 v = ld2(vc + i);
            const double2 xa = ld2(x0 + (X0PAD ? pad_idx(i) : i));
            a0 = fma(v.x, xa.x, a0);
            a1 = fma(v.y, xa.y, a1);
            if (NQ == 2) {
                const double2 xb = ld2(x1 + pad_idx(i));
                b0 = fma(v.x, xb.x, b0);
                b1 = fma(v.y, xb.y, b1);
            }
        }
        part[(s * pc + c) * NQ] = a0 + a1;
        if (NQ == 2) part[(s * pc + c) * NQ + 1] = b0 + b1;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < pc * NQ; v += blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < nsl; ++s) acc += part[s * pc * NQ + v];
        red[v] = acc;
    }
    __syncthreads();
}

// red[q] = ||v_q||^2 for up to two system-local vectors (any alignment), fixed slices.
__device__ void b_sumsq(const Sys &S, const double *v0, const double *v1, int nv, double *part,
                        double *red)
{
    const int nsl = slices_hi(S.n2);
    const int nitems = nv * nsl;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
        const int q = it % nv, s = it / nv;
        const double *v = q == 0 ? v0 : v1;
        const int i0 = s * S.n / nsl;
        const int i1 = (s + 1) * S.n / nsl;
        double a0 = 0.0, a1 = 0.0;
        int i = i0;
        for (; i + 1 < i1; i += 2) {
            a0 = fma(v[i], v[i], a0);
            a1 = fma(v[i + 1], v[i + 1], a1);
        }
        if (i < i1) a0 = fma(v[i], v[i], a0);
        part[s * nv + q] = a0 + a1;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nv; q += blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < nsl; ++s) acc += part[s * nv + q];
        red[q] = acc;
    }
    __syncthreads();
}

// out[i] = alpha * src[i] - sum_{c < pc} V[i, c] coef[c] for rows i < n2 (pairs of rows per
// thread).  When nc >= 0 (then nc = pc - 1), column nc of V is first scaled in place by
// scale_nc (the lagged normalisation of step 7) and the scaled column enters the sum.
template <bool SRC_PAD, bool OUT_PAD>
__device__ void b_update(const Sys &S, double *V, int pc, const double *coef, double alpha,
                         const double *src, double *out, int nc, double scale_nc)
{
    const int npairs = S.n2 >> 1;
    // the normalised column (always the last, nc = pc - 1) is scaled and stored before the
    // other columns are streamed, so that no store sits between their loads; its term is
    // still added last
    const int ps = nc >= 0 ? nc : pc;
    for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
        const int i = 2 * pr;
        double2 vn = make_double2(0.0, 0.0);
        if (nc >= 0) {
            vn = ld2(V + (int64_t)nc * S.ldv + i);
            vn.x *= scale_nc;
            vn.y *= scale_nc;
            st2(V + (int64_t)nc * S.ldv + i, vn);
        }
        double sx = 0.0, sy = 0.0;
        int c = 0;
        for (; c + 4 <= ps; c += 4) {
            double2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ld2(V + (int64_t)(c + u) * S.ldv + i);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double cf = coef[c + u];
                sx = fma(v[u].x, cf, sx);
                sy = fma(v[u].y, cf, sy);
            }
        }
        for (; c < ps; ++c) {
            const double2 v = ld2(V + (int64_t)c * S.ldv + i);
            const double cf = coef[c];
            sx = fma(v.x, cf, sx);
            sy = fma(v.y, cf, sy);
        }
        if (nc >= 0) {
            const double cf = coef[nc];
            sx = fma(vn.x, cf, sx);
            sy = fma(vn.y, cf, sy);
        }
        const double2 sv = ld2(src + (SRC_PAD ? pad_idx(i) : i));
        double2 o;
        o.x = alpha * sv.x - sx;
        o.y = alpha * sv.y - sy;
        st2(out + (OUT_PAD ? pad_idx(i) : i), o);
    }
}

// x[i] = x[i] + sum_{c < p} V[i, c] y[c] for i < n (x system-local, any alignment).
__device__ void b_xupdate(const Sys &S, const double *V, int p, const double *y, double *x)
{
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < p; ++c) s = fma(V[(int64_t)c * S.ldv + i], y[c], s);
        x[i] = x[i] + s;
    }
}

// Warp 0: out = (I + L_p)^{-1} rhs by forward substitution (Alg. 4.1 steps 12 and 15),
// p <= 64, lane l owns rows l and l + 32.
__device__ void w_lower_solve(int p, const double *L, int m, const double *rhs, double *out)
{
    const int lane = threadIdx.x & 31;
    double x0 = lane < p ? rhs[lane] : 0.0;
    double x1 = lane + 32 < p ? rhs[lane + 32] : 0.0;
    for (int c = 0; c + 1 < p; ++c) {
        const double xc = __shfl_sync(0xffffffffu, c < 32 ? x0 : x1, c & 31);
        const int base = lower_base(c, m);
        if (c < 31 && lane > c && lane < p) x0 = fma(-L[base + lane], xc, x0);
        if (p > 32) {
            const int i = lane + 32;
            if (i > c && i < p) x1 = fma(-L[base + i], xc, x1);
        }
    }
    if (lane < p) out[lane] = x0;
    if (lane + 32 < p) out[lane + 32] = x1;
}

// Warp 0: y = R_p^{-1} g by back substitution (R packed upper), p <= 64.
__device__ void w_upper_solve(int p, const double *R, const double *g, double *y)
{
    const int lane = threadIdx.x & 31;
    double a0 = lane < p ? g[lane] : 0.0;
    double a1 = lane + 32 < p ? g[lane + 32] : 0.0;
    for (int c = p - 1; c >= 0; --c) {
        const int ol = c & 31;
        const int base = upper_base(c);
        double yc = 0.0;
        if (lane == ol) yc = (c >= 32 ? a1 : a0) / R[base + c];
        yc = __shfl_sync(0xffffffffu, yc, ol);
        if (lane == 0) y[c] = yc;
        if (lane < c) a0 = fma(-R[base + lane], yc, a0);
        if (lane + 32 < c) a1 = fma(-R[base + lane + 32], yc, a1);
    }
}

// Warp 0: bring Hessenberg column j (entries h[0..j], subdiagonal hsub) into the Givens QR
// (eq. "llse").  The j earlier rotations are applied as a warp scan of the affine maps
// a -> -s_i a + c_i h_{i+1} (lane l owns maps 2l and 2l+1), then the new rotation.  Writes
// R column j, cs[j], sn[j], g[j], g[j+1]; returns |g_{j+1}| on every lane.
__device__ double w_givens(int j, const double *h, double hsub, double *cs, double *sn, double *g,
                           double *R)
{
    const int lane = threadIdx.x & 31;
    const int m0 = 2 * lane;
    double cA = 1.0, cB = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
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
    for (int q = 0; q < 2; ++q) {
        const int i = m0 + q;
        if (i < j) {
            const double hi1 = h[i + 1];
            R[rb + i] = fma(cs[i], av, sn[i] * hi1);
            av = fma(-sn[i], av, cs[i] * hi1);
        }
    }
    const double aj = j == 0 ? h[0] : __shfl_sync(0xffffffffu, av, (j - 1) >> 1);
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

// Warp 0: sum of squares of h[0..len) (lane-strided, then a fixed shuffle tree).
__device__ double w_sumsq(const double *h, int len)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < len; i += 32) s = fma(h[i], h[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Warp 0: complete Hessenberg column j (pending entries hcol[0..j]) with subdiagonal
// gamma: numeric check, Givens, breakdown test, in-cycle stop test.  Returns 1 to stop.
__device__ int w_complete_column(int j, double gamma, double *sm, const SmemLayout &L, double *R,
                                 Shared &sh, double tol)
{
    const int lane = threadIdx.x & 31;
    int stop = 0;
    if (!isfinite(gamma)) {
        if (lane == 0) sh.cst = IGS_ENUMERIC;
        return 1;
    }
    const double hn2 = w_sumsq(sm + L.hcol, j + 1);
    const double res = w_givens(j, sm + L.hcol, gamma, sm + L.cs, sm + L.sn, sm + L.g, R);
    if (gamma == 0.0 || gamma <= kBreakdownFactor * sqrt(hn2)) {
        if (lane == 0) sh.cst = IGS_BREAKDOWN;
        stop = 1;
    } else if (sh.stop_den > 0.0 && res / sh.stop_den <= tol) {
        stop = 1;
    }
    if (lane == 0) sh.done = j + 1;
    return stop;
}

// One Arnoldi cycle of Alg. 4.1 on the residual held in V[:, 0] (norm sh.rho).  Sets
// sh.done (completed columns), sh.cst (IGS_OK, IGS_BREAKDOWN or IGS_ENUMERIC); the Givens
// factorisation of the completed columns is left in R, g.
__device__ void b_cycle(const Args &a, const Run &run, const Sys &S, double *V, double *sm,
                        const SmemLayout &L, Shared &sh)
{
    const int m = a.m, gs = run.gs;
    const bool w0 = (int)(threadIdx.x >> 5) == sh.swarp;  // the warp doing the scalar work
    double *R = V + a.r_offset;
    const int lane = threadIdx.x & 31;
    double *zu = sm + L.zu, *part = sm + L.part, *red = sm + L.red;
    if (threadIdx.x == 0) {
        sh.cst = IGS_OK;
        sh.done = 0;
        sh.stop = 0;
        sm[L.g] = sh.rho;
    }
    // Step 1: v_1 = r_0 / rho (in place).
    b_update<false, false>(S, V, 0, nullptr, 1.0 / sh.rho, V, V, -1, 0.0);
    __syncthreads();
    // Step 2: w_2 = A v_1, H_11 = v_1^T w_2, w_2 = w_2 - H_11 v_1.
    b_spmv<false>(a, S, V, nullptr, V + S.ldv);
    __syncthreads();
    b_dots<1, false>(S, V, 1, V + S.ldv, nullptr, part, red);
    if (threadIdx.x == 0) {
        sm[L.hcol] = red[0];
        sm[L.r1] = red[0];
    }
    __syncthreads();
    b_update<false, false>(S, V, 1, sm + L.r1, 1.0, V + S.ldv, V + S.ldv, -1, 0.0);
    __syncthreads();

    for (int k = 3; k <= m + 1; ++k) {
        const int p = k - 1;
        double *w = V + (int64_t)(p - 1) * S.ldv;
        // Step 4: z = A w_{k-1}.
        b_spmv<true>(a, S, w, nullptr, zu);
        __syncthreads();
        // Step 5: L row = V_{k-2}^T w, r^(0) = V_{k-1}^T z, ||w||^2, in one pass over V.
        b_dots<2, false>(S, V, p, w, zu, part, red);
        if (w0) {
            // Step 6: gamma = ||w||, the subdiagonal of column p-2, which is now complete.
            const double gamma = sqrt(red[2 * (p - 1)]);
            int stop = w_complete_column(p - 2, gamma, sm, L, R, sh, run.tol);
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
                w_lower_solve(p, sm + L.L, m, sm + L.r0, sm + L.r1);
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
        double *wk = V + (int64_t)p * S.ldv;
        if (gs == 2) {
            // Steps 7, 11, 13: v_{k-1} = w / gamma in place; u = z / gamma - V_{k-1} r^(1).
            b_update<true, true>(S, V, p, sm + L.r1, inv, zu, zu, p - 1, inv);
            __syncthreads();
            // Step 14: r^(2) = V_{k-1}^T u.
            b_dots<1, true>(S, V, p, zu, nullptr, part, red);
            if (w0) {
                // Step 15: r^(3) = (I + L)^{-1} r^(2); step 17: H column = r^(1) + r^(3).
                w_lower_solve(p, sm + L.L, m, red, sm + L.r3);
                __syncwarp();
                for (int c = lane; c < p; c += 32) sm[L.hcol + c] = sm[L.r1 + c] + sm[L.r3 + c];
            }
            __syncthreads();
            // Step 16: w_k = u - V_{k-1} r^(3).
            b_update<true, false>(S, V, p, sm + L.r3, 1.0, zu, wk, -1, 0.0);
        } else {
            // One Gauss-Seidel iteration: w_k = u.
            b_update<true, false>(S, V, p, sm + L.r1, inv, zu, wk, p - 1, inv);
        }
        __syncthreads();
    }
    // Flush: gamma_{m+1} = ||w_{m+1}|| completes column m-1.
    if (!sh.stop && sh.cst == IGS_OK && sh.done == m - 1) {
        b_sumsq(S, V + (int64_t)m * S.ldv, nullptr, 1, part, red);
        if (w0) w_complete_column(m - 1, sqrt(red[0]), sm, L, R, sh, run.tol);
        __syncthreads();
    }
}

// Restarted IGS-GMRES(m) on system `sid`, the same control flow as the single-system solver.
__device__ void b_solve_system(const Args &a, const Run &run, int sid, double *V, double *sm,
                               const SmemLayout &L, Shared &sh)
{
    Sys S;
    S.row0 = a.sys_row0[sid];
    S.n = (int)(a.sys_row0[sid + 1] - S.row0);
    S.n2 = round_up(S.n, 2);
    S.ldv = round_up(S.n, 4);
    S.slice0 = a.sys_slice0[sid];
    const double *b = run.b + S.row0;
    double *x = run.x + S.row0;
    const double *x0 = run.x0_given ? run.x0 + S.row0 : nullptr;
    double *part = sm + L.part, *red = sm + L.red;

    for (int i = threadIdx.x; i < S.n; i += blockDim.x) x[i] = x0 ? x0[i] : 0.0;
    b_sumsq(S, b, nullptr, 1, part, red);
    if (threadIdx.x == 0) {
        sh.nb = sqrt(red[0]);
        sh.normA = a.normA[sid];
        sh.cycles = 0;
        sh.steps = 0;
        sh.status = IGS_NOT_CONVERGED;
        sh.beta = nan("");
    }
    __syncthreads();
    for (;;) {
        // r_0 = b - A x_0 into V[:, 0]; beta(x) per eq. "nrbe" (zero residual: beta = 0).
        b_spmv<false>(a, S, x, b, V);
        __syncthreads();
        b_sumsq(S, V, x, 2, part, red);
        int brk = 0;
        if (threadIdx.x == 0) {
            const double rn = sqrt(red[0]), xn = sqrt(red[1]);
            const double beta = rn == 0.0 ? 0.0 : rn / (sh.nb + sh.normA * xn);
            sh.beta = beta;
            if (!isfinite(beta)) {
                sh.status = IGS_ENUMERIC;
                brk = 1;
            } else if (beta <= run.tol || rn == 0.0) {
                sh.status = IGS_OK;
                brk = 1;
            } else if (sh.cycles >= run.max_cycles) {
                sh.status = IGS_NOT_CONVERGED;
                brk = 1;
            }
            sh.rho = rn;
            sh.stop_den = sh.nb + sh.normA * xn;
            sh.stop = brk;
        }
        __syncthreads();
        if (sh.stop) break;
        b_cycle(a, run, S, V, sm, L, sh);
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
        // x_m = x_0 + V_m y_m (y by back substitution on the Givens factor).
        if (done > 0) {
            if ((int)(threadIdx.x >> 5) == sh.swarp) w_upper_solve(done, V + a.r_offset, sm + L.g, sm + L.y);
            __syncthreads();
            b_xupdate(S, V, done, sm + L.y, x);
        }
        __syncthreads();
        if (cst == IGS_BREAKDOWN) {
            b_spmv<false>(a, S, x, b, V);
            __syncthreads();
            b_sumsq(S, V, x, 2, part, red);
            if (threadIdx.x == 0) {
                const double rn = sqrt(red[0]), xn = sqrt(red[1]);
                const double beta = rn == 0.0 ? 0.0 : rn / (sh.nb + sh.normA * xn);
                sh.beta = beta;
                sh.status = (isfinite(beta) && beta <= run.tol) ? IGS_OK : IGS_BREAKDOWN;
            }
            __syncthreads();
            break;
        }
    }
    if (threadIdx.x == 0) {
        if (run.beta) run.beta[sid] = sh.beta;
        if (run.status) run.status[sid] = sh.status;
        if (run.steps) run.steps[sid] = sh.steps;
        if (run.cycles) run.cycles[sid] = sh.cycles;
        atomicAdd(&a.summary[0], (unsigned long long)sh.steps);
        const int k = sh.status + 6;  // status codes -6..2 -> 0..8
        if (k >= 0 && k < 9) atomicAdd(&a.summary[1 + k], 1ull);
    }
    __syncthreads();
}

// The persistent batched solver: CTAs take systems from the queue until it is empty.
// Instantiated per block size T with the register budget of MINB resident CTAs per SM.
template <int T, int MINB>
__global__ void __launch_bounds__(T, MINB) k_batch_solve(Args a, const Run *__restrict__ runp)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ Shared sh;
    __shared__ Run run;
    __shared__ int s_next;
    if (threadIdx.x == 0) {
        run = *runp;
        // Single-warp steps go to warp (hardware warp slot / 4) mod warps: CTAs that share an
        // SM then put them on different SM sub-partitions.  Any choice gives the same results.
        unsigned wid;
        asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid));
        sh.swarp = (int)((wid >> 2) % (blockDim.x >> 5));
    }
    const SmemLayout L = smem_layout(a.nmax, a.m);
    double *V = a.vslots + (int64_t)blockIdx.x * a.slot_stride;
    for (;;) {
        if (threadIdx.x == 0) s_next = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int q = s_next;
        __syncthreads();
        if (q >= run.count) break;
        b_solve_system(a, run, run.order[q], V, sm, L, sh);
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
    __shared__ double s_lam;
    const SmemLayout L = smem_layout(a.nmax, a.m);
    double *V = a.vslots + (int64_t)blockIdx.x * a.slot_stride;
    Args at = a;  // A^T in the same SELL form and slicing
    at.sell_off = at_off;
    at.sell_col = at_col;
    at.sell_val = at_val;
    for (int sid = blockIdx.x; sid < count; sid += gridDim.x) {
        Sys S;
        S.row0 = a.sys_row0[sid];
        S.n = (int)(a.sys_row0[sid + 1] - S.row0);
        S.n2 = round_up(S.n, 2);
        S.ldv = round_up(S.n, 4);
        S.slice0 = a.sys_slice0[sid];
        double *xv = V, *yv = V + S.ldv, *uv = V + 2 * (int64_t)S.ldv;
        const double sc = 1.0 / sqrt((double)S.n);
        for (int i = threadIdx.x; i < S.n; i += blockDim.x) {
            uint64_t hsh = (uint64_t)i * 0x9E3779B97F4A7C15ull;
            hsh ^= hsh >> 29;
            xv[i] = sc * (0.5 + (double)(hsh >> 11) * 0x1p-53);
        }
        __syncthreads();
        double lam = 0.0;
        for (int it = 0; it < iters; ++it) {
            b_spmv<false>(a, S, xv, nullptr, yv);
            __syncthreads();
            b_spmv<false>(at, S, yv, nullptr, uv);
            __syncthreads();
            b_sumsq(S, uv, nullptr, 1, sm + L.part, sm + L.red);
            if (threadIdx.x == 0) s_lam = sqrt(sm[L.red]);
            __syncthreads();
            lam = s_lam;
            const double f = lam > 0.0 ? 1.0 / lam : 0.0;
            for (int i = threadIdx.x; i < S.n; i += blockDim.x) xv[i] = uv[i] * f;
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
        if (cudaFuncSetAttribute(batch_kernel(t), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem) !=
            cudaSuccess)
            return bail(IGS_ECUDA);
    }
    if (cudaFuncSetAttribute(k_batch_norm2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem) !=
        cudaSuccess)
        return bail(IGS_ECUDA);

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
}

extern "C" int igs_batch_set_config(igs_batch *bt, int block_threads, int blocks_per_sm)
{
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
}

extern "C" int igs_batch_tune(igs_batch *bt, int gs_iters, double tol_beta, int max_restarts)
{
    if (!bt) return IGS_EINVAL;
    if (gs_iters < 1 || gs_iters > 2 || !(tol_beta >= 0.0) || max_restarts < 1)
        return fail(bt, IGS_EINVAL, "invalid tuning options");
    if (cudaSetDevice(bt->device) != cudaSuccess) return fail(bt, IGS_ECUDA, "cudaSetDevice");
    return autotune(bt, gs_iters, tol_beta, max_restarts);
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
