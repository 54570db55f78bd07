// Block reductions of Alg. 4.1 (steps 5 and 14) and Alg. 4.2 (step 4), and the basis
// updates of Alg. 4.1 (steps 13 and 16), evaluated in double-float arithmetic on the FP32
// pipes: the IGS_PREC_FP64_DF form of igs_solve.
//
// Why: on GB300 the FP64 pipe retires 2 FMAs per clock per SM (1.26 TFLOP/s), so the FP64
// multi-dot [V, w]^T [w, z] (2 FMAs per 8-byte basis element) runs at about a third of
// HBM bandwidth.  The FP32 pipes are 64 times faster.  Here every FP64 operand a is split
// without any FP64 instruction into a = hi + lo (+ r), hi = a's sign, exponent and top 24
// significant bits, lo = the remaining 29 bits rounded to 23 (|r| <= 2^-47 |a|); the
// product of two split numbers is formed as the exact product hi*hi' = p + e (FMA) plus the
// cross terms hi*lo' + lo*hi' in FP32 (per-product error <= ~2^-45 |a a'|, dropped lo*lo'
// included), and the products are summed per lane with TwoSum (Knuth) into a double-float
// accumulator, folded into a double-float total every 32 elements; the lanes' totals are
// added in a fixed order (double-float) and each block's sum is converted to FP64 once, into
// the FP64 kernel's per-block partial-sum layout, so the single-block steps that follow are
// unchanged.
//
// Accuracy: each product carries a relative error of at most ~2^-45 (against 2^-53 for an
// FP64 product), but these errors are independent across the n terms of a dot product, so
// for vectors spread over n >= 2^14 rows their contribution (~2^-46 ||a|| ||a'|| / sqrt(n))
// is below the FP64 accumulation error the FP64 kernel itself makes; the library uses these
// kernels only from that size on.  Range: the split is exact to 2^-47 for
// 2^-100 <= |a| < 2^127; smaller operands lose low-order bits (lo becomes an FP32
// subnormal) down to FP32 precision at 2^-126, below which they count as 0; |a| >= 2^127
// makes the sum non-finite (the solve then stops with IGS_ENUMERIC).
#include "igs_internal.h"

namespace igs {

namespace {

__device__ __forceinline__ bool df_halted(const DevState *st) { return st->halt != 0; }

// (S, s) += (ah + al) * (xh + xl): exact product of the high parts by FMA, cross terms in
// FP32, TwoSum of the high part into S (the intrinsics are never contracted into FMAs).
__device__ __forceinline__ void df_acc(float &S, float &s, float ah, float al, float xh, float xl)
{
    const float p = __fmul_rn(ah, xh);
    const float e = __fmaf_rn(ah, xh, -p);
    const float c = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
    const float t = __fadd_rn(S, p);
    const float bp = __fsub_rn(t, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    S = t;
    s = __fadd_rn(s, __fadd_rn(err, c));
}

// The FP64 value of a finite FP32 number, assembled from its bits with integer operations
// (no FP64-pipe conversion): sign, exponent rebiased by 1023 - 127 = 896, fraction shifted
// up by 29.  Exact for normal numbers and zero; FP32 subnormals (|f| < 2^-126) give 0.
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned hw = e == 0u ? (u & 0x80000000u) : (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
    const unsigned lw = e == 0u ? 0u : (u << 29);
    return __hiloint2double((int)hw, (int)lw);
}

// (A, a) += (B, b) for double-float numbers (TwoSum of the high parts, the low parts added
// to its error, renormalised by Fast2Sum): error ~2^-48 of the operands' magnitude.  FP32
// only: an FP64 instruction holds a sub-partition's FP64 pipe for 64 clocks on GB300, so
// the reductions below stay off that pipe until one conversion per block and column.
__device__ __forceinline__ void df_add(float &A, float &a, float B, float b)
{
    const float t = __fadd_rn(A, B);
    const float bp = __fsub_rn(t, A);
    float e = __fadd_rn(__fsub_rn(A, __fsub_rn(t, bp)), __fsub_rn(B, bp));
    e = __fadd_rn(e, __fadd_rn(a, b));
    A = __fadd_rn(t, e);
    a = __fsub_rn(e, __fsub_rn(A, t));
}

}  // namespace

// =====================================================================================
// Double-float block multi-dot: the grid, partial-sum layout and summation of the lane sums
// are those of the FP64 multi-dot (part[rb*(NQ*p) + q*p + c] = sum over row block rb of
// V[:,c] . X_q); what differs is that each warp streams ALL the group's columns over its
// row sub-slice (so each X row is loaded and split once per block, not once per column)
// and the products are accumulated in double-float.  Each lane handles two consecutive rows
// per 64-row segment: one copy instruction of a warp moves 512 contiguous bytes of a column.
// The segments are staged in shared memory by cp.async, double-buffered: while a warp
// computes on segment g, the copies of segment g+1 are in flight, so the HBM latency is
// hidden without holding the next segment in registers.  Each lane
// reads back only the 16-byte chunks it copied itself, so no barrier is needed.  Lane sums
// are folded into a double-float total every 32 elements, combined over the warp by a
// double-float shuffle tree and over the block's warps in order, and converted to FP64 once
// per block and column (FP64 instructions would serialise on the narrow FP64 pipe).
// =====================================================================================
constexpr int kDfStreams = kDotsColsPerBlock + 2;           // up to 4 columns and 2 vectors
constexpr int kDfStageDoubles = kDfStreams * 64;            // one 64-row segment of each stream
constexpr int kDfStages = 2;  // a power of two: segment in use + one in flight (a third
                               // stage measured slower: by 9 % with modulo stage indices,
                               // by 1-2 % with rotating ones)
constexpr size_t kDfDotsSmem = sizeof(double) * kDfStages * kDfStageDoubles * (kStreamThreads / 32);

__device__ __forceinline__ void cp_async16(double *dst, const double *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// VDF false: V and the vectors are FP64, split on the fly; true: all of them stored split.
template <int NQ, bool VDF>
__global__ void __launch_bounds__(kStreamThreads, kDotsBlocksPerSM)
k_dots_df(const double *__restrict__ V, int64_t ld, int p, int64_t n4, int64_t rows,
          const double *__restrict__ x0, const double *__restrict__ x1, double *__restrict__ part,
          const DevState *st, int check_halt)
{
    IGS_PDL_ENTER();
    if (check_halt && df_halted(st)) return;
    constexpr int W = kStreamThreads / 32;
    constexpr int CW = kDotsColsPerBlock;
    constexpr int kFold = 16;  // segments (32 elements per lane) between folds
    extern __shared__ double dsm[];
    __shared__ float2 red[NQ][CW][W];
    const int rb = blockIdx.x, G = gridDim.y, cg = blockIdx.y;
    const int c_lo = (int)((int64_t)cg * p / G), c_hi = (int)((int64_t)(cg + 1) * p / G);
    const int cw = c_hi - c_lo;  // <= CW (the launcher's plan guarantees it)
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t r_lo = (int64_t)rb * rows;
    const int64_t r_hi = r_lo + rows < n4 ? r_lo + rows : n4;
    double *stage0 = dsm + (size_t)wid * kDfStages * kDfStageDoubles + 2 * lane;  // this lane's slots
    const double *vbase = V + (int64_t)c_lo * ld;
    float A[CW][NQ], a[CW][NQ], S[CW][NQ], s[CW][NQ];  // fold total and running chunk
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            A[c][q] = 0.f;
            a[c][q] = 0.f;
            S[c][q] = 0.f;
            s[c][q] = 0.f;
        }
    const int64_t nseg = r_lo < r_hi ? (r_hi - r_lo + 63) >> 6 : 0;
    const int64_t g0 = nseg * wid / W, g1 = nseg * (wid + 1) / W;
    // copy segment g into stage buffer b: streams 0..NQ-1 = X, NQ.. = the columns
    auto issue = [&](int64_t g, int b) {
        const int64_t i = r_lo + (g << 6) + 2 * lane;
        if (i < r_hi) {
            double *dst = stage0 + b * kDfStageDoubles;
            cp_async16(dst, x0 + i);
            if (NQ == 2) cp_async16(dst + 64, x1 + i);
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (c < cw) cp_async16(dst + 64 * (NQ + c), vbase + (int64_t)c * ld + i);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int since = 0;
    // the products of one staged segment (ncol of the group's columns) and the periodic fold
    auto consume = [&](const double *src, int ncol) {
        float xh[NQ][2], xl[NQ][2];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (VDF) {  // stored split: (hi, lo) of two rows
                const float4 xv = *reinterpret_cast<const float4 *>(src + 64 * q);
                xh[q][0] = xv.x;
                xl[q][0] = xv.y;
                xh[q][1] = xv.z;
                xl[q][1] = xv.w;
            } else {
                const double2 xv = *reinterpret_cast<const double2 *>(src + 64 * q);
                df_split(xv.x, xh[q][0], xl[q][0]);
                df_split(xv.y, xh[q][1], xl[q][1]);
            }
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            if (c < ncol) {
                float h0, l0, h1, l1;
                if (VDF) {
                    const float4 v = *reinterpret_cast<const float4 *>(src + 64 * (NQ + c));
                    h0 = v.x;
                    l0 = v.y;
                    h1 = v.z;
                    l1 = v.w;
                } else {
                    const double2 v = *reinterpret_cast<const double2 *>(src + 64 * (NQ + c));
                    df_split(v.x, h0, l0);
                    df_split(v.y, h1, l1);
                }
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    df_acc(S[c][q], s[c][q], h0, l0, xh[q][0], xl[q][0]);
                    df_acc(S[c][q], s[c][q], h1, l1, xh[q][1], xl[q][1]);
                }
            }
        }
    };
    auto fold = [&]() {
        if (++since == kFold) {
            since = 0;
#pragma unroll
            for (int c = 0; c < CW; ++c)
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    df_add(A[c][q], a[c][q], S[c][q], s[c][q]);
                    S[c][q] = 0.f;
                    s[c][q] = 0.f;
                }
        }
    };
    if (cw == CW && r_lo + (g1 << 6) <= r_hi) {
        // Fast path (warp-uniform: every segment of this warp lies inside the row block, and
        // the group has all CW columns): the copies come from running source pointers into
        // fixed shared-memory addresses, with no per-lane bounds or column tests.  Same
        // segments, same order, same arithmetic as the general path below.
        const int nsg = (int)(g1 - g0);
        const int64_t i0 = r_lo + (g0 << 6) + 2 * lane;
        const double *sp[NQ + CW];
        sp[0] = x0 + i0;
        if (NQ == 2) sp[1] = x1 + i0;
#pragma unroll
        for (int c = 0; c < CW; ++c) sp[NQ + c] = vbase + (int64_t)c * ld + i0;
        const unsigned d0 = (unsigned)__cvta_generic_to_shared(stage0);
        auto issue_next = [&](int b) {  // the next segment into stage b, then advance
            const unsigned d = d0 + (unsigned)(b * kDfStageDoubles * sizeof(double));
#pragma unroll
            for (int k = 0; k < NQ + CW; ++k) {
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 512u * k), "l"(sp[k]) : "memory");
                sp[k] += 64;
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        static_assert(kDfStages == 2, "the fast path alternates two stage buffers");
        if (nsg > 0)
            issue_next(0);
        else
            asm volatile("cp.async.commit_group;" ::: "memory");
        for (int j = 0; j < nsg; ++j) {
            const int b = j & 1;
            if (j + 1 < nsg)
                issue_next(b ^ 1);
            else
                asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            consume(stage0 + b * kDfStageDoubles, CW);
            fold();
        }
    } else {
        // general path: a ragged last row block or a narrower column group
        // prologue: the first kDfStages - 1 segments (an empty group where there are fewer)
#pragma unroll
        for (int j = 0; j < kDfStages - 1; ++j) {
            if (g0 + j < g1)
                issue(g0 + j, j);
            else
                asm volatile("cp.async.commit_group;" ::: "memory");
        }
        for (int64_t g = g0; g < g1; ++g) {
            const int b = (int)(g - g0) & (kDfStages - 1);
            if (g + kDfStages - 1 < g1)
                issue(g + kDfStages - 1, (int)(g + kDfStages - 1 - g0) & (kDfStages - 1));
            else
                asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group %0;" ::"n"(kDfStages - 1) : "memory");
            const int64_t i = r_lo + (g << 6) + 2 * lane;
            if (i < r_hi) consume(stage0 + b * kDfStageDoubles, cw);
            fold();
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // lane totals, a fixed-order double-float warp tree, the W warp sums in order, and one
    // conversion to FP64 per (vector, column)
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float h = A[c][q], l = a[c][q];
            df_add(h, l, S[c][q], s[c][q]);
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_down_sync(0xffffffffu, h, o);
                const float ol = __shfl_down_sync(0xffffffffu, l, o);
                df_add(h, l, oh, ol);
            }
            if (lane == 0) red[q][c][wid] = make_float2(h, l);
        }
    __syncthreads();
    if (t < NQ * CW) {
        const int q = t / CW, c = t % CW;
        if (c < cw) {
            float h = 0.f, l = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) df_add(h, l, red[q][c][k].x, red[q][c][k].y);
            part[(int64_t)rb * NQ * p + (int64_t)q * p + c_lo + c] = (double)h + (double)l;
        }
    }
}

// =====================================================================================
// Double-float basis update (Alg. 4.1 steps 7, 11, 13 and 16 in the IGS_PREC_FP64_DF form):
//   out[i] = a * src[i] - sum_{c<p} V[i,c] coef[c]
// with the same row ownership as the FP64 update (two rows per thread, a whole number of
// blocks per SM, block-contiguous row ranges) and the same norm_last semantics (column p-1
// first scaled in place by st->inv_gamma, which is also a).  Each row's sum over the
// columns is a double-float accumulation of split products (the coefficients are split
// once per block, in shared memory); a * src[i] and the final subtraction are FP64.
// The columns stream through shared memory in chunks of kUpdChunk, kUpdStages chunks in
// flight per thread (cp.async; each thread copies and reads back only its own 16-byte
// slots), so the loads' latency is covered without holding them in registers.
// Error of out[i]: <= ~2^-45 sum_c |V[i,c] coef[c]| (FP64: p 2^-53 of the same sum).
// =====================================================================================
constexpr int kUpdChunk = 4;
constexpr int kUpdStages = 3;
constexpr size_t kUpdStageBytes = (size_t)kUpdChunk * 16 * kStreamThreads;  // one chunk, all threads
constexpr size_t kUpdSmemFixed = kUpdStages * kUpdStageBytes;              // + 8 p for the coefficients

// V: FP64 basis (VDF false; split on the fly) or the split basis of the double-float form
// (VDF true: each element stored as its (hi, lo) FP32 pair in the same 8 bytes).  With
// norm_last, column p-1 is the lagged w: FP64 V scales it in place; the split basis takes the
// FP64 w from wsrc and stores the split of w * a into column p-1.  out (FP64) always; out_df
// (nullable) also gets the split of each output row.  neg_coef negates coef; p_from_state
// takes p from st->ncols (the x update at the cycle's end).
template <bool VDF>
__global__ void __launch_bounds__(kStreamThreads, kUpdateBlocksPerSM)
k_update_df(double *V, int64_t ld, int p, int64_t n, const double *__restrict__ coef, int neg_coef, double alpha,
            const double *src, double *out, float2 *out_df, const double *wsrc, int norm_last, int p_from_state,
            DevState *st, int check_halt)
{
    IGS_PDL_ENTER();
    if (check_halt && df_halted(st)) return;
    extern __shared__ double usm[];
    if (p_from_state) p = st->ncols;
    // stage buffers: [stage][column in chunk][thread] of 16 bytes; then the coefficient splits
    double2 *stg = reinterpret_cast<double2 *>(usm);
    float *scf = reinterpret_cast<float *>(usm + kUpdSmemFixed / sizeof(double));  // hi [0,p), lo [p,2p)
    const double a = norm_last ? st->inv_gamma : alpha;
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        float h, l;
        df_split(neg_coef ? -coef[c] : coef[c], h, l);
        scf[c] = h;
        scf[p + c] = l;
    }
    __syncthreads();
    const int pc = norm_last ? p - 1 : p;
    const int nchunks = (pc + kUpdChunk - 1) / kUpdChunk;
    const int64_t npairs = (n + 1) >> 1;
    const int64_t ppb = (npairs + gridDim.x - 1) / gridDim.x;
    const int64_t pr_lo = (int64_t)blockIdx.x * ppb;
    const int64_t pr_hi = pr_lo + ppb < npairs ? pr_lo + ppb : npairs;
    const int t = threadIdx.x;
    for (int64_t pr = pr_lo + t; pr < pr_hi; pr += blockDim.x) {
        const int64_t i = 2 * pr;
        const double *vi = V + i;
        // the next chunk to copy (js), its stage (ss) and its first column's address; the
        // stages rotate without a modulo and the columns advance by pointer increments
        const unsigned sbase = (unsigned)__cvta_generic_to_shared(stg + t);
        const double *colp = vi;
        int js = 0, ss = 0;
        auto issue = [&]() {
            if (js < nchunks) {
                const unsigned d = sbase + (unsigned)(ss * kUpdChunk * kStreamThreads * 16);
                const int left = pc - js * kUpdChunk;
#pragma unroll
                for (int q = 0; q < kUpdChunk; ++q)
                    if (q < left)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                     ::"r"(d + (unsigned)(q * kStreamThreads * 16)), "l"(colp + (int64_t)q * ld)
                                     : "memory");
                colp += (int64_t)kUpdChunk * ld;
                if (++ss == kUpdStages) ss = 0;
                ++js;
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
#pragma unroll
        for (int j = 0; j < kUpdStages - 1; ++j) issue();
        float S0 = 0.f, s0 = 0.f, S1 = 0.f, s1 = 0.f;
        int cs = 0;  // the stage chunk j was copied into
        for (int j = 0; j < nchunks; ++j) {
            issue();
            asm volatile("cp.async.wait_group %0;" ::"n"(kUpdStages - 1) : "memory");
            const double2 *cur = stg + (size_t)cs * kUpdChunk * kStreamThreads + t;
            if (++cs == kUpdStages) cs = 0;
#pragma unroll
            for (int q = 0; q < kUpdChunk; ++q) {
                const int c = j * kUpdChunk + q;
                if (c < pc) {
                    float h0, l0, h1, l1;
                    if (VDF) {
                        const float4 v = *reinterpret_cast<const float4 *>(cur + q * kStreamThreads);
                        h0 = v.x;
                        l0 = v.y;
                        h1 = v.z;
                        l1 = v.w;
                    } else {
                        const double2 v = cur[q * kStreamThreads];
                        df_split(v.x, h0, l0);
                        df_split(v.y, h1, l1);
                    }
                    df_acc(S0, s0, h0, l0, scf[c], scf[p + c]);
                    df_acc(S1, s1, h1, l1, scf[c], scf[p + c]);
                }
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (norm_last) {
            double2 v = *reinterpret_cast<const double2 *>((VDF ? wsrc : V + (int64_t)(p - 1) * ld) + i);
            v.x *= a;
            v.y *= a;
            float h0, l0, h1, l1;
            df_split(v.x, h0, l0);
            df_split(v.y, h1, l1);
            if (VDF)
                *reinterpret_cast<float4 *>(V + (int64_t)(p - 1) * ld + i) = make_float4(h0, l0, h1, l1);
            else
                *reinterpret_cast<double2 *>(V + (int64_t)(p - 1) * ld + i) = v;
            df_acc(S0, s0, h0, l0, scf[p - 1], scf[2 * p - 1]);
            df_acc(S1, s1, h1, l1, scf[p - 1], scf[2 * p - 1]);
        }
        const double2 sv = *reinterpret_cast<const double2 *>(src + i);
        double2 o;
        o.x = fma(a, sv.x, -(f2d_bits(S0) + f2d_bits(s0)));
        o.y = fma(a, sv.y, -(f2d_bits(S1) + f2d_bits(s1)));
        *reinterpret_cast<double2 *>(out + i) = o;
        if (out_df) {
            float h0, l0, h1, l1;
            df_split(o.x, h0, l0);
            df_split(o.y, h1, l1);
            *reinterpret_cast<float4 *>(out_df + i) = make_float4(h0, l0, h1, l1);
        }
    }
}

// Alg. 4.2's fused update (steps 10-11 and 13) on the split basis, double-float: per row
//   v_{k-1} = (u - V_nb r^(2)) / gamma        (split into column nb, where split(u) was)
//   u_k     = z / gamma - V_nb r^(1) - v_{k-1} r^(1)_nb   (FP64 into wu, split into column nb+1)
// with u taken in FP64 from wu (each thread reads its rows of wu before writing them) and the
// two sums over the nb split columns accumulated in double-float (two products per basis
// element, one pass over V).  vonly (the flush): v_{k-1} only.  Same row ownership and
// column staging as k_update_df.
__global__ void __launch_bounds__(kStreamThreads, kUpdateBlocksPerSM)
k_update_1r_df(double *V, int64_t ld, int nb, int64_t n, const double *__restrict__ r2,
               const double *__restrict__ r1, const double *__restrict__ z, double *wu, int vonly,
               const DevState *st)
{
    IGS_PDL_ENTER();
    if (df_halted(st)) return;
    extern __shared__ double usm[];
    double2 *stg = reinterpret_cast<double2 *>(usm);
    float *sc = reinterpret_cast<float *>(usm + kUpdSmemFixed / sizeof(double));
    float *r2h = sc, *r2l = sc + nb, *r1h = sc + 2 * nb, *r1l = sc + 3 * nb;
    for (int c = threadIdx.x; c < nb; c += blockDim.x) {
        float h, l;
        df_split(r2[c], h, l);
        r2h[c] = h;
        r2l[c] = l;
        df_split(vonly ? 0.0 : r1[c], h, l);
        r1h[c] = h;
        r1l[c] = l;
    }
    __syncthreads();
    const double ig = st->inv_gamma;
    const double r1nb = vonly ? 0.0 : r1[nb];
    const int nchunks = (nb + kUpdChunk - 1) / kUpdChunk;
    const int64_t npairs = (n + 1) >> 1;
    const int64_t ppb = (npairs + gridDim.x - 1) / gridDim.x;
    const int64_t pr_lo = (int64_t)blockIdx.x * ppb;
    const int64_t pr_hi = pr_lo + ppb < npairs ? pr_lo + ppb : npairs;
    const int t = threadIdx.x;
    for (int64_t pr = pr_lo + t; pr < pr_hi; pr += blockDim.x) {
        const int64_t i = 2 * pr;
        const double *vi = V + i;
        // the next chunk to copy (js), its stage (ss) and its first column's address; the
        // stages rotate without a modulo and the columns advance by pointer increments
        const unsigned sbase = (unsigned)__cvta_generic_to_shared(stg + t);
        const double *colp = vi;
        int js = 0, ss = 0;
        auto issue = [&]() {
            if (js < nchunks) {
                const unsigned d = sbase + (unsigned)(ss * kUpdChunk * kStreamThreads * 16);
                const int left = nb - js * kUpdChunk;
#pragma unroll
                for (int q = 0; q < kUpdChunk; ++q)
                    if (q < left)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                     ::"r"(d + (unsigned)(q * kStreamThreads * 16)), "l"(colp + (int64_t)q * ld)
                                     : "memory");
                colp += (int64_t)kUpdChunk * ld;
                if (++ss == kUpdStages) ss = 0;
                ++js;
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
#pragma unroll
        for (int j = 0; j < kUpdStages - 1; ++j) issue();
        float A0 = 0.f, a0 = 0.f, A1 = 0.f, a1 = 0.f, B0 = 0.f, b0 = 0.f, B1 = 0.f, b1 = 0.f;
        int cs = 0;  // the stage chunk j was copied into
        for (int j = 0; j < nchunks; ++j) {
            issue();
            asm volatile("cp.async.wait_group %0;" ::"n"(kUpdStages - 1) : "memory");
            const double2 *cur = stg + (size_t)cs * kUpdChunk * kStreamThreads + t;
            if (++cs == kUpdStages) cs = 0;
#pragma unroll
            for (int q = 0; q < kUpdChunk; ++q) {
                const int c = j * kUpdChunk + q;
                if (c < nb) {
                    const float4 v = *reinterpret_cast<const float4 *>(cur + q * kStreamThreads);
                    df_acc(A0, a0, v.x, v.y, r2h[c], r2l[c]);
                    df_acc(A1, a1, v.z, v.w, r2h[c], r2l[c]);
                    if (!vonly) {
                        df_acc(B0, b0, v.x, v.y, r1h[c], r1l[c]);
                        df_acc(B1, b1, v.z, v.w, r1h[c], r1l[c]);
                    }
                }
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        const double2 u = *reinterpret_cast<const double2 *>(wu + i);
        double2 vn;
        vn.x = (u.x - (f2d_bits(A0) + f2d_bits(a0))) * ig;
        vn.y = (u.y - (f2d_bits(A1) + f2d_bits(a1))) * ig;
        float h0, l0, h1, l1;
        df_split(vn.x, h0, l0);
        df_split(vn.y, h1, l1);
        *reinterpret_cast<float4 *>(V + (int64_t)nb * ld + i) = make_float4(h0, l0, h1, l1);
        if (!vonly) {
            const double2 zz = *reinterpret_cast<const double2 *>(z + i);
            double2 un;
            un.x = fma(zz.x, ig, -((f2d_bits(B0) + f2d_bits(b0)) + vn.x * r1nb));
            un.y = fma(zz.y, ig, -((f2d_bits(B1) + f2d_bits(b1)) + vn.y * r1nb));
            *reinterpret_cast<double2 *>(wu + i) = un;
            df_split(un.x, h0, l0);
            df_split(un.y, h1, l1);
            *reinterpret_cast<float4 *>(V + (int64_t)(nb + 1) * ld + i) = make_float4(h0, l0, h1, l1);
        }
    }
}

// dst_df[i] = split(src[i] * scale) and, when dst64 is given, dst64[i] = src[i] * scale, with
// scale = st->inv_rho (which = 0) or st->inv_gamma (which = 1): v_1 = r_0 / rho at a cycle's
// start and the flush's v_{m+1} = w_{m+1} / gamma into the split basis.
__global__ void __launch_bounds__(kStreamThreads)
k_scale_df(int64_t n, const double *src, float2 *dst_df, double *dst64, int which, const DevState *st, int check_halt)
{
    IGS_PDL_ENTER();
    if (check_halt && df_halted(st)) return;
    const double sc = which == 0 ? st->inv_rho : st->inv_gamma;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = src[i] * sc;
        float h, l;
        df_split(v, h, l);
        dst_df[i] = make_float2(h, l);
        if (dst64) dst64[i] = v;
    }
}

// x[i] += sum_{c < st->ncols} V[i,c] y[c] over the split basis, in FP64: each stored element
// is exactly hi + lo, rebuilt from its bits with integer operations and one FP64 addition,
// then one FP64 FMA per element (x = x0 + V_m y_m at the cycle's end; once per cycle).
__global__ void __launch_bounds__(kStreamThreads)
k_xupdate_vdf(const double *V, int64_t ld, int64_t n, const double *__restrict__ y, double *x, const DevState *st)
{
    IGS_PDL_ENTER();
    extern __shared__ double ys[];
    const int p = st->ncols;
    for (int c = threadIdx.x; c < p; c += blockDim.x) ys[c] = y[c];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double s = 0.0;
        for (int c = 0; c < p; ++c) {
            const float2 v = reinterpret_cast<const float2 *>(V + (int64_t)c * ld)[i];
            s = fma(f2d_bits(v.x) + f2d_bits(v.y), ys[c], s);
        }
        x[i] += s;
    }
}

// In place: the split basis (rows < ld, cols columns) back to FP64, hi + lo (for igs_arnoldi's
// output of the double-float form).
__global__ void __launch_bounds__(kStreamThreads) k_df_to_f64(double *V, int64_t count)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const float2 v = reinterpret_cast<const float2 *>(V)[i];
        V[i] = (double)v.x + (double)v.y;
    }
}

bool dots_df_applies(const Workspace &w) { return w.n >= kDfMinRows; }

cudaError_t launch_update_df(const Workspace &w, int p, const double *coef, double alpha, const double *src,
                             double *out, bool norm_last, cudaStream_t s)
{
    return launch_update_df_ex(w, p, coef, false, alpha, src, out, nullptr, nullptr, norm_last, false, false, s);
}

cudaError_t launch_update_df_ex(const Workspace &w, int p, const double *coef, bool neg_coef, double alpha,
                                const double *src, double *out, float2 *out_df, const double *wsrc, bool norm_last,
                                bool p_from_state, bool vdf, cudaStream_t s)
{
    const int pmax = p_from_state ? w.mmax + 1 : p;
    const size_t smem = kUpdSmemFixed + 2 * sizeof(float) * (size_t)(pmax > 0 ? pmax : 1);
    const int grid = w.num_sms * kUpdateBlocksPerSM;
    if (vdf)
        launch_k(w.pdl, k_update_df<true>, dim3(grid), dim3(kStreamThreads), smem, s, w.V, w.ld, p, w.n, coef,
                 neg_coef ? 1 : 0, alpha, src, out, out_df, wsrc, norm_last ? 1 : 0, p_from_state ? 1 : 0, w.st, 1);
    else
        launch_k(w.pdl, k_update_df<false>, dim3(grid), dim3(kStreamThreads), smem, s, w.V, w.ld, p, w.n, coef,
                 neg_coef ? 1 : 0, alpha, src, out, out_df, wsrc, norm_last ? 1 : 0, p_from_state ? 1 : 0, w.st, 1);
    return cudaGetLastError();
}

cudaError_t launch_update_1r_df(const Workspace &w, int nb, const double *z, double *wu, bool vonly, cudaStream_t s)
{
    const size_t smem = kUpdSmemFixed + 4 * sizeof(float) * (size_t)(nb + 1);
    launch_k(w.pdl, k_update_1r_df, dim3(w.num_sms * kUpdateBlocksPerSM), dim3(kStreamThreads), smem, s, w.V, w.ld,
             nb, w.n, (const double *)w.r2v, (const double *)w.r1v, z, wu, vonly ? 1 : 0, (const DevState *)w.st);
    return cudaGetLastError();
}

cudaError_t launch_scale_df(const Workspace &w, const double *src, float2 *dst_df, double *dst64, int which,
                            bool check_halt, cudaStream_t s)
{
    launch_k(false, k_scale_df, dim3(w.num_sms * kBlocksPerSM), dim3(kStreamThreads), 0, s, w.n, src, dst_df, dst64,
             which, (const DevState *)w.st, check_halt ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_xupdate_vdf(const Workspace &w, cudaStream_t s)
{
    const size_t smem = sizeof(double) * (size_t)(w.mmax + 1);
    launch_k(w.pdl, k_xupdate_vdf, dim3(w.num_sms * kUpdateBlocksPerSM), dim3(kStreamThreads), smem, s,
             (const double *)w.V, w.ld, w.n, (const double *)w.y, w.x, (const DevState *)w.st);
    return cudaGetLastError();
}

cudaError_t launch_df_to_f64(double *V, int64_t count, int num_sms, cudaStream_t s)
{
    launch_k(false, k_df_to_f64, dim3(num_sms * kBlocksPerSM), dim3(kStreamThreads), 0, s, V, count);
    return cudaGetLastError();
}

cudaError_t launch_dots_df(const Workspace &w, int p, const double *x0, const double *x1, bool check_halt,
                           cudaStream_t s, DotsPlan *plan_out)
{
    return launch_dots_df_ex(w, p, x0, x1, check_halt, false, s, plan_out);
}

cudaError_t launch_dots_df_ex(const Workspace &w, int p, const double *x0, const double *x1, bool check_halt,
                              bool vdf, cudaStream_t s, DotsPlan *plan_out)
{
    const DotsPlan pl = plan_dots(w, p);
    if (plan_out) *plan_out = pl;
    if ((p + pl.groups - 1) / pl.groups > kDotsColsPerBlock) return cudaErrorInvalidValue;
    const int64_t n4 = (w.n + 3) & ~int64_t(3);
    dim3 grid(pl.rblocks, pl.groups);
    const DevState *st = w.st;
    const int ch = check_halt ? 1 : 0;
    const size_t sm = kDfDotsSmem;
    const dim3 bl(kStreamThreads);
    const double *none = nullptr;
    if (x1 && vdf)
        launch_k(false, k_dots_df<2, true>, grid, bl, sm, s, w.V, w.ld, p, n4, pl.rows, x0, x1, w.part, st, ch);
    else if (x1)
        launch_k(false, k_dots_df<2, false>, grid, bl, sm, s, w.V, w.ld, p, n4, pl.rows, x0, x1, w.part, st, ch);
    else if (vdf)
        launch_k(false, k_dots_df<1, true>, grid, bl, sm, s, w.V, w.ld, p, n4, pl.rows, x0, none, w.part, st, ch);
    else
        launch_k(false, k_dots_df<1, false>, grid, bl, sm, s, w.V, w.ld, p, n4, pl.rows, x0, none, w.part, st, ch);
    return cudaGetLastError();
}

cudaError_t configure_df_kernels()
{
    // 48 KiB of stage buffers per block (3 blocks per SM): above the default dynamic limit
    const size_t dm = kDfDotsSmem;
    const size_t um = kUpdSmemFixed + 2 * sizeof(float) * (kMaxRestart + 1);
    cudaError_t e = raise_smem_limit((const void *)k_dots_df<1, false>, dm);
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_dots_df<2, false>, dm);
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_dots_df<1, true>, dm);
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_dots_df<2, true>, dm);
    // stage buffers (48 KiB) plus the coefficient splits of up to kMaxRestart + 1 columns
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_update_df<false>, um);
    if (e == cudaSuccess) e = raise_smem_limit((const void *)k_update_df<true>, um);
    if (e == cudaSuccess)
        e = raise_smem_limit((const void *)k_update_1r_df, kUpdSmemFixed + 4 * sizeof(float) * (kMaxRestart + 2));
    return e;
}

}  // namespace igs
