// Internal declarations shared by the kernels (igs_kernels.cu) and the C interface
// (igs_api.cu) of the GB300 IGS-GMRES library.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

namespace igs {

// Threads per block of the streaming kernels and of the small single-block kernels.
constexpr int kStreamThreads = 256;
constexpr int kSmallThreads = 256;
constexpr int kGivensThreads = 128;
// Target columns per block of the multi-dot kernel (few columns per block keep the number of
// per-block partial sums, which one block must add up afterwards, small).
constexpr int kDotsColsPerBlock = 4;
// Most columns one multi-dot block can take (its warps split into at most 8 column lanes).
constexpr int kDotsMaxGroupCols = 8;
// Resident blocks per SM assumed when sizing grids (256 threads, <= 128 registers).
constexpr int kBlocksPerSM = 2;
// Resident blocks per SM of the multi-dot kernel (256 threads, <= 80 registers).
constexpr int kDotsBlocksPerSM = 3;
// Basis update grid: a whole number of blocks per SM, each with an equal row range (the update
// is bound by the FP64 pipe, so an uneven block count per SM costs its share directly).
constexpr int kUpdateBlocksPerSM = 4;
// Largest restart length supported.  The small single-block steps hold L_p packed in shared
// memory: 8 (5p + p(p-1)/2) bytes <= 227 KiB gives p <= 232.
constexpr int kMaxRestart = 232;
// Widest uniform slice the ELL SpMV handles, and the largest padding (relative to SELL-32)
// accepted to use it.
constexpr int kMaxEllWidth = 8;
constexpr double kEllMaxPadding = 1.25;
// Breakdown threshold factor: gamma <= 64 eps ||H(1:j, j)||.
constexpr double kBreakdownFactor = 64.0 * 2.220446049250313e-16;

// Programmatic dependent launch: every kernel of a cycle first waits for its predecessor's
// results (griddepcontrol.wait; a no-op without PDL) and immediately allows its own
// dependents to be launched, so that a kernel's launch overlaps the tail of the previous one.
#define IGS_PDL_ENTER()                                              \
    do {                                                             \
        asm volatile("griddepcontrol.wait;" ::: "memory");           \
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
    } while (0)

// Launch with the programmatic-stream-serialization attribute when `pdl` is set.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Raise (never lower) a kernel's dynamic shared-memory limit to `bytes`.  The limit is an
// attribute of the function, shared by every context of the process, so a context that
// needs less must not lower it beneath another context's launches (contexts of different
// restart lengths alive at once: the server's norm estimates beside its graph lanes, two
// solvers, two batches).  One process-wide lock orders the read and the write.
// (The default limit is 48 KiB less the kernel's static shared memory, so the comparison is
// with the kernel's current attribute, not with 48 KiB.)
inline cudaError_t raise_smem_limit(const void *fn, size_t bytes)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Double-float split of an FP64 value (the IGS_PREC_FP64_DF form, igs_df.cu; also used by the
// SpMV when it writes a split copy of its output).
// a = hi + lo + r, |r| <= 2^-47 |a| for 2^-100 <= |a| < 2^127 (integer and FP32 operations
// only, none on the narrow FP64 pipe: the remaining 29 bits are rounded to 23 and turned
// into a float exactly by placing them in the mantissa of 2^23 and subtracting 2^23; two
// power-of-two scalings follow, exact unless lo is subnormal).
__device__ __forceinline__ void df_split(double a, float &hi, float &lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sign = hw & 0x80000000u, ahw = hw & 0x7fffffffu;
    // (hw:lw) << 3 puts the top 23 fraction bits in bits 22..0 and the low 9 exponent bits
    // in bits 31..23; subtracting 384 << 23 turns FP64's exponent bias (1023) into FP32's
    // (127) for every exponent of the FP32 normal range.
    unsigned hb = (__funnelshift_l(lw, hw, 3) - 0xC0000000u) | sign;
    hb = ahw < (897u << 20) ? sign : hb;                                // |a| < 2^-126: 0
    hb = ahw >= (1150u << 20) ? (sign | 0x7f800000u) : hb;             // |a| >= 2^127: inf
    hi = __uint_as_float(hb);
    // the remaining 29 fraction bits times 2^(e - 1075) = rem * 2^-52 * (+-2^(e - 1023)),
    // with rem rounded to a multiple of 64: ((rem + 32) >> 6) * 2^-46 * (+-2^(e - 1023))
    const float scale = __uint_as_float(hb & 0xff800000u);
    const unsigned r23 = ((lw & 0x1fffffffu) + 32u) >> 6;  // <= 2^23
    const float fr = __fsub_rn(__uint_as_float(0x4B000000u | r23), 8388608.0f);
    lo = __fmul_rn(__fmul_rn(fr, 0x1p-46f), scale);
}

// Scalars of one solve, kept in device memory so that no step needs the host.
struct DevState {
    double rho;        // ||r0|| of the current cycle
    double inv_rho;
    double inv_gamma;  // 1 / gamma of the current step
    double stop_den;   // ||b|| + ||A||_2 ||x0|| (in-cycle stop test denominator)
    double tol;        // tol_beta
    double normA;      // ||A||_2
    double bnorm;      // ||b||
    double rnorm, xnorm, beta;  // end-of-cycle residual norm, ||x||, backward error
    double inner_tol;  // FP32 cycles of the precision form: stop when |g| <= inner_tol * rho
    double stop_floor; // inner_tol * rho of the current cycle (0 for FP64 solves)
    double lag_g2;     // Alg. 4.2: gamma^2 of the last step (its column's breakdown test)
    int halt;          // nonzero: the remaining step kernels of this cycle do nothing
    int stop_cols;     // > 0: columns the cycle ends with (early stop or breakdown)
    int stop_reason;   // 0 running, 1 converged, 2 breakdown, -4 numeric error
    int ncols;         // columns used by the least-squares solve of this cycle
    int neumann_terms; // terms used by the last (I+L) application (0: substitution)
    int pad[3];
};

// Device memory of one context.
struct Workspace {
    int64_t n = 0, ld = 0, nnz = 0;
    int mmax = 0;
    int num_sms = 0;
    bool spmv_warp_rows = false;   // warp-per-row SpMV (long rows) instead of thread-per-row
    bool pdl = true;               // programmatic dependent launch of the single-block steps
    const int *rowptr = nullptr, *colind = nullptr;
    const double *val = nullptr;
    double *V = nullptr;           // ld x (mmax+1), column-major
    double *z = nullptr, *u = nullptr, *r = nullptr, *b = nullptr, *x = nullptr, *t = nullptr;
    double *H = nullptr;           // (mmax+1) x mmax column-major, ldh = mmax+1
    double *L = nullptr;           // (mmax+1) x (mmax+1) column-major: L(i,c) at L[c*ldl + i]
    double *Lrow = nullptr;        // the same, row-packed: L(i,c) at Lrow[i(i-1)/2 + c]
    double *Lout = nullptr;        // (mmax+1)^2 staging for the row-major copy handed out
    double *R = nullptr;           // Givens-rotated copy of H, same layout as H
    double *cs = nullptr, *sn = nullptr, *g = nullptr;  // rotations and rotated rhs
    double *lfro2 = nullptr;       // cumulative ||L rows 0..i||_F^2, mmax+1 entries
    double *r1v = nullptr, *r2v = nullptr, *r3v = nullptr, *y = nullptr;
    double *part = nullptr;        // per-block partial sums
    int64_t part_cap = 0;
    double *hist_res = nullptr, *hist_lfro = nullptr;  // per-cycle history (mmax entries)
    DevState *st = nullptr;
    // precision form (allocated when the context is created with an FP32 basis)
    float *V32 = nullptr;          // ld x (mmax+1), column-major, zero padding rows
    float *z32 = nullptr, *u32 = nullptr;
    float *val32 = nullptr;        // A's values rounded to FP32 (same rowptr / colind)
    // SELL-32 copy of A for the short-row FP64 SpMV: slices of 32 rows, each as wide as its
    // longest row; entry k of row r at sell_off[r/32] + 32k + r%32 (CSR order, padding -1)
    const int64_t *sell_off = nullptr;
    const int *sell_col = nullptr;
    const double *sell_val = nullptr;
    // > 0: every slice of the SELL-32 copy is this many entries wide (ELL; offset of slice k
    // = 32 * ell_width * k, sell_off unused by the SpMV), 1..kMaxEllWidth
    int ell_width = 0;
    int ldh() const { return mmax + 1; }
    int ldl() const { return mmax + 1; }
};

// Launch geometry of the multi-dot kernel for p columns.
struct DotsPlan {
    int groups;      // column groups (grid.y)
    int rblocks;     // row blocks (grid.x)
    int64_t rows;    // rows per row block (multiple of 4)
};
DotsPlan plan_dots(const Workspace &w, int p);
// The same plan for a grid of at most `slots` blocks (groups x row blocks).
DotsPlan plan_dots_slots(const Workspace &w, int p, int slots);

// Kernel classes (match IGS_KCLASS_* in igs.h).
enum KClass { KC_SPMV = 0, KC_DOTS = 1, KC_UPDATE = 2, KC_SMALL = 3, KC_CYCLE = 4 };

// ---- launchers (enqueue on `s`; return cudaGetLastError()) ----
// y = A x, or y = b - A x when b != nullptr.
// With y_df, also its split copy (the double-float form).
cudaError_t launch_spmv(const Workspace &w, const double *x, double *y, const double *b,
                        bool check_halt, cudaStream_t s, float2 *y_df = nullptr);
// Partial sums part[rb*(nq*p) + q*p + c] = sum over row block rb of V[:,c] . X_q, q < nq.
cudaError_t launch_dots(const Workspace &w, int p, const double *x0, const double *x1,
                        bool check_halt, cudaStream_t s, DotsPlan *plan_out);
// out = alpha*src - V[:, 0:p] coef (coef negated when neg_coef); when norm_last, column p-1
// of V is first scaled in place by st->inv_gamma and alpha is taken as st->inv_gamma.
// When p_from_state, p = st->ncols.
cudaError_t launch_update(const Workspace &w, int p, const double *coef, bool neg_coef,
                          double alpha, const double *src, double *out, bool norm_last,
                          bool p_from_state, bool check_halt, cudaStream_t s);
// Double-float block multi-dot (igs_df.cu), same partial layout and plan as launch_dots;
// used by the IGS_PREC_FP64_DF form for n >= kDfMinRows (dots_df_applies).
constexpr int64_t kDfMinRows = 16384;
bool dots_df_applies(const Workspace &w);
cudaError_t launch_dots_df(const Workspace &w, int p, const double *x0, const double *x1,
                           bool check_halt, cudaStream_t s, DotsPlan *plan_out);
// Dynamic shared-memory limits of the double-float kernels (once per context, before capture).
cudaError_t configure_df_kernels();
// Double-float basis update of the same form (steps 7, 11, 13, 16; out = a src - V coef, with
// column p-1 normalised in place first when norm_last, a = st->inv_gamma then).
cudaError_t launch_update_df(const Workspace &w, int p, const double *coef, double alpha, const double *src,
                             double *out, bool norm_last, cudaStream_t s);
// The split basis (vdf: each basis element stored as its FP32 (hi, lo) pair in V's bytes) of
// the double-float Alg. 4.1 cycle.  Update: also out_df = split(out) when given; with
// norm_last and vdf the FP64 w comes from wsrc and split(w * inv_gamma) goes to column p-1;
// neg_coef and p_from_state as in launch_update.  Multi-dot: vdf reads V, x0 and x1 split.
cudaError_t launch_update_df_ex(const Workspace &w, int p, const double *coef, bool neg_coef, double alpha,
                                const double *src, double *out, float2 *out_df, const double *wsrc, bool norm_last,
                                bool p_from_state, bool vdf, cudaStream_t s);
cudaError_t launch_dots_df_ex(const Workspace &w, int p, const double *x0, const double *x1, bool check_halt,
                              bool vdf, cudaStream_t s, DotsPlan *plan_out);
// dst_df = split(src * st->inv_rho (which 0) or st->inv_gamma (which 1)), dst64 (nullable) the
// same in FP64.
cudaError_t launch_scale_df(const Workspace &w, const double *src, float2 *dst_df, double *dst64, int which,
                            bool check_halt, cudaStream_t s);
// Alg. 4.2's fused update on the split basis (v_{k-1} split into column nb; unless vonly, the
// next u in FP64 into wu, which holds u on entry, and split into column nb+1).
cudaError_t launch_update_1r_df(const Workspace &w, int nb, const double *z, double *wu, bool vonly,
                                cudaStream_t s);
// x += V y over the split basis in FP64 (p = st->ncols).
cudaError_t launch_xupdate_vdf(const Workspace &w, cudaStream_t s);
// In place: count split elements of V back to FP64.
cudaError_t launch_df_to_f64(double *V, int64_t count, int num_sms, cudaStream_t s);
// Partial sums of squares of up to three vectors (part[blk*nvec + q]).
cudaError_t launch_norms(const Workspace &w, const double *a, const double *b,
                         const double *c, int *blocks_out, cudaStream_t s);
// v = scale * w with scale = st->inv_rho (which=0) or st->inv_gamma (which=1).
cudaError_t launch_scale(const Workspace &w, const double *src, double *dst, int which,
                         bool check_halt, cudaStream_t s);

// Small single-block steps.
cudaError_t launch_cycle_start(const Workspace &w, int nblk, cudaStream_t s);
cudaError_t launch_prime(const Workspace &w, const DotsPlan &pl, cudaStream_t s);
cudaError_t launch_step_a(const Workspace &w, int k, int gs, const DotsPlan &pl, cudaStream_t s);
cudaError_t launch_step_b(const Workspace &w, int k, const DotsPlan &pl, cudaStream_t s);
cudaError_t launch_flush(const Workspace &w, int m, const DotsPlan &pl, cudaStream_t s);
cudaError_t launch_givens(const Workspace &w, int j, cudaStream_t s);
// Alg. 4.2 (one-reduce): the single-block step (nb normalised columns; flush: completion of
// the last column only) and the fused basis update (v and the next u in one pass).
cudaError_t launch_step_1r(const Workspace &w, int nb, bool flush, const DotsPlan &pl, cudaStream_t s);
cudaError_t launch_update_1r(const Workspace &w, int nb, const double *z, bool vonly, cudaStream_t s);
cudaError_t launch_lsq(const Workspace &w, int m, cudaStream_t s);
cudaError_t launch_beta(const Workspace &w, int nblk, cudaStream_t s);
cudaError_t launch_init_state(const Workspace &w, double tol, double normA, double inner_tol,
                              cudaStream_t s);
cudaError_t launch_bnorm(const Workspace &w, int nblk, cudaStream_t s);

// dst(i, c) = src(i, c) for i < rows, c < cols: src column-major (ld_src), dst row-major
// (ld_dst).
cudaError_t launch_transpose(const double *src, int ld_src, int rows, int cols, double *dst,
                             int ld_dst, cudaStream_t s);

// FP32-basis kernels of the precision form (igs_fp32.cu).  Same grids and FP64 partial-sum
// layout as the FP64 kernels; all return cudaGetLastError().
cudaError_t launch_spmv32(const Workspace &w, const float *x, float *y, cudaStream_t s);
cudaError_t launch_dots32(const Workspace &w, int p, const float *x0, const float *x1, cudaStream_t s,
                          DotsPlan *plan_out);
cudaError_t launch_update32(const Workspace &w, int p, const double *coef, double alpha, const float *src,
                            float *out, bool norm_last, cudaStream_t s);
cudaError_t launch_scale_to32(const Workspace &w, const double *src, float *dst, cudaStream_t s);
cudaError_t launch_scale32(const Workspace &w, float *v, cudaStream_t s);
cudaError_t launch_xupdate32(const Workspace &w, cudaStream_t s);

// Per-context kernel configuration (dynamic shared-memory limits); call before any capture.
cudaError_t configure_kernels(const Workspace &w);

// ||A||_2 estimate: power iteration on A^T A (At in CSR = A^T).
cudaError_t estimate_norm2(const Workspace &w, const int *at_rowptr, const int *at_colind,
                           const double *at_val, int iters, double *out, cudaStream_t s);

}  // namespace igs
