// k-truncated Arnoldi with on-the-fly sketching (Algorithm 2, Sec. 2.2), with
// the basis stored in FP32 or BF16, the matrix values in FP32, and the SpMV and
// the orthogonalisation in FP32 arithmetic.  The sketches S v_j and S A v_j,
// the Hessenberg coefficients and everything after the Arnoldi loop stay FP64.
//
// Storage as in the FP64 variant: column j of V holds w_j (a positive multiple
// of v_j, sigma_j = 1/||w_j||), rounded to the storage type; every quantity is
// computed from the stored (rounded) vectors, so that SV = S V_m and
// SAV = S A V_m hold for the basis the caller receives.
//
// Rows are dealt out in chunks of kChunkRows, chunk c to CTA c mod G (G = SMs,
// one 1024-thread CTA per SM), in every kernel: all CTAs sweep the rows
// together, so the stencil gathers of the SpMV stay within a few MB of L2, and
// every kernel's fixed-point sketch partials share one bin-load bound.
//
// Two kernels per step:
//   spmv   (step j): S w_{j-1} and S A v_{j-2} from the previous partials
//                    (prologue); y_j = A w_j -> Y; partial <w_i, y_j> for the
//                    window and max|y_j|.  For slices at most 8 wide the loads
//                    are software-pipelined across chunks.
//   update (step j): MGS coefficients from the dots and the window Gram
//                    matrix; w_{j+1} = sigma_j y_j - sum_i h_ij sigma_i w_i in
//                    FP32, rounded and stored; ||w_{j+1}||^2, Gram entries,
//                    max|w_{j+1}|; exact two-limb fixed-point sketch of the
//                    stored w_j (its maximum is known), in per-lane copies of
//                    the shared-memory bins so that a warp's atomics do not
//                    collide.
// S y_j is not scattered: the update step is the Arnoldi relation
//   sigma_j y_j = w_{j+1} + sum_i h_ij sigma_i w_i     (FP32 coefficients),
// so S y_j follows from the sketches of stored vectors once S w_{j+1} is
// known.  Each S y_j uses only directly sketched columns, so no error is
// carried from one column to the next; what is left out is the FP32 rounding
// of that one update (about (k+1) u_32 ||sigma_j y_j||).  With BF16 storage the
// rounding residual bf16(w_{j+1}) - w_{j+1}, exact in FP32, is sketched with
// one fixed-point limb and taken off.  The last column S y_{m-1} is scattered
// directly, with the a-priori scale ||A||_inf max|w_{m-1}| (its maximum is not
// known before the SpMV ends).
#pragma once

#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "skf_internal.cuh"
#include "skf_step.cuh"

namespace skf {
namespace lp {
namespace {   // internal linkage: each instantiating translation unit has its own copy

constexpr int kP1 = kMaxK + 1;             // slots of one spmv partial: d[kMaxK], ymax
constexpr int kP2 = kMaxK + 2;             // slots of one update partial: ||w||^2, max|w|, g[kMaxK]
constexpr int kSpmvThreads = kChunkRows;   // one row per thread and chunk; one CTA per SM
constexpr int kUpdThreads = kChunkRows;    // one row per thread and chunk; one CTA per SM
constexpr int kCoef = kMaxK + 1;           // per step: sigma_j, then h_ij sigma_i of the window (FP32 values)
// Happy breakdown in FP32 arithmetic: ||w_{j+1}|| <= 2^-17 ||A v_j|| (64 FP32
// unit roundoffs; below that w_{j+1} is rounding noise).
constexpr double kBreakTol = 7.62939453125e-06;

template <typename TB> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float rnd(float x) { return x; }
    static __device__ __forceinline__ void st(float *p, float x) { *p = x; }
    static constexpr bool kExact = true;   // FP32 values are stored as computed
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float rnd(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
    static constexpr bool kExact = false;
};

// Round x 2^shift to the nearest integer (ties away from zero), with integer
// instructions only.  Requires |x| 2^shift < 2^62.
__device__ __forceinline__ long long fixed_point_f32(float x, int shift) {
    const unsigned bits = __float_as_uint(x);
    const int e = (int)((bits >> 23) & 0xFFu);
    if (e == 0) return 0;   // zero or subnormal: far below any quantum used here
    const unsigned long long mant = (unsigned long long)((bits & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 150 + shift;   // x 2^shift = mant 2^sh
    unsigned long long v;
    if (sh >= 0) {
        v = mant << sh;
    } else if (sh > -64) {
        const int r = -sh;
        v = (mant >> r) + ((mant >> (r - 1)) & 1ull);
    } else {
        v = 0;
    }
    return (bits >> 31) ? -(long long)v : (long long)v;
}

__device__ __forceinline__ unsigned abs_key_f32(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }

// The two limbs (l0, l1) of round(x 2^shift) = l1 2^L + l0, from FP32
// operations on |x|: t = |x| 2^(shift - L) (exact scaling), l1 = floor(t), and
// l0 = rint((t - l1) 2^L) (the fractional part of a non-negative float is
// exact); both limbs carry the sign of x.  0 <= |l0| <= 2^L, which keeps the
// bin sums within the limb-width rule.  Requires |x| 2^shift < 2^(2L).  The
// scales come from LimbScale, set once per kernel.
struct LimbScale {
    float hi, lo;   // 2^(shift - L) (0 if outside the float range), 2^L
    int k;          // shift - L
    __device__ __forceinline__ LimbScale(int shift, int L) {
        k = shift - L;
        hi = (k >= -126 && k <= 127) ? __int_as_float((127 + k) << 23) : 0.f;
        lo = __int_as_float((127 + L) << 23);
    }
};
__device__ __forceinline__ void limbs_f32(float x, const LimbScale &ls, int &l0, int &l1) {
    const float t = ls.hi != 0.f ? fabsf(x) * ls.hi : ldexpf(fabsf(x), ls.k);
    const float fl = floorf(t);
    const int h = __float2int_rz(fl);
    const int lo = __float2int_rn((t - fl) * ls.lo);
    const bool ng = x < 0.f;
    l1 = ng ? -h : h;
    l0 = ng ? -lo : lo;
}

struct LpCtx {
    RowSplit rs;               // long rows of a skewed operator (row split)
    float *seg_part;           // [rs.nseg] partial sums of the long rows' segments
    int64_t n;
    const int64_t *sell_off;   // SELL-32 operator with FP32 values (see skf_csr)
    const int32_t *sell_w;
    const float *sell_val;
    const int32_t *sell_col;
    double norm_inf;           // ||A||_inf
    SparseSign sp;
    const uint16_t *pattern;   // 16-bit sparse-sign pattern
    const uint8_t *pattern8;   // compact pattern (zeta <= 8, stripes <= 128 rows) or nullptr
    int p8_block;              // its sign offset: 64 or 128
    const int *binmax_chunk;   // bin-load maximum of the chunk partition
    int identity;              // S = I
    int split;                 // update bins laid out [stripe][sign][p8_block] (compact pattern, zeta = 8)
    int m, k;
    void *V;                   // TB [m][ldv] (or [vring][ldv], see vcol)
    int64_t ldv;
    int vring;                 // 0: all m columns stored; > 0: ring of vring slots (two-pass)
    int64_t woff[kMaxK];       // element offsets of the window columns i0 .. j of this launch's step
                               // (filled on the host per launch, so no kernel computes ring slots)
    double *vscale, *SV, *SAV, *H;
    float *Y;                  // [n] y_j = A w_j
    double *p1;                // [G][kP1]
    double *p2;                // [G][kP2]
    double *fin_d;             // [m][kP1] reduced dots of step j, max|y_j|
    double *fin_w;             // [m+1][2] ||w_j||^2, max|w_j|
    double *stepsc;            // [m+1][4] 1/||w_j||, ||w_j||, stop flag
    double *gram;              // [m+1][kMaxK] <w_j, w_{j-d}>
    double *coef;              // [m][kCoef] the FP32 coefficients update j applied
    double *skw;               // [m][s] S w_j in units of the +-1 pattern
    double *sd;                // [s] S (residual of w_j), BF16 storage only
    long long *skWp;           // [2][G][s] fixed-point partials of S w_j, by parity of j
    long long *skYp;           // [G][s] fixed-point partials of S y_{m-1}
    long long *skDp;           // [G][s] fixed-point partials of the BF16 residual of w_{j+1}
    int *ex;                   // exponents: [0, m) S w_j, [m, 2m) residual of w_j, [2m] S y_{m-1}
    double *epscol;            // [m]
    double inv_sqrt_zeta;
    unsigned *cnt;             // [2] arrival tickets
    int *iscal;                // [0] stopped, [1] m_eff, [2] status, [3] step that stopped
    int G;                     // CTAs of every kernel (chunk partition)
    int lc;                    // log2 of the per-lane bin copies of the update kernel
};

// (row of S, sign) of the zeta nonzeros of column r, from the compact or the
// 16-bit pattern table.
template <int ZCAP>
__device__ __forceinline__ void pattern_row(const LpCtx &c, int64_t r, int (&row)[ZCAP], bool (&neg)[ZCAP]) {
    if (ZCAP == 8 && c.pattern8 != nullptr) {
        const uint2 v = __ldg((const uint2 *)(c.pattern8 + r * 8));
#pragma unroll
        for (int q = 0; q < ZCAP; ++q) {
            const int e = (int)(((q < 4 ? v.x : v.y) >> (8 * (q & 3))) & 0xFFu);
            neg[q] = e >= c.p8_block;
            row[q] = c.sp.start[q] + (neg[q] ? e - c.p8_block : e);
        }
    } else {
        uint16_t e[ZCAP];
        load_pattern<ZCAP>(c.pattern, c.sp.zeta, r, e);
#pragma unroll
        for (int q = 0; q < ZCAP; ++q) pattern_entry(c.sp, e[q], q, row[q], neg[q]);
    }
}

// Chunk-partition row of thread `threadIdx.x` (< kChunkRows) in the i-th
// chunk of this CTA, or -1; and the number of chunks of this CTA.
__device__ __forceinline__ int64_t chunk_row(const LpCtx &c, int64_t i) {
    const int64_t r = ((int64_t)blockIdx.x + i * c.G) * kChunkRows + threadIdx.x;
    return r < c.n ? r : -1;
}
__device__ __forceinline__ int64_t chunks_of_cta(const LpCtx &c) {
    const int64_t nch = (c.n + kChunkRows - 1) / kChunkRows;
    return blockIdx.x < nch ? (nch - blockIdx.x + c.G - 1) / c.G : 0;
}

template <typename TB>
__global__ void __launch_bounds__(kChunkRows) k_arnoldi_init_lp(LpCtx c, const double *__restrict__ b) {
    __shared__ double red[64];
    TB *V = (TB *)c.V;
    double nrm[1] = {0.0};
    double mx = 0.0;
    const int64_t nc = chunks_of_cta(c);
    for (int64_t i = 0; i < nc; ++i) {
        const int64_t r = chunk_row(c, i);
        if (r < 0) continue;
        const float x = Store<TB>::rnd((float)b[r]);   // b rounded to FP32, then to the storage type
        Store<TB>::st(V + r, x);
        nrm[0] = fma((double)x, (double)x, nrm[0]);
        mx = fmax(mx, fabs((double)x));
    }
    block_sum<1, kChunkRows>(nrm, red);
    mx = block_max<kChunkRows>(mx, red);
    if (threadIdx.x == 0) {
        c.p2[(size_t)blockIdx.x * kP2 + 0] = nrm[0];
        c.p2[(size_t)blockIdx.x * kP2 + 1] = mx;
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < (c.m + 1) * c.m; i += kChunkRows) c.H[i] = 0.0;
        if (threadIdx.x == 0) {
            c.iscal[0] = 0;
            c.iscal[1] = c.m;
            c.iscal[2] = SKF_OK;
            c.iscal[3] = c.m;
        }
    }
    if (last_to_arrive(c.cnt + 1)) {
        const int warp = threadIdx.x >> 5;
        if (warp < 2) {
            const double v = warp_reduce_partials(c.p2 + warp, gridDim.x, kP2, warp == 1);
            if ((threadIdx.x & 31) == 0) c.fin_w[warp] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double n2 = c.fin_w[0];
            const double hn = sqrt(n2);
            c.stepsc[0] = n2 > 0.0 ? 1.0 / hn : 0.0;
            c.stepsc[1] = hn;
            c.stepsc[2] = n2 > 0.0 ? 0.0 : 1.0;   // zero right-hand side
            c.cnt[1] = 0u;
        }
    }
}

// S w_jw from the partials of the update kernel (or of a stopping SpMV) for
// this CTA's slice of the rows of S; with `store`, skw and SV[:, jw].  Then,
// for jw >= 1, S y_{jw-1} from the Arnoldi relation of update jw - 1:
//   sigma_{jw-1} y_{jw-1} = (w_jw - residual_jw) + sum_i cf_i w_i,
// SAV[:, jw-1] = sigma_{jw-1} S y_{jw-1} / sqrt(zeta).  With `next_resid`
// (BF16 storage, called from SpMV jw + 1), sd <- S residual_{jw+1} afterwards.
// With `ylast`, SAV[:, jw] from the directly scattered S y_jw.
template <typename TB>
__device__ __forceinline__ void finalize_column(const LpCtx &c, int jw, bool store, bool next_resid, bool ylast) {
    const int s = c.sp.s;
    const int G = gridDim.x;
    const int L = limb_bits(*c.binmax_chunk);
    const int P = sketch_fraction_bits_from_limb(L);
    const int ew = c.ex[jw];
    const int ey = c.ex[2 * c.m];
    const int edn = next_resid ? c.ex[c.m + jw + 1] : kNoExp;
    const double sig = c.stepsc[4 * (size_t)jw];
    const int jm = jw - 1;
    const int i0 = max(0, jm - c.k + 1);
    const int nw = jm - i0 + 1;
    const double *cf = c.coef + (size_t)max(jm, 0) * kCoef;
    const double sig_m = jw >= 1 ? c.stepsc[4 * (size_t)jm] : 0.0;
    const long long *wp = c.skWp + (size_t)(jw & 1) * c.G * s;
    const int per = (s + G - 1) / G;
    const int b0 = blockIdx.x * per, b1 = min(s, b0 + per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = b0 + warp; i < b1; i += blockDim.x / 32) {
        double sw = 0.0;
        if (ew != kNoExp) sw = scale_pow2(warp_sum_i64_exact(wp + i, c.G, (size_t)s), ew - P);
        double sy = 0.0;
        if (ylast && ey != kNoExp) sy = scale_pow2(warp_sum_i64_exact(c.skYp + i, c.G, (size_t)s), ey - P);
        double sdn = 0.0;
        if (next_resid && edn != kNoExp) sdn = scale_pow2(warp_sum_i64_exact(c.skDp + i, c.G, (size_t)s), edn - L);
        if (lane == 0) {
            if (store) {
                c.skw[(size_t)jw * s + i] = sw;
                c.SV[i + (size_t)jw * s] = sig * sw * c.inv_sqrt_zeta;
            }
            if (jw >= 1) {
                double u = sw - (Store<TB>::kExact ? 0.0 : c.sd[i]);
                for (int a = 0; a < nw; ++a) u += cf[1 + a] * c.skw[(size_t)(i0 + a) * s + i];
                c.SAV[i + (size_t)jm * s] = (u / cf[0]) * sig_m * c.inv_sqrt_zeta;
            }
            if (next_resid) c.sd[i] = sdn;
            if (ylast) c.SAV[i + (size_t)jw * s] = sig * sy * c.inv_sqrt_zeta;
        }
    }
}

// Fixed-point sketch of one value into two-limb bins [2][s], signs selected.
template <int ZCAP>
__device__ __forceinline__ void scatter2(const LpCtx &c, int64_t r, long long v, int L, int *a0, int *a1) {
    int row[ZCAP];
    bool neg[ZCAP];
    pattern_row<ZCAP>(c, r, row, neg);
    const int l0 = (int)(v & ((1ll << L) - 1)), l1 = (int)(v >> L);
#pragma unroll
    for (int q = 0; q < ZCAP; ++q)
        if (q < c.sp.zeta) red_limbs(a0, a1, row[q], l0, l1, neg[q]);
}

// Common start of the SpMV kernels: stop test, H subdiagonal, finalisation of
// the previous column's sketches.  Returns false when nothing more is to be
// done by this launch (stopped earlier, zero right-hand side, or S = I at a
// stop); `stopping` = m_eff is j.
template <typename TB>
__device__ __forceinline__ bool spmv_begin(const LpCtx &c, int j, bool &stopping) {
    if (c.iscal[0] && c.iscal[3] < j) return false;   // stopped at an earlier step
    const double *sc_j = c.stepsc + 4 * (size_t)j;
    // h_{j,j-1} of the relation the stored basis satisfies: update j - 1 formed
    // w_j = sigf y_{j-1} - ... with sigf = cf[0], the FP32 value of sigma_{j-1},
    // so A v_{j-1} = sigma_{j-1} y_{j-1} has the coefficient
    // sigma_{j-1} ||w_j|| / sigf on v_j = w_j / ||w_j|| (||w_j|| up to one FP32
    // rounding of sigma_{j-1})
    if (j >= 1 && blockIdx.x == 0 && threadIdx.x == 0)
        c.H[j + (size_t)(j - 1) * (c.m + 1)] =
            c.stepsc[4 * (size_t)(j - 1)] * sc_j[1] / c.coef[(size_t)(j - 1) * kCoef];
    // zero right-hand side (j = 0) or happy breakdown, decided by the previous
    // launch: m_eff = j.  S w_j is still formed (S y_{j-1} needs it).
    stopping = sc_j[2] != 0.0;
    if (stopping && blockIdx.x == 0 && threadIdx.x == 0) {
        c.iscal[0] = 1;
        c.iscal[1] = j;
        c.iscal[3] = j;
        if (j == 0) c.iscal[2] = SKF_ERR_ZERO_RHS;
    }
    if (stopping && (j == 0 || c.identity)) return false;
    if (!c.identity && j >= 1) finalize_column<TB>(c, j - 1, true, !Store<TB>::kExact, false);
    return true;
}

// At a stop (j >= 1, S sparse): S w_j into the partials of parity j & 1.
// bins: [2 s] ints of shared memory.
template <int ZCAP, typename TB>
__device__ __forceinline__ void spmv_stop_sketch(const LpCtx &c, int j, int *bins) {
    const int s = c.sp.s;
    const int L = limb_bits(*c.binmax_chunk);
    const int P = sketch_fraction_bits_from_limb(L);
    const TB *wj = (const TB *)c.V + vcol(c, j);
    const double wmax = c.fin_w[2 * (size_t)j + 1];
    const int ew = positive_finite(wmax) ? bound_exponent(wmax) : kNoExp;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.ex[j] = ew;
    for (int i = threadIdx.x; i < 2 * s; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    const int64_t nc = chunks_of_cta(c);
    for (int64_t i = 0; i < nc; ++i) {
        const int64_t r = chunk_row(c, i);
        if (r >= 0 && ew != kNoExp)
            scatter2<ZCAP>(c, r, fixed_point_f32(Store<TB>::ld(wj + r), P - ew), L, bins, bins + s);
    }
    __syncthreads();
    long long *ow = c.skWp + ((size_t)(j & 1) * c.G + blockIdx.x) * s;
    for (int i = threadIdx.x; i < s; i += blockDim.x) ow[i] = combine_limbs(bins[i], bins[s + i], L);
}

// Common end: sketch partials of S y_{m-1} (last step), dot/max partials and
// the last-arriving CTA's fixed-order reduction.
template <int KW>
__device__ __forceinline__ void spmv_end(const LpCtx &c, int j, int nw, bool last, int L, const int *ybins,
                                         float (&acc)[KW], unsigned ykey, double *red) {
    const int s = c.sp.s;
    if (last) {
        __syncthreads();
        long long *oy = c.skYp + (size_t)blockIdx.x * s;
        for (int i = threadIdx.x; i < s; i += kSpmvThreads) oy[i] = combine_limbs(ybins[i], ybins[s + i], L);
    }
    double accd[KW];
#pragma unroll
    for (int a = 0; a < KW; ++a) accd[a] = (double)acc[a];
    block_sum<KW, kSpmvThreads>(accd, red);
    const unsigned ymk = (unsigned)block_max_key<kSpmvThreads>((unsigned long long)ykey, (unsigned long long *)red);
    if (threadIdx.x == 0) {
        double *o = c.p1 + (size_t)blockIdx.x * kP1;
        for (int a = 0; a < KW; ++a) o[a] = accd[a];
        o[kP1 - 1] = (double)__uint_as_float(ymk);
    }
    if (last_to_arrive(c.cnt)) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int v = warp; v <= nw; v += kSpmvThreads / 32) {
            const int slot = (v < nw) ? v : kP1 - 1;
            const double rr = warp_reduce_partials(c.p1 + slot, gridDim.x, kP1, slot == kP1 - 1);
            if (lane == 0) c.fin_d[(size_t)j * kP1 + slot] = rr;
        }
        if (threadIdx.x == 0) c.cnt[0] = 0u;
    }
}

// Scale of the directly scattered S y_{m-1}: |y_r| <= ||A||_inf max|w_{m-1}|.
__device__ __forceinline__ int last_y_exponent(const LpCtx &c, int j) {
    const double ybound = c.norm_inf * c.fin_w[2 * (size_t)j + 1] * (1.0 + 1.0 / 1024.0);   // FP32 row-sum margin
    const int ey = positive_finite(ybound) ? bound_exponent(ybound) : kNoExp;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.ex[2 * c.m] = ey;
    return ey;
}

// Row split: one warp per segment of a long row, FP32 products and sums
// (lane-strided, then a butterfly whose lane-0 result is the partial).
template <typename TB>
__global__ void __launch_bounds__(256) k_spmv_long_lp(LpCtx c, int j) {
    asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent (see k_arnoldi_spmv_lp)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (c.iscal[0] && c.iscal[3] < j) return;
    const TB *x = (const TB *)c.V + vcol(c, j);
    const float *vals = (const float *)c.rs.values;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < c.rs.nseg; g += nwarps) {
        const int b = __ldg(c.rs.seg_beg + g), e = __ldg(c.rs.seg_end + g);
        float acc = 0.f;
        for (int p = b + lane; p < e; p += 32) acc = fmaf(__ldg(vals + p), Store<TB>::ld(x + __ldg(c.rs.colind + p)), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) c.seg_part[g] = acc;
    }
}

// SpMV with the SELL values and columns loaded per row (any slice width).
template <int KW, int ZCAP, typename TB>
__global__ void __launch_bounds__(kSpmvThreads, 1) k_arnoldi_spmv_lp(LpCtx c, int j) {
    extern __shared__ int bins[];   // [2 s]: limbs of S w_j (stopping step) or of S y_{m-1} (last step)
    __shared__ double red[32 * KW];
    // programmatic dependent of the previous launch: every CTA waits for it
    // in full before reading anything (and before any exit), then releases
    // the next launch so that its CTAs are placed while this one runs
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool stopping;
    if (!spmv_begin<TB>(c, j, stopping)) return;
    if (stopping) {
        spmv_stop_sketch<ZCAP, TB>(c, j, bins);
        return;
    }
    const int s = c.sp.s;
    const TB *V = (const TB *)c.V;
    const TB *wj = V + vcol(c, j);
    const int L = c.identity ? 0 : limb_bits(*c.binmax_chunk);
    const int P = sketch_fraction_bits_from_limb(L);
    const bool last = (j == c.m - 1) && !c.identity;
    const int ey = last ? last_y_exponent(c, j) : kNoExp;
    if (last)
        for (int i2 = threadIdx.x; i2 < 2 * s; i2 += kSpmvThreads) bins[i2] = 0;
    __syncthreads();
    const int shift_y = P - (ey == kNoExp ? 0 : ey);
    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;
    float acc[KW];
#pragma unroll
    for (int a = 0; a < KW; ++a) acc[a] = 0.f;
    unsigned ykey = 0;
    const int lane = threadIdx.x & 31;
    const int64_t nc = chunks_of_cta(c);
    for (int64_t i = 0; i < nc; ++i) {
        const int64_t rw = ((int64_t)blockIdx.x + i * c.G) * kChunkRows + (threadIdx.x & ~31);   // warp's slice
        if (rw >= c.n) continue;                                                                // whole warp
        int wt = 0;
        long long so = 0;
        uint2 sl = make_uint2(0u, 0u);
        if (lane == 0) {
            wt = __ldg(c.sell_w + (rw >> 5));
            so = __ldg(c.sell_off + (rw >> 5));
            if (c.rs.sell_long) sl = __ldg(c.rs.sell_long + (rw >> 5));
        }
        wt = __shfl_sync(0xffffffffu, wt, 0);
        so = __shfl_sync(0xffffffffu, so, 0);
        sl.x = __shfl_sync(0xffffffffu, sl.x, 0);
        sl.y = __shfl_sync(0xffffffffu, sl.y, 0);
        if (rw + lane >= c.n) continue;   // no warp-collective operation below
        const int64_t r = c.rs.perm ? (int64_t)__ldg(c.rs.perm + rw + lane) : rw + lane;   // the lane's row
        // window values first: independent of the SpMV, their latency overlaps it
        float wv[KW];
#pragma unroll
        for (int a = 0; a < KW; ++a) wv[a] = a < nw ? Store<TB>::ld(V + c.woff[a] + r) : 0.f;
        const float *pv = c.sell_val + so + lane;   // entry p at pv[32 p]
        const int32_t *pc = c.sell_col + so + lane;
        float y = 0.f;
        // eight entries of the row in flight at a time
        for (int p0 = 0; p0 < wt; p0 += 8) {
            float av[8], xv[8];
            int cv[8];
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p0 + p < wt) {
                    av[p] = __ldcs(pv + 32 * (p0 + p));
                    cv[p] = __ldcs(pc + 32 * (p0 + p));
                }
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p0 + p < wt) xv[p] = Store<TB>::ld(wj + cv[p]);
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p0 + p < wt) y = fmaf(av[p], xv[p], y);
        }
        if (sl.x) y = add_long_row(c.rs, c.seg_part, sl, lane, y);
        c.Y[r] = y;
#pragma unroll
        for (int a = 0; a < KW; ++a)
            if (a < nw) acc[a] = fmaf(wv[a], y, acc[a]);
        ykey = max(ykey, abs_key_f32(y));
        if (last && ey != kNoExp) scatter2<ZCAP>(c, r, fixed_point_f32(y, shift_y), L, bins, bins + s);
    }
    spmv_end<KW>(c, j, nw, last, L, bins, acc, ykey, red);
}

// Pipelined SpMV for operators whose SELL slices are at most 8 wide.  Chunk i
// of the CTA is in three stages at once: its values and gathers are loaded
// (the gathers use column indices loaded one iteration earlier), the column
// indices of chunk i + 1 are loaded, and the slice width and offset of chunk
// i + 2 are loaded.  One memory round trip per chunk instead of two (column,
// then gather), with 8 extra registers per thread.
template <int KW, int ZCAP, typename TB>
__global__ void __launch_bounds__(kSpmvThreads, 1) k_arnoldi_spmv_lp_pipe(LpCtx c, int j) {
    extern __shared__ int bins[];   // [2 s]: limbs of S w_j (stopping step) or of S y_{m-1} (last step)
    __shared__ double red[32 * KW];
    asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent (see k_arnoldi_spmv_lp)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool stopping;
    if (!spmv_begin<TB>(c, j, stopping)) return;
    if (stopping) {
        spmv_stop_sketch<ZCAP, TB>(c, j, bins);
        return;
    }
    const int s = c.sp.s;
    const TB *V = (const TB *)c.V;
    const TB *wj = V + vcol(c, j);
    const int L = c.identity ? 0 : limb_bits(*c.binmax_chunk);
    const int P = sketch_fraction_bits_from_limb(L);
    const bool last = (j == c.m - 1) && !c.identity;
    const int ey = last ? last_y_exponent(c, j) : kNoExp;
    if (last)
        for (int i2 = threadIdx.x; i2 < 2 * s; i2 += kSpmvThreads) bins[i2] = 0;
    __syncthreads();
    const int shift_y = P - (ey == kNoExp ? 0 : ey);
    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;
    float acc[KW];
#pragma unroll
    for (int a = 0; a < KW; ++a) acc[a] = 0.f;
    unsigned ykey = 0;
    const int lane = threadIdx.x & 31;
    const int64_t nc = chunks_of_cta(c);
    const int64_t step = (int64_t)c.G * kChunkRows;
    const int64_t rw0 = (int64_t)blockIdx.x * kChunkRows + (threadIdx.x & ~31);   // warp's slice in chunk 0

    // slice metadata: chunk i (broadcast, wt_c / so_c) and chunk i + 1 (lane-0
    // values, broadcast one iteration later)
    int wt_c = 0, mw_raw = 0;
    long long so_c = 0, mo_raw = 0;
    if (lane == 0 && nc > 0 && rw0 < c.n) {
        wt_c = __ldg(c.sell_w + (rw0 >> 5));
        so_c = __ldg(c.sell_off + (rw0 >> 5));
    }
    wt_c = __shfl_sync(0xffffffffu, wt_c, 0);
    so_c = __shfl_sync(0xffffffffu, so_c, 0);
    if (lane == 0 && nc > 1 && rw0 + step < c.n) {
        mw_raw = __ldg(c.sell_w + ((rw0 + step) >> 5));
        mo_raw = __ldg(c.sell_off + ((rw0 + step) >> 5));
    }
    int cv[8];
    {
        const int32_t *pc = c.sell_col + so_c + lane;
#pragma unroll
        for (int p = 0; p < 8; ++p)
            if (p < wt_c) cv[p] = __ldcs(pc + 32 * p);
    }
    for (int64_t i = 0; i < nc; ++i) {
        const int64_t rw = rw0 + i * step;
        const int64_t r = rw + lane;
        const bool ok = rw < c.n && r < c.n;   // padded rows of the last slice do no work
        // (1) values, gathers and window of chunk i
        float av[8], xv[8], wv[KW];
        {
            const float *pv = c.sell_val + so_c + lane;
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p < wt_c) {
                    av[p] = __ldcs(pv + 32 * p);
                    xv[p] = Store<TB>::ld(wj + cv[p]);
                }
#pragma unroll
            for (int a = 0; a < KW; ++a) wv[a] = (ok && a < nw) ? Store<TB>::ld(V + c.woff[a] + r) : 0.f;
        }
        // (2) metadata of chunk i + 1 (loaded one iteration ago) and its column indices
        const int wt_n = __shfl_sync(0xffffffffu, mw_raw, 0);
        const long long so_n = __shfl_sync(0xffffffffu, mo_raw, 0);
        int cvn[8];
        {
            const int32_t *pc = c.sell_col + so_n + lane;
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p < wt_n) cvn[p] = __ldcs(pc + 32 * p);
        }
        // (3) metadata of chunk i + 2
        mw_raw = 0;
        mo_raw = 0;
        if (lane == 0 && i + 2 < nc && rw + 2 * step < c.n) {
            mw_raw = __ldg(c.sell_w + ((rw + 2 * step) >> 5));
            mo_raw = __ldg(c.sell_off + ((rw + 2 * step) >> 5));
        }
        // (4) y of chunk i
        if (ok) {
            float y = 0.f;
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p < wt_c) y = fmaf(av[p], xv[p], y);
            c.Y[r] = y;
#pragma unroll
            for (int a = 0; a < KW; ++a)
                if (a < nw) acc[a] = fmaf(wv[a], y, acc[a]);
            ykey = max(ykey, abs_key_f32(y));
            if (last && ey != kNoExp) scatter2<ZCAP>(c, r, fixed_point_f32(y, shift_y), L, bins, bins + s);
        }
        wt_c = wt_n;
        so_c = so_n;
#pragma unroll
        for (int p = 0; p < 8; ++p) cv[p] = cvn[p];
    }
    spmv_end<KW>(c, j, nw, last, L, bins, acc, ykey, red);
}

// Several right-hand sides on one operator (a block B = [b_1 .. b_r] of
// Arnoldi processes in lockstep, same m, k and sketch): the SpMV of step j
// for up to RB of them in one launch, reading each chunk of A once.  Per
// right-hand side q everything is as in k_arnoldi_spmv_lp_pipe: the same
// prologue, the same rows per thread, products and dots in the same order
// (results bitwise equal to its own launch), its own partials, counter and
// last-CTA reduction.  Not for the last step (S y_{m-1} is scattered there
// by the single-vector kernel) nor for a row split.
template <int RB>
struct SpmmArgs {
    LpCtx c[RB];
    int nr;
};

template <int KW, int ZCAP, typename TB, int RB>
__global__ void __launch_bounds__(kSpmvThreads, 1) k_arnoldi_spmm_lp(SpmmArgs<RB> g, int j) {
    extern __shared__ int bins[];   // [2 s]: limbs of S w_j at a stopping step
    __shared__ double red[32 * KW];
    asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent (see k_arnoldi_spmv_lp)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool act[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
        act[q] = false;
        if (q < g.nr) {
            bool stopping = false;
            act[q] = spmv_begin<TB>(g.c[q], j, stopping);
            if (act[q] && stopping) {   // a stop at this step: S w_j only, as the single-vector kernel does
                __syncthreads();
                spmv_stop_sketch<ZCAP, TB>(g.c[q], j, bins);
                act[q] = false;
            }
        }
    }
    const LpCtx &c0 = g.c[0];   // operator and partition: common to the block
    const int i0 = max(0, j - c0.k + 1);
    const int nw = j - i0 + 1;
    float acc[RB][KW];
    unsigned ykey[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
        ykey[q] = 0;
#pragma unroll
        for (int a = 0; a < KW; ++a) acc[q][a] = 0.f;
    }
    const int lane = threadIdx.x & 31;
    const int64_t nc = chunks_of_cta(c0);
    const int64_t step = (int64_t)c0.G * kChunkRows;
    const int64_t rw0 = (int64_t)blockIdx.x * kChunkRows + (threadIdx.x & ~31);   // warp's slice in chunk 0
    int wt_c = 0, mw_raw = 0;
    long long so_c = 0, mo_raw = 0;
    if (lane == 0 && nc > 0 && rw0 < c0.n) {
        wt_c = __ldg(c0.sell_w + (rw0 >> 5));
        so_c = __ldg(c0.sell_off + (rw0 >> 5));
    }
    wt_c = __shfl_sync(0xffffffffu, wt_c, 0);
    so_c = __shfl_sync(0xffffffffu, so_c, 0);
    if (lane == 0 && nc > 1 && rw0 + step < c0.n) {
        mw_raw = __ldg(c0.sell_w + ((rw0 + step) >> 5));
        mo_raw = __ldg(c0.sell_off + ((rw0 + step) >> 5));
    }
    int cv[8];
    {
        const int32_t *pc = c0.sell_col + so_c + lane;
#pragma unroll
        for (int p = 0; p < 8; ++p)
            if (p < wt_c) cv[p] = __ldcs(pc + 32 * p);
    }
    for (int64_t i = 0; i < nc; ++i) {
        const int64_t rw = rw0 + i * step;
        const int64_t r = rw + lane;
        const bool ok = rw < c0.n && r < c0.n;
        float av[8];
        {
            const float *pv = c0.sell_val + so_c + lane;
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p < wt_c) av[p] = __ldcs(pv + 32 * p);
        }
        const int wt_n = __shfl_sync(0xffffffffu, mw_raw, 0);
        const long long so_n = __shfl_sync(0xffffffffu, mo_raw, 0);
        int cvn[8];
        {
            const int32_t *pc = c0.sell_col + so_n + lane;
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p < wt_n) cvn[p] = __ldcs(pc + 32 * p);
        }
        mw_raw = 0;
        mo_raw = 0;
        if (lane == 0 && i + 2 < nc && rw + 2 * step < c0.n) {
            mw_raw = __ldg(c0.sell_w + ((rw + 2 * step) >> 5));
            mo_raw = __ldg(c0.sell_off + ((rw + 2 * step) >> 5));
        }
        // per right-hand side: gathers of w_j and the window, y, dots (the
        // chunk of A is in registers for all of them); the loads of column
        // q + 1 are issued before the products of column q
        if (ok) {
            float xa[8], wa[KW];
            auto load_col = [&](int q, float (&x)[8], float (&w)[KW]) {
                const TB *__restrict__ V = (const TB *)g.c[q].V;
                const TB *__restrict__ wj = V + vcol(g.c[q], j);
#pragma unroll
                for (int p = 0; p < 8; ++p) x[p] = p < wt_c ? Store<TB>::ld(wj + cv[p]) : 0.f;
#pragma unroll
                for (int a = 0; a < KW; ++a) w[a] = a < nw ? Store<TB>::ld(V + g.c[q].woff[a] + r) : 0.f;
            };
            load_col(0, xa, wa);
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                if (q >= g.nr) break;
                float xb[8], wb[KW];
                if (q + 1 < RB && q + 1 < g.nr) load_col(q + 1, xb, wb);
                if (act[q]) {
                    float y = 0.f;
#pragma unroll
                    for (int p = 0; p < 8; ++p)
                        if (p < wt_c) y = fmaf(av[p], xa[p], y);
                    float *__restrict__ Yq = g.c[q].Y;
                    Yq[r] = y;
#pragma unroll
                    for (int a = 0; a < KW; ++a)
                        if (a < nw) acc[q][a] = fmaf(wa[a], y, acc[q][a]);
                    ykey[q] = max(ykey[q], abs_key_f32(y));
                }
                if (q + 1 < RB && q + 1 < g.nr) {
#pragma unroll
                    for (int p = 0; p < 8; ++p) xa[p] = xb[p];
#pragma unroll
                    for (int a = 0; a < KW; ++a) wa[a] = wb[a];
                }
            }
        }
        wt_c = wt_n;
        so_c = so_n;
#pragma unroll
        for (int p = 0; p < 8; ++p) cv[p] = cvn[p];
    }
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (act[q]) spmv_end<KW>(g.c[q], j, nw, false, 0, bins, acc[q], ykey[q], red);
}

// S = I (tests): SV[:, j] = sigma_j w_j, SAV[:, j] = sigma_j y_j.
template <typename TB>
__global__ void __launch_bounds__(kThreads) k_identity_cols_lp(LpCtx c, int j) {
    if (c.iscal[0] && c.iscal[3] <= j) return;
    const TB *wj = (const TB *)c.V + vcol(c, j);
    const double sigma = c.stepsc[4 * (size_t)j];
    const int s = c.sp.s;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < c.n; r += (int64_t)gridDim.x * blockDim.x) {
        c.SV[r + (size_t)j * s] = sigma * (double)Store<TB>::ld(wj + r);
        c.SAV[r + (size_t)j * s] = sigma * (double)c.Y[r];
    }
}

// Sum of the per-lane copies of bin i (C = 1 << lc copies, copy index in the
// low bits) by one warp: exact in int32, since every copy holds a subset of
// the bin's contributions and all of them together fit (limb width rule; a
// split sign bin holds a subset too).
__device__ __forceinline__ int sum_copies(const int *b, int i, int lc) {
    const int lane = threadIdx.x & 31;
    int v = lane < (1 << lc) ? b[(i << lc) + lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-lane bin copies of the split layout: 2 * SB * 8 bins per limb, C copies,
// 64 KB per limb either way.
template <int SB> struct SplitGeom {
    static constexpr int kLc = SB == 64 ? 4 : 3;
    static constexpr int kBins = 8 * 2 * SB;
};

// SB = 0: general bins [s] per limb (signs selected), lc per-lane copies;
// SB = 64 or 128: split bins [stripe][sign][SB] (compact pattern, zeta = 8).
template <int KW, int ZCAP, typename TB, int SB>
__global__ void __launch_bounds__(kUpdThreads, 1) k_arnoldi_update_lp(LpCtx c, int j) {
    // per-lane copies of the bins: [limb 0 | limb 1 of S w_j | residual limb][nbin << lc]
    extern __shared__ int bins[];
    __shared__ double red[32 * (KW + 1)];
    __shared__ double sh[kMaxK];     // MGS coefficients h_ij
    __shared__ float scf[kMaxK];     // h_ij sigma_i in FP32, as applied
    __shared__ float sigf_s;
    asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent (see k_arnoldi_spmv_lp)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (c.iscal[0] && c.iscal[3] <= j) return;   // stopped at this step (set by its spmv launch) or earlier
    TB *V = (TB *)c.V;
    const int G = gridDim.x;
    const double *fd = c.fin_d + (size_t)j * kP1;
    const double sigma = c.stepsc[4 * (size_t)j];
    const double ymax = fd[kP1 - 1];
    const int s = c.sp.s;
    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;

    if (threadIdx.x == 0) {
        // MGS in the window, ascending, from the dots and the Gram matrix:
        // h_i = <v_i, y> - sum_{i' < i} h_i' <v_i, v_i'>.
        for (int a = 0; a < nw; ++a) {
            const int ia = i0 + a;
            const double sa = (ia == j) ? sigma : c.vscale[ia];
            double h = sa * sigma * fd[a];
            for (int b2 = 0; b2 < a; ++b2) {
                const int ib = i0 + b2;
                const double sb = c.vscale[ib];
                const double gab = c.gram[(size_t)ia * kMaxK + (ia - ib)];
                h -= sh[b2] * sa * sb * gab;
            }
            sh[a] = h;
            scf[a] = (float)(h * sa);
        }
        sigf_s = (float)sigma;
    }
    const bool do_update = j < c.m - 1;
    const bool sk = !c.identity;
    constexpr bool split = SB != 0;
    const bool resid = !Store<TB>::kExact && sk && do_update;
    const int L = sk ? limb_bits(*c.binmax_chunk) : 0;
    const int P = sketch_fraction_bits_from_limb(L);
    const double wmax = c.fin_w[2 * (size_t)j + 1];
    const int ew = (sk && positive_finite(wmax)) ? bound_exponent(wmax) : kNoExp;
    const int shift_w = P - (ew == kNoExp ? 0 : ew);
    const LimbScale lsw(shift_w, L);
    const int lc = split ? SplitGeom<SB>::kLc : c.lc, cm = (1 << lc) - 1;
    const int ns = split ? (SplitGeom<SB>::kBins << SplitGeom<SB>::kLc) : (s << lc);
    int *wb0 = bins, *wb1 = bins + ns, *db = bins + 2 * ns;
    if (sk)
        for (int i = threadIdx.x; i < (resid ? 3 : 2) * ns; i += kUpdThreads) bins[i] = 0;
    __syncthreads();
    const float sigf = sigf_s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c.vscale[j] = sigma;
        double *cf = c.coef + (size_t)j * kCoef;
        cf[0] = (double)sigf;
        for (int a = 0; a < nw; ++a) cf[1 + a] = (double)scf[a];
        // H holds the coefficients of the relation the stored basis satisfies
        // with the FP32 coefficients applied (the one S A v_j is formed from):
        // A v_j = (sigma_j / sigf) (v_{j+1} / sigma_{j+1} + sum_a scf_a v_{i0+a} / sigma_{i0+a}),
        // each within one FP32 rounding of the MGS coefficient h_a
        if (do_update)
            for (int a = 0; a < nw; ++a) {
                const double sa = (i0 + a == j) ? sigma : c.vscale[i0 + a];
                c.H[(i0 + a) + (size_t)j * (c.m + 1)] = sigma * (double)scf[a] / ((double)sigf * sa);
            }
        c.ex[j] = ew;
    }
    // one-limb fixed point for the BF16 residual: |bf16(w) - w| <= 2^-8 |w|
    // and |w| <= sigma_j max|y_j| + sum_i |h_ij sigma_i| max|w_i|
    int ed = kNoExp;
    if (resid) {
        double wb = (double)sigf * ymax;
        for (int a = 0; a < nw; ++a) wb += fabs((double)scf[a]) * c.fin_w[2 * (size_t)(i0 + a) + 1];
        const double dbd = wb * (1.0 / 256.0) * (1.0 + 1.0 / 1024.0);
        ed = positive_finite(dbd) ? bound_exponent(dbd) : kNoExp;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && do_update) c.ex[c.m + j + 1] = ed;
    const int shift_d = L - (ed == kNoExp ? 0 : ed);

    const int ng = min(j + 1, c.k - 1);
    float part[KW + 1];
#pragma unroll
    for (int i = 0; i <= KW; ++i) part[i] = 0.f;
    unsigned nkey = 0;
    TB *wn = V + vcol(c, j + 1);
    const int lane = threadIdx.x & 31;
    const int64_t nc = chunks_of_cta(c);
    constexpr int U = KW <= 2 ? 4 : (KW <= 4 ? 2 : 1);   // chunks in flight per thread
    for (int64_t i = 0; i < nc; i += U) {
        float yv[U], wv[U][KW];
        int64_t rr[U];
        uint2 pvu[U];   // compact pattern words (split layout), loaded with the rest
#pragma unroll
        for (int u = 0; u < U; ++u) {
            rr[u] = i + u < nc ? chunk_row(c, i + u) : -1;
            const bool ok = rr[u] >= 0;
            yv[u] = (ok && do_update) ? c.Y[rr[u]] : 0.f;
#pragma unroll
            for (int a = 0; a < KW; ++a)
                wv[u][a] = (ok && a < nw) ? Store<TB>::ld(V + c.woff[a] + rr[u]) : 0.f;
            pvu[u] = make_uint2(0u, 0u);
            if constexpr (split)
                if (ok) pvu[u] = __ldg((const uint2 *)(c.pattern8 + rr[u] * 8));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = rr[u];
            if (r < 0) continue;
            float wjr = wv[u][0];
#pragma unroll
            for (int a = 1; a < KW; ++a)
                if (a == nw - 1) wjr = wv[u][a];
            int row[ZCAP];
            bool neg[ZCAP];
            const uint2 pv = pvu[u];
            if constexpr (!split)
                if (sk) pattern_row<ZCAP>(c, r, row, neg);
            if (sk && ew != kNoExp) {
                // exact sketch of the stored w_j, per-lane bin copies
                int l0, l1;
                limbs_f32(wjr, lsw, l0, l1);
                if constexpr (split) {
                    // bin 2 SB stripe + pattern byte: signs in separate bins
                    constexpr int LC = SplitGeom<SB>::kLc;
                    int *b0l = wb0 + (lane & ((1 << LC) - 1)), *b1l = wb1 + (lane & ((1 << LC) - 1));
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int e = (int)__byte_perm(q < 4 ? pv.x : pv.y, 0u, 0x4440u + (q & 3));
                        const int bi = ((2 * SB * q) | e) << LC;
                        atomicAdd(b0l + bi, l0);
                        atomicAdd(b1l + bi, l1);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < ZCAP; ++q)
                        if (q < c.sp.zeta) {
                            const int bi = (row[q] << lc) | (lane & cm);
                            atomicAdd(wb0 + bi, neg[q] ? -l0 : l0);
                            atomicAdd(wb1 + bi, neg[q] ? -l1 : l1);
                        }
                }
            }
            if (do_update) {
                float w = sigf * yv[u];
#pragma unroll
                for (int a = 0; a < KW; ++a)
                    if (a < nw) w = fmaf(-scf[a], wv[u][a], w);
                const float wr = Store<TB>::rnd(w);
                Store<TB>::st(wn + r, wr);
                part[0] = fmaf(wr, wr, part[0]);
                nkey = max(nkey, abs_key_f32(wr));
#pragma unroll
                for (int a = 0; a < KW; ++a)
                    if (a < nw && nw - a <= ng) part[1 + a] = fmaf(wr, wv[u][a], part[1 + a]);
                if (resid && ed != kNoExp) {
                    // wr - w is exact in FP32 (Sterbenz: wr and w lie within a factor 2)
                    const int vd = (int)fixed_point_f32(wr - w, shift_d);
                    if constexpr (split) {
                        constexpr int LC = SplitGeom<SB>::kLc;
                        int *dl = db + (lane & ((1 << LC) - 1));
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int e = (int)__byte_perm(q < 4 ? pv.x : pv.y, 0u, 0x4440u + (q & 3));
                            atomicAdd(dl + (((2 * SB * q) | e) << LC), vd);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < ZCAP; ++q)
                            if (q < c.sp.zeta) atomicAdd(db + ((row[q] << lc) | (lane & cm)), neg[q] ? -vd : vd);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (sk) {
        // per-CTA partials: copies summed by one warp per bin
        const int warp = threadIdx.x >> 5;
        long long *ow = c.skWp + ((size_t)(j & 1) * G + blockIdx.x) * s;
        long long *od = c.skDp + (size_t)blockIdx.x * s;
        for (int i = warp; i < s; i += kUpdThreads / 32) {
            long long v0, v1, vd = 0;
            if constexpr (split) {
                int q = 0;
                while (q + 1 < 8 && i >= c.sp.start[q + 1]) ++q;
                const int bp = 2 * SB * q + (i - c.sp.start[q]), bn = bp + SB;   // positive and negative bins
                v0 = (long long)sum_copies(wb0, bp, lc) - sum_copies(wb0, bn, lc);
                v1 = (long long)sum_copies(wb1, bp, lc) - sum_copies(wb1, bn, lc);
                if (resid) vd = (long long)sum_copies(db, bp, lc) - sum_copies(db, bn, lc);
            } else {
                v0 = sum_copies(wb0, i, lc);
                v1 = sum_copies(wb1, i, lc);
                if (resid) vd = sum_copies(db, i, lc);
            }
            if (lane == 0) {
                ow[i] = (v1 << L) + v0;
                if (resid) od[i] = vd;
            }
        }
    }
    if (!do_update) return;
    double partd[KW + 1];
#pragma unroll
    for (int i = 0; i <= KW; ++i) partd[i] = (double)part[i];
    block_sum<KW + 1, kUpdThreads>(partd, red);
    const unsigned nmk = (unsigned)block_max_key<kUpdThreads>((unsigned long long)nkey, (unsigned long long *)red);
    if (threadIdx.x == 0) {
        double *o = c.p2 + (size_t)blockIdx.x * kP2;
        o[0] = partd[0];
        o[1] = (double)__uint_as_float(nmk);
        for (int a = 0; a < KW; ++a) o[2 + a] = partd[1 + a];
    }
    if (last_to_arrive(c.cnt + 1)) {
        const int warp = threadIdx.x >> 5;
        for (int v = warp; v < 2 + nw; v += kUpdThreads / 32) {
            const int d = nw - (v - 2);   // Gram distance of slot v - 2
            if (v >= 2 && (d < 1 || d > ng)) continue;
            const double rv = warp_reduce_partials(c.p2 + v, G, kP2, v == 1);
            if ((threadIdx.x & 31) == 0) {
                if (v < 2) c.fin_w[2 * (size_t)(j + 1) + v] = rv;
                else c.gram[(size_t)(j + 1) * kMaxK + d] = rv;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // ||A v_j||^2 = sum_i h_ij^2 + ||w_{j+1}||^2 for the orthonormal window
            const double n2 = c.fin_w[2 * (size_t)(j + 1)];
            double hs = 0.0;
            for (int a = 0; a < nw; ++a) hs += sh[a] * sh[a];
            const double hn = sqrt(n2);
            double *o = c.stepsc + 4 * (size_t)(j + 1);
            o[0] = hn > 0.0 ? 1.0 / hn : 0.0;
            o[1] = hn;
            o[2] = (hn > kBreakTol * sqrt(hs + n2)) ? 0.0 : 1.0;
            c.cnt[1] = 0u;
        }
    }
}

// After the loop: the pending column.  Ran to the end: S w_{m-1} (SV), S y_{m-2}
// by the relation and the scattered S y_{m-1} (SAV).  Stopped at step me: S w_me
// (not a basis column) gives S y_{me-1} by the relation.
template <typename TB>
__global__ void __launch_bounds__(kThreads) k_arnoldi_finish_lp(LpCtx c) {
    const int me = c.iscal[1];
    if (me == 0 || c.identity) return;
    if (c.iscal[0] == 2) return;   // stopped by the criterion: columns < me already final
    const bool stopped = c.iscal[0] != 0;
    if (stopped) finalize_column<TB>(c, me, false, false, false);
    else finalize_column<TB>(c, c.m - 1, true, false, true);
}

// | ||S v_j||^2 - 1 | per column (the embedding-quality estimate of Sec. 4.3).
__global__ void __launch_bounds__(kThreads) k_arnoldi_eps_lp(LpCtx c) {
    const int me = c.iscal[1];
    const int j = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= me) return;
    const int s = c.sp.s;
    double acc = 0.0;
    for (int i = lane; i < s; i += 32) acc = fma(c.SV[i + (size_t)j * s], c.SV[i + (size_t)j * s], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) c.epscol[j] = fabs(acc - 1.0);
}

__global__ void __launch_bounds__(kThreads) k_arnoldi_info_lp(LpCtx c, skf_info *info) {
    __shared__ double red[64];
    const int me = c.iscal[1];
    double eps = 0.0;
    for (int j = threadIdx.x; j < me; j += kThreads) eps = fmax(eps, c.epscol[j]);
    eps = block_max(eps, red);
    if (threadIdx.x == 0 && info != nullptr) {
        info->status = c.iscal[2];
        info->m_eff = me;
        info->breakdown = (c.iscal[0] == 1 && me > 0) ? 1 : 0;
        info->beta = me > 0 ? 1.0 / c.vscale[0] : 0.0;
        info->eps_est = eps;
    }
}

template <int KW, int ZCAP, typename TB>
void launch_steps(const LpCtx &c, bool pipe, size_t smem_spmv, size_t smem_upd, cudaStream_t st,
                  const StepHook *hook, const skf_sketch *dense, void *dwork) {
    auto spmv = pipe ? k_arnoldi_spmv_lp_pipe<KW, ZCAP, TB> : k_arnoldi_spmv_lp<KW, ZCAP, TB>;
    auto update = k_arnoldi_update_lp<KW, ZCAP, TB, 0>;
    if constexpr (ZCAP == 8) {
        if (c.split) update = c.p8_block == 64 ? k_arnoldi_update_lp<KW, 8, TB, 64> : k_arnoldi_update_lp<KW, 8, TB, 128>;
    }
    if (smem_spmv > 48 * 1024)
        cudaFuncSetAttribute(spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_spmv);
    if (smem_upd > 48 * 1024)
        cudaFuncSetAttribute(update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd);
    const unsigned gid = (unsigned)std::min<int64_t>((c.n + kThreads - 1) / kThreads, 8ll * c.G);
    // the step kernels are launched as programmatic dependents of the launch
    // before them (each waits for it in full; only the placement overlaps)
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    auto config = [&](unsigned grid, unsigned block, size_t smem) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = pdl;
        cfg.numAttrs = 1;
        return cfg;
    };
    const cudaLaunchConfig_t cfg_l = config((unsigned)long_ctas(c.rs.nseg, num_sms()), 256, 0);
    const cudaLaunchConfig_t cfg_s = config((unsigned)c.G, kSpmvThreads, smem_spmv);
    const cudaLaunchConfig_t cfg_u = config((unsigned)c.G, kUpdThreads, smem_upd);
    for (int j = 0; j < c.m; ++j) {
        LpCtx cj = c;
        window_offsets(cj, j);
        if (c.rs.sell_long) cudaLaunchKernelEx(&cfg_l, k_spmv_long_lp<TB>, cj, j);
        cudaLaunchKernelEx(&cfg_s, spmv, cj, j);
        if (j >= 1) call_hook(hook, j - 1, st);   // S v_i, S A v_i final for i < j - 1
        if (dense) {   // SRHT / SRDCT: SV[:, j] = sigma_j S w_j, SAV[:, j] = sigma_j S y_j
            DenseCols dc{};
            dc.ncols = 2;
            dc.x[0] = (const float *)c.V + vcol(c, j);
            dc.x[1] = c.Y;
            dc.out[0] = c.SV + (size_t)j * c.sp.s;
            dc.out[1] = c.SAV + (size_t)j * c.sp.s;
            dc.colscale = c.stepsc + 4 * (size_t)j;
            dc.iscal = c.iscal;
            dc.step = j;
            dense_sketch_f32(dense, dc, dwork, st);
        } else if (c.identity) {
            k_identity_cols_lp<TB><<<gid, kThreads, 0, st>>>(cj, j);
        }
        cudaLaunchKernelEx(&cfg_u, update, cj, j);
        if (j + 1 < c.m) call_col_hook(hook, j + 1, st);
    }
}

template <int ZCAP, typename TB>
void launch_steps_k(const LpCtx &c, bool pipe, size_t s1, size_t s2, cudaStream_t st, const StepHook *hook,
                    const skf_sketch *dense, void *dwork) {
    if (c.k <= 2) launch_steps<2, ZCAP, TB>(c, pipe, s1, s2, st, hook, dense, dwork);
    else if (c.k <= 4) launch_steps<4, ZCAP, TB>(c, pipe, s1, s2, st, hook, dense, dwork);
    else if (c.k <= 8) launch_steps<8, ZCAP, TB>(c, pipe, s1, s2, st, hook, dense, dwork);
    else launch_steps<16, ZCAP, TB>(c, pipe, s1, s2, st, hook, dense, dwork);
}

// Context, launch shapes and workspace of one reduced-precision Arnoldi
// process (the workspace is the caller's to release with dfree).
struct LpRun {
    LpCtx c;
    bool pipe;
    size_t smem_spmv, smem_upd;
    const skf_sketch *dense;
    void *dwork;
    char *ws;
};

template <typename TB>
skf_status lp_setup(const skf_csr *A, const skf_sketch *S, int m, int k, TB *V, int64_t ldv, double *vscale,
                    double *SV, double *SAV, double *H, int *iscal, cudaStream_t st, int vring, LpRun &run) {
    LpCtx c{};
    c.n = A->n;
    c.sell_off = A->sell_off;
    c.sell_w = A->sell_w;
    c.sell_val = (const float *)A->sell_val;
    c.sell_col = A->sell_col;
    c.norm_inf = A->norm_inf;
    // an SRHT or SRDCT (F32 basis) is applied by its own kernels to w_j and
    // y_j after each SpMV; the step kernels then run as for S = I (no
    // fixed-point sketch work of their own)
    const skf_sketch *dense = (S->kind == SKF_SKETCH_SRHT || S->kind == SKF_SKETCH_SRDCT) ? S : nullptr;
    c.identity = S->kind == SKF_SKETCH_IDENTITY || dense != nullptr;
    if (!c.identity) {
        c.sp = make_sparse_sign(S);
        c.pattern = S->pattern;
        c.pattern8 = S->pattern8;
        c.p8_block = S->p8_block;
        c.binmax_chunk = S->binmax_chunk;
    }
    c.sp.s = S->s;
    c.sp.zeta = c.identity ? 1 : S->zeta;
    c.inv_sqrt_zeta = 1.0 / sqrt((double)c.sp.zeta);
    c.m = m;
    c.k = k;
    c.V = V;
    c.ldv = ldv;
    c.vring = vring;
    c.vscale = vscale;
    c.SV = SV;
    c.SAV = SAV;
    c.H = H;
    c.iscal = iscal;
    chunk_partition(A->n, &c.G);
    const int G = c.G;
    const int s = S->s;
    const bool bf = !Store<TB>::kExact;

    // per-lane bin copies of the update kernel: as many (up to 32) as fit;
    // bins [stripe][sign][128] with the compact pattern and zeta = 8
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    c.split = (!c.identity && S->pattern8 != nullptr && S->zeta == 8) ? 1 : 0;
    const int nlimb = bf ? 3 : 2;
    const size_t static_upd = sizeof(double) * 32 * (kMaxK + 1) + sizeof(double) * kMaxK + sizeof(float) * (kMaxK + 1) +
                              256;
    c.lc = 5;
    while (c.lc > 0 && sizeof(int) * (size_t)nlimb * ((size_t)s << c.lc) + static_upd > (size_t)optin) --c.lc;
    // split layout: 16 * block bins per limb, 64 / block * 128 copies: 64 KB per limb
    const size_t per_limb = c.split ? (size_t)16 * c.p8_block * (c.p8_block == 64 ? 16 : 8) : ((size_t)s << c.lc);
    const size_t smem_upd = c.identity ? 0 : sizeof(int) * (size_t)nlimb * per_limb;
    const size_t smem_spmv = c.identity ? 0 : sizeof(int) * 2 * (size_t)s;
    if (smem_upd + static_upd > (size_t)optin || smem_spmv > (size_t)optin)
        return fail(SKF_ERR_NOT_SUPPORTED, "sketch size s too large for the shared-memory bins");
    // slices at most 8 wide: the pipelined SpMV (a row split takes the generic one)
    const bool pipe = A->max_width <= 8 && A->nlong == 0 && A->perm == nullptr;
    c.rs = row_split_of(A);

    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t szY = sizeof(float) * A->n;
    const size_t szP1 = sizeof(double) * (size_t)G * kP1;
    const size_t szP2 = sizeof(double) * (size_t)G * kP2;
    const size_t szFd = sizeof(double) * (size_t)m * kP1;
    const size_t szFw = sizeof(double) * (size_t)(m + 1) * 2;
    const size_t szSc = sizeof(double) * (size_t)(m + 1) * 4;
    const size_t szGram = sizeof(double) * (size_t)(m + 1) * kMaxK;
    const size_t szCoef = sizeof(double) * (size_t)m * kCoef;
    const size_t szSk = c.identity ? 0 : sizeof(double) * (size_t)m * s;
    const size_t szSd = (c.identity || !bf) ? 0 : sizeof(double) * (size_t)s;
    const size_t szPart = c.identity ? 0 : sizeof(long long) * (size_t)G * s;
    const size_t szEx = sizeof(int) * (size_t)(2 * m + 1);
    const size_t szEps = sizeof(double) * (size_t)m;
    const size_t szCnt = sizeof(unsigned) * 4;
    const size_t szSeg = sizeof(float) * (size_t)std::max<int64_t>(c.rs.nseg, 1);
    const size_t szDense = dense ? dense_sketch_work_bytes(S) : 0;
    const size_t total = al(szY) + al(szP1) + al(szP2) + al(szFd) + al(szFw) + al(szSc) + al(szGram) + al(szCoef) +
                         al(szSk) + al(szSd) + al(2 * szPart) + al(szPart) + (bf ? al(szPart) : 0) + al(szEx) +
                         al(szEps) + al(szCnt) + al(szSeg) + al(szDense);
    char *ws = nullptr;
    skf_status stt = dalloc((void **)&ws, total, st);
    if (stt != SKF_OK) return stt;
    size_t off = 0;
    auto take = [&](size_t sz) {
        char *p = ws + off;
        off += al(sz);
        return p;
    };
    c.Y = (float *)take(szY);
    c.seg_part = (float *)take(szSeg);
    c.p1 = (double *)take(szP1);
    c.p2 = (double *)take(szP2);
    c.fin_d = (double *)take(szFd);
    c.fin_w = (double *)take(szFw);
    c.stepsc = (double *)take(szSc);
    c.gram = (double *)take(szGram);
    c.coef = (double *)take(szCoef);
    c.skw = (double *)take(szSk);
    c.sd = (double *)take(szSd);
    c.skWp = (long long *)take(2 * szPart);
    c.skYp = (long long *)take(szPart);
    c.skDp = bf ? (long long *)take(szPart) : nullptr;
    c.ex = (int *)take(szEx);
    c.epscol = (double *)take(szEps);
    c.cnt = (unsigned *)take(szCnt);
    void *dwork = szDense ? (void *)take(szDense) : nullptr;
    cudaMemsetAsync(c.cnt, 0, szCnt, st);
    run.c = c;
    run.pipe = pipe;
    run.smem_spmv = smem_spmv;
    run.smem_upd = smem_upd;
    run.dense = dense;
    run.dwork = dwork;
    run.ws = ws;
    return SKF_OK;
}

// Host driver: init, m x (spmv, update), finish, eps, info on `st`.
template <typename TB>
skf_status arnoldi_run_lp(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, TB *V, int64_t ldv,
                          double *vscale, double *SV, double *SAV, double *H, int *iscal, skf_info *info,
                          cudaStream_t st, const StepHook *hook = nullptr, int vring = 0) {
    LpRun run{};
    skf_status stt = lp_setup<TB>(A, S, m, k, V, ldv, vscale, SV, SAV, H, iscal, st, vring, run);
    if (stt != SKF_OK) return stt;
    const LpCtx &c = run.c;
    const int G = c.G;
    const bool pipe = run.pipe;
    const size_t smem_spmv = run.smem_spmv, smem_upd = run.smem_upd;
    const skf_sketch *dense = run.dense;
    void *dwork = run.dwork;
    char *ws = run.ws;

    k_arnoldi_init_lp<TB><<<G, kChunkRows, 0, st>>>(c, b);
    call_col_hook(hook, 0, st);
    if (c.sp.zeta <= 8) launch_steps_k<8, TB>(c, pipe, smem_spmv, smem_upd, st, hook, dense, dwork);
    else launch_steps_k<16, TB>(c, pipe, smem_spmv, smem_upd, st, hook, dense, dwork);
    k_arnoldi_finish_lp<TB><<<G, kThreads, 0, st>>>(c);
    call_hook(hook, m, st);
    k_arnoldi_eps_lp<<<(m + (kThreads / 32) - 1) / (kThreads / 32), kThreads, 0, st>>>(c);
    k_arnoldi_info_lp<<<1, kThreads, 0, st>>>(c, info);
    count_launches(4 + ((c.identity && !dense ? 3ll : 2ll) + (c.rs.sell_long ? 1 : 0)) * m);   // + dense_sketch_f32's own
    cudaError_t e = cudaGetLastError();
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "reduced-precision Arnoldi kernels");
    return SKF_OK;
}

// A block of nr Arnoldi processes on one operator and one sketch (same m
// and k, right-hand sides b[q]), in lockstep: per step one SpMM launch per
// group of kSpmmBlock right-hand sides (each chunk of A read once per group),
// then each process's own update.  Every process computes exactly what its
// own arnoldi_run_lp computes.  Falls back to one process after another
// where the SpMM kernel does not apply (slices wider than 8, a row split,
// sorted slices, sketches other than sparse-sign with zeta <= 8, k > 2).
constexpr int kSpmmBlock = 4;

template <typename TB>
skf_status arnoldi_run_lp_block(const skf_csr *A, const skf_sketch *S, int nr, const double *const *b, int m, int k,
                                TB *const *V, int64_t ldv, double *const *vscale, double *const *SV,
                                double *const *SAV, double *const *H, int *const *iscal, skf_info *const *info,
                                cudaStream_t st) {
    const bool fits = S->kind == SKF_SKETCH_SPARSE_SIGN && S->zeta <= 8 && k <= 2 && A->max_width <= 8 &&
                      A->nlong == 0 && A->perm == nullptr;
    if (!fits || nr <= 1) {
        for (int q = 0; q < nr; ++q) {
            const skf_status e = arnoldi_run_lp<TB>(A, S, b[q], m, k, V[q], ldv, vscale[q], SV[q], SAV[q], H[q],
                                                    iscal[q], info[q], st);
            if (e != SKF_OK) return e;
        }
        return SKF_OK;
    }
    std::vector<LpRun> runs((size_t)nr);
    skf_status stt = SKF_OK;
    int made = 0;
    for (; made < nr && stt == SKF_OK; ++made)
        stt = lp_setup<TB>(A, S, m, k, V[made], ldv, vscale[made], SV[made], SAV[made], H[made], iscal[made], st, 0,
                           runs[made]);
    if (stt != SKF_OK) {
        for (int q = 0; q + 1 < made; ++q) dfree(runs[q].ws, st);
        return stt;
    }
    const int G = runs[0].c.G;
    for (int q = 0; q < nr; ++q) k_arnoldi_init_lp<TB><<<G, kChunkRows, 0, st>>>(runs[q].c, b[q]);
    auto spmm = k_arnoldi_spmm_lp<2, 8, TB, kSpmmBlock>;
    auto spmv = k_arnoldi_spmv_lp_pipe<2, 8, TB>;
    auto update = k_arnoldi_update_lp<2, 8, TB, 0>;
    if (runs[0].c.split)
        update = runs[0].c.p8_block == 64 ? k_arnoldi_update_lp<2, 8, TB, 64> : k_arnoldi_update_lp<2, 8, TB, 128>;
    const size_t smem_spmv = runs[0].smem_spmv, smem_upd = runs[0].smem_upd;
    if (smem_spmv > 48 * 1024) {
        cudaFuncSetAttribute(spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_spmv);
        cudaFuncSetAttribute(spmm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_spmv);
    }
    if (smem_upd > 48 * 1024) cudaFuncSetAttribute(update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd);
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    auto config = [&](unsigned grid, unsigned block, size_t smem) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = pdl;
        cfg.numAttrs = 1;
        return cfg;
    };
    const cudaLaunchConfig_t cfg_s = config((unsigned)G, kSpmvThreads, smem_spmv);
    const cudaLaunchConfig_t cfg_u = config((unsigned)G, kUpdThreads, smem_upd);
    long long nlaunch = nr;
    std::vector<LpCtx> cj((size_t)nr);
    for (int j = 0; j < m; ++j) {
        for (int q = 0; q < nr; ++q) {
            cj[q] = runs[q].c;
            window_offsets(cj[q], j);
        }
        if (j < m - 1) {
            for (int q0 = 0; q0 < nr; q0 += kSpmmBlock) {
                SpmmArgs<kSpmmBlock> args{};
                args.nr = std::min(kSpmmBlock, nr - q0);
                for (int q = 0; q < args.nr; ++q) args.c[q] = cj[q0 + q];
                cudaLaunchKernelEx(&cfg_s, spmm, args, j);
                ++nlaunch;
            }
        } else {
            for (int q = 0; q < nr; ++q) cudaLaunchKernelEx(&cfg_s, spmv, cj[q], j);
            nlaunch += nr;
        }
        for (int q = 0; q < nr; ++q) cudaLaunchKernelEx(&cfg_u, update, cj[q], j);
        nlaunch += nr;
    }
    for (int q = 0; q < nr; ++q) {
        const LpCtx &c = runs[q].c;
        k_arnoldi_finish_lp<TB><<<G, kThreads, 0, st>>>(c);
        k_arnoldi_eps_lp<<<(m + (kThreads / 32) - 1) / (kThreads / 32), kThreads, 0, st>>>(c);
        k_arnoldi_info_lp<<<1, kThreads, 0, st>>>(c, info[q]);
        nlaunch += 3;
    }
    count_launches(nlaunch);
    const cudaError_t e = cudaGetLastError();
    for (int q = 0; q < nr; ++q) dfree(runs[q].ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "reduced-precision block Arnoldi kernels");
    return SKF_OK;
}

}  // namespace
}  // namespace lp
}  // namespace skf
