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
// Two kernels per step:
//   spmv   (step j): y_j = A w_j in FP32 on chunk-interleaved rows -> Y;
//                    partial <w_i, y_j> for the window, max|y_j|; exact
//                    fixed-point sketch of the stored w_j (two limbs; its
//                    maximum is known from the previous step).
//   update (step j): S w_j from the integer partials; MGS coefficients from
//                    the dots and the window Gram matrix; w_{j+1} =
//                    sigma_j y_j - sum_i h_ij sigma_i w_i in FP32, rounded and
//                    stored; ||w_{j+1}||^2, Gram entries, max|w_{j+1}|.
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
constexpr int kUpdThreads = 512;
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

struct LpCtx {
    int64_t n;
    const int64_t *sell_off;   // SELL-32 operator with FP32 values (see skf_csr)
    const int32_t *sell_w;
    const float *sell_val;
    const int32_t *sell_col;
    double norm_inf;           // ||A||_inf
    SparseSign sp;
    const uint16_t *pattern;
    const int *binmax;         // bin-load maximum of the update kernel's row partition
    const int *binmax_chunk;   // bin-load maximum of the SpMV kernel's chunk partition
    int identity;              // S = I
    int m, k;
    void *V;                   // TB [m][ldv]
    int64_t ldv;
    double *vscale, *SV, *SAV, *H;
    float *Y;                  // [n] y_j = A w_j
    double *p1;                // [Gs][kP1]
    double *p2;                // [G][kP2]
    double *fin_d;             // [m][kP1] reduced dots of step j, max|y_j|
    double *fin_w;             // [m+1][2] ||w_j||^2, max|w_j|
    double *stepsc;            // [m+1][4] 1/||w_j||, ||w_j||, stop flag
    double *gram;              // [m+1][kMaxK] <w_j, w_{j-d}>
    double *coef;              // [m][kCoef] the FP32 coefficients update j applied
    double *skw;               // [m][s] S w_j in units of the +-1 pattern
    long long *skWp;           // [Gs][s] fixed-point partials of S w_j
    long long *skYp;           // [Gs][s] fixed-point partials of S y_{m-1}
    long long *skDp;           // [G][s]  fixed-point partials of the BF16 residual of w_{j+1}
    int *ex;                   // exponents: [0, m) S w_j, [m, 2m) residual of w_j, [2m] S y_{m-1}
    double *epscol;            // [m]
    double inv_sqrt_zeta;
    unsigned *cnt;             // [2] arrival tickets
    int *iscal;                // [0] stopped, [1] m_eff, [2] status, [3] step that stopped
    int64_t rows_per_cta;      // contiguous partition of the init and update kernels
    int G_upd, G_spmv;
};

template <typename TB>
__global__ void __launch_bounds__(kThreads) k_arnoldi_init_lp(LpCtx c, const double *__restrict__ b) {
    __shared__ double red[64];
    TB *V = (TB *)c.V;
    const int64_t r0 = (int64_t)blockIdx.x * c.rows_per_cta;
    const int64_t r1 = min(c.n, r0 + c.rows_per_cta);
    double nrm[1] = {0.0};
    double mx = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) {
        const float x = Store<TB>::rnd((float)b[r]);   // b rounded to FP32, then to the storage type
        Store<TB>::st(V + r, x);
        nrm[0] = fma((double)x, (double)x, nrm[0]);
        mx = fmax(mx, fabs((double)x));
    }
    block_sum<1>(nrm, red);
    mx = block_max(mx, red);
    if (threadIdx.x == 0) {
        c.p2[(size_t)blockIdx.x * kP2 + 0] = nrm[0];
        c.p2[(size_t)blockIdx.x * kP2 + 1] = mx;
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < (c.m + 1) * c.m; i += kThreads) c.H[i] = 0.0;
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

// Finalise S w_j for this CTA's slice of the rows of S (SV[:, j]); then, for
// j >= 1, S y_{j-1} from the Arnoldi relation (SAV[:, j-1]); at the last step
// also the directly scattered S y_{m-1} (SAV[:, m-1]).  Sketch values are in
// units of the +-1 pattern; SV and SAV carry the 1/sqrt(zeta) scale.
template <typename TB>
__device__ __forceinline__ void finalize_sketches(const LpCtx &c, int j, bool last) {
    const int s = c.sp.s;
    const int G = gridDim.x;
    const int L = limb_bits(*c.binmax_chunk);
    const int P = sketch_fraction_bits_from_limb(L);
    const int Ld = Store<TB>::kExact ? 0 : limb_bits(*c.binmax);
    const int ew = c.ex[j];
    const int ed = j >= 1 ? c.ex[c.m + j] : kNoExp;
    const int ey = c.ex[2 * c.m];
    const double sig_j = c.stepsc[4 * (size_t)j];
    const int jm = j - 1;
    const int i0 = max(0, jm - c.k + 1);
    const int nw = jm - i0 + 1;
    const double *cf = c.coef + (size_t)max(jm, 0) * kCoef;
    const double sig_jm = j >= 1 ? c.stepsc[4 * (size_t)jm] : 0.0;
    const int per = (s + G - 1) / G;
    const int b0 = blockIdx.x * per, b1 = min(s, b0 + per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = b0 + warp; i < b1; i += blockDim.x / 32) {
        double sw = 0.0;
        if (ew != kNoExp) sw = ldexp(warp_sum_i64_exact(c.skWp + i, c.G_spmv, (size_t)s), ew - P);
        double sd = 0.0;
        if (!Store<TB>::kExact && ed != kNoExp) sd = ldexp(warp_sum_i64_exact(c.skDp + i, c.G_upd, (size_t)s), ed - Ld);
        double sy = 0.0;
        if (last && ey != kNoExp) sy = ldexp(warp_sum_i64_exact(c.skYp + i, c.G_spmv, (size_t)s), ey - P);
        if (lane == 0) {
            c.skw[(size_t)j * s + i] = sw;
            c.SV[i + (size_t)j * s] = sig_j * sw * c.inv_sqrt_zeta;
            if (j >= 1) {
                // sigma_{j-1} y_{j-1} = (w_j - residual) + sum_i h_i,j-1 sigma_i w_i, FP32 coefficients cf
                double u = sw - sd;
                for (int a = 0; a < nw; ++a) u += cf[1 + a] * c.skw[(size_t)(i0 + a) * s + i];
                c.SAV[i + (size_t)jm * s] = (u / cf[0]) * sig_jm * c.inv_sqrt_zeta;
            }
            if (last) c.SAV[i + (size_t)j * s] = sig_j * sy * c.inv_sqrt_zeta;
        }
    }
}

template <int KW, int ZCAP, typename TB>
__global__ void __launch_bounds__(kSpmvThreads, 1) k_arnoldi_spmv_lp(LpCtx c, int j) {
    extern __shared__ int bins[];   // [4 s]: two limbs of S w_j, then two limbs of S y_{m-1} (last step)
    __shared__ double red[BlockSumTraits<KW, kSpmvThreads>::kSmem];
    // stopped at an earlier step
    if (c.iscal[0] && c.iscal[3] < j) return;
    const int s = c.sp.s;
    const TB *V = (const TB *)c.V;
    const double *sc_j = c.stepsc + 4 * (size_t)j;
    if (j >= 1 && blockIdx.x == 0 && threadIdx.x == 0) c.H[j + (size_t)(j - 1) * (c.m + 1)] = sc_j[1];
    // zero right-hand side (j = 0) or happy breakdown, decided by the previous
    // launch: m_eff = j.  S w_j is still formed (S y_{j-1} needs it).
    const bool stopping = sc_j[2] != 0.0;
    if (stopping) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c.iscal[0] = 1;
            c.iscal[1] = j;
            c.iscal[3] = j;
            if (j == 0) c.iscal[2] = SKF_ERR_ZERO_RHS;
        }
        if (j == 0 || c.identity) return;
    }
    const bool last = (j == c.m - 1) && !stopping;

    const double sigma = sc_j[0];
    const double wmax = c.fin_w[2 * (size_t)j + 1];
    const int ew = wmax > 0.0 ? bound_exponent(wmax) : kNoExp;
    const double ybound = c.norm_inf * wmax * (1.0 + 1.0 / 1024.0);   // margin for the FP32 row sums
    const int ey = (last && ybound > 0.0) ? bound_exponent(ybound) : kNoExp;
    const int L = c.identity ? 0 : limb_bits(*c.binmax_chunk);
    const int P = sketch_fraction_bits_from_limb(L);
    const long long lmask = (1ll << L) - 1;
    const int shift_w = P - (ew == kNoExp ? 0 : ew);
    const int shift_y = P - (ey == kNoExp ? 0 : ey);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c.ex[j] = ew;
        if (last) c.ex[2 * c.m] = ey;
    }
    int *aw0 = bins, *aw1 = bins + s, *ay0 = bins + 2 * s, *ay1 = bins + 3 * s;
    if (!c.identity)
        for (int i = threadIdx.x; i < (last ? 4 : 2) * s; i += kSpmvThreads) bins[i] = 0;
    __syncthreads();

    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;
    float acc[KW];
#pragma unroll
    for (int a = 0; a < KW; ++a) acc[a] = 0.f;
    unsigned ykey = 0;
    const TB *wj = V + (size_t)j * c.ldv;
    const int lane = threadIdx.x & 31;
    const int64_t nch = (c.n + kChunkRows - 1) / kChunkRows;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int64_t rw = ch * kChunkRows + (threadIdx.x & ~31);   // first row of the warp's slice
        if (rw >= c.n) continue;                                    // whole warp
        const int64_t t = rw >> 5;
        int wt = 0;
        long long so = 0;
        if (lane == 0 && !stopping) {
            wt = __ldg(c.sell_w + t);
            so = __ldg(c.sell_off + t);
        }
        wt = __shfl_sync(0xffffffffu, wt, 0);
        so = __shfl_sync(0xffffffffu, so, 0);
        const int64_t r = rw + lane;
        if (r >= c.n) continue;   // no warp-collective operation below
        const int64_t base = so + lane;
        float y = 0.f;
        // eight entries of the row in flight at a time
        for (int p0 = 0; p0 < wt; p0 += 8) {
            float av[8], xv[8];
            int cv[8];
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p0 + p < wt) {
                    const int64_t o = base + 32ll * (p0 + p);
                    av[p] = __ldcs(c.sell_val + o);
                    cv[p] = __ldcs(c.sell_col + o);
                }
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p0 + p < wt) xv[p] = Store<TB>::ld(wj + cv[p]);
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p0 + p < wt) y = fmaf(av[p], xv[p], y);
        }
        float wv[KW];
#pragma unroll
        for (int a = 0; a < KW; ++a)
            wv[a] = (a < nw && (!stopping || a == nw - 1)) ? Store<TB>::ld(V + (size_t)(i0 + a) * c.ldv + r) : 0.f;
        float wjr = wv[0];
#pragma unroll
        for (int a = 1; a < KW; ++a)
            if (a == nw - 1) wjr = wv[a];
        if (!stopping) {
            c.Y[r] = y;
#pragma unroll
            for (int a = 0; a < KW; ++a)
                if (a < nw) acc[a] = fmaf(wv[a], y, acc[a]);
            ykey = max(ykey, abs_key_f32(y));
        }
        if (c.identity) {
            c.SV[r + (size_t)j * s] = sigma * (double)wjr;
            c.SAV[r + (size_t)j * s] = sigma * (double)y;
        } else {
            uint16_t e[ZCAP];
            load_pattern<ZCAP>(c.pattern, c.sp.zeta, r, e);
            const long long vw = ew == kNoExp ? 0 : fixed_point_f32(wjr, shift_w);
            const int w0 = (int)(vw & lmask), w1 = (int)(vw >> L);
            const long long vy = last && ey != kNoExp ? fixed_point_f32(y, shift_y) : 0;
            const int y0 = (int)(vy & lmask), y1 = (int)(vy >> L);
#pragma unroll
            for (int q = 0; q < ZCAP; ++q) {
                if (q < c.sp.zeta) {
                    int row;
                    bool neg;
                    pattern_entry(c.sp, e[q], q, row, neg);
                    red_limbs(aw0, aw1, row, w0, w1, neg);
                    if (last) red_limbs(ay0, ay1, row, y0, y1, neg);
                }
            }
        }
    }
    if (!c.identity) {
        __syncthreads();
        long long *ow = c.skWp + (size_t)blockIdx.x * s, *oy = c.skYp + (size_t)blockIdx.x * s;
        for (int i = threadIdx.x; i < s; i += kSpmvThreads) {
            ow[i] = combine_limbs(aw0[i], aw1[i], L);
            if (last) oy[i] = combine_limbs(ay0[i], ay1[i], L);
        }
    }
    if (stopping) return;
    double accd[KW];
#pragma unroll
    for (int a = 0; a < KW; ++a) accd[a] = (double)acc[a];
    block_sum_auto<KW, kSpmvThreads>(accd, red);
    const unsigned ymk = (unsigned)block_max_key<kSpmvThreads>((unsigned long long)ykey, (unsigned long long *)red);
    if (threadIdx.x == 0) {
        double *o = c.p1 + (size_t)blockIdx.x * kP1;
        for (int a = 0; a < KW; ++a) o[a] = accd[a];
        o[kP1 - 1] = (double)__uint_as_float(ymk);
    }
    if (last_to_arrive(c.cnt)) {
        const int warp = threadIdx.x >> 5, lane2 = threadIdx.x & 31;
        for (int v = warp; v <= nw; v += kSpmvThreads / 32) {
            const int slot = (v < nw) ? v : kP1 - 1;
            const double r = warp_reduce_partials(c.p1 + slot, gridDim.x, kP1, slot == kP1 - 1);
            if (lane2 == 0) c.fin_d[(size_t)j * kP1 + slot] = r;
        }
        if (threadIdx.x == 0) c.cnt[0] = 0u;
    }
}

template <int KW, int ZCAP, typename TB>
__global__ void __launch_bounds__(kUpdThreads) k_arnoldi_update_lp(LpCtx c, int j) {
    extern __shared__ int bins[];   // [s]: one limb of the BF16 residual sketch
    __shared__ double red[BlockSumTraits<KW + 1, kUpdThreads>::kSmem];
    __shared__ double sh[kMaxK];     // MGS coefficients h_ij
    __shared__ float scf[kMaxK];     // h_ij sigma_i in FP32, as applied
    __shared__ float sigf_s;
    // stopped at an earlier step; at the stopping step only the sketches are finalised
    if (c.iscal[0] && c.iscal[3] < j) return;
    if (!c.identity) finalize_sketches<TB>(c, j, j == c.m - 1 && !c.iscal[0]);
    if (c.iscal[0]) return;
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
    __syncthreads();
    const float sigf = sigf_s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c.vscale[j] = sigma;
        double *cf = c.coef + (size_t)j * kCoef;
        cf[0] = (double)sigf;
        for (int a = 0; a < nw; ++a) cf[1 + a] = (double)scf[a];
        if (j < c.m - 1)
            for (int a = 0; a < nw; ++a) c.H[(i0 + a) + (size_t)j * (c.m + 1)] = sh[a];
    }
    const bool do_update = j < c.m - 1;
    if (!do_update) return;
    // one-limb fixed point for the BF16 residual: |bf16(w) - w| <= 2^-8 |w|
    // and |w| <= sigma_j max|y_j| + sum_i |h_ij sigma_i| max|w_i|
    const bool resid = !Store<TB>::kExact && !c.identity;
    int ed = kNoExp;
    const int Ld = resid ? limb_bits(*c.binmax) : 0;
    if (resid) {
        double wb = (double)sigf * ymax;
        for (int a = 0; a < nw; ++a) wb += fabs((double)scf[a]) * c.fin_w[2 * (size_t)(i0 + a) + 1];
        const double db = wb * (1.0 / 256.0) * (1.0 + 1.0 / 1024.0);
        ed = db > 0.0 ? bound_exponent(db) : kNoExp;
        for (int i = threadIdx.x; i < s; i += kUpdThreads) bins[i] = 0;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) c.ex[c.m + j + 1] = ed;
    const int shift_d = Ld - (ed == kNoExp ? 0 : ed);

    const int ng = min(j + 1, c.k - 1);
    float part[KW + 1];
#pragma unroll
    for (int i = 0; i <= KW; ++i) part[i] = 0.f;
    unsigned nkey = 0;
    const int64_t r0 = (int64_t)blockIdx.x * c.rows_per_cta;
    const int64_t r1 = min(c.n, r0 + c.rows_per_cta);
    TB *wn = V + (size_t)(j + 1) * c.ldv;
    constexpr int U = 4;
    for (int64_t rb = r0 + threadIdx.x; rb < r1; rb += U * kUpdThreads) {
        float yv[U], wv[U][KW];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = rb + (int64_t)u * kUpdThreads;
            const bool ok = r < r1;
            yv[u] = ok ? c.Y[r] : 0.f;
#pragma unroll
            for (int a = 0; a < KW; ++a)
                wv[u][a] = (ok && a < nw) ? Store<TB>::ld(V + (size_t)(i0 + a) * c.ldv + r) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = rb + (int64_t)u * kUpdThreads;
            if (r < r1) {
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
                    const long long vd = fixed_point_f32(wr - w, shift_d);
                    uint16_t e[ZCAP];
                    load_pattern<ZCAP>(c.pattern, c.sp.zeta, r, e);
#pragma unroll
                    for (int q = 0; q < ZCAP; ++q)
                        if (q < c.sp.zeta) {
                            int row;
                            bool neg;
                            pattern_entry(c.sp, e[q], q, row, neg);
                            atomicAdd(bins + row, neg ? -(int)vd : (int)vd);
                        }
                }
            }
        }
    }
    double partd[KW + 1];
#pragma unroll
    for (int i = 0; i <= KW; ++i) partd[i] = (double)part[i];
    block_sum_auto<KW + 1, kUpdThreads>(partd, red);
    const unsigned nmk = (unsigned)block_max_key<kUpdThreads>((unsigned long long)nkey, (unsigned long long *)red);
    if (threadIdx.x == 0) {
        double *o = c.p2 + (size_t)blockIdx.x * kP2;
        o[0] = partd[0];
        o[1] = (double)__uint_as_float(nmk);
        for (int a = 0; a < KW; ++a) o[2 + a] = partd[1 + a];
    }
    if (resid) {
        __syncthreads();
        long long *od = c.skDp + (size_t)blockIdx.x * s;
        for (int i = threadIdx.x; i < s; i += kUpdThreads) od[i] = (long long)bins[i];
    }
    if (last_to_arrive(c.cnt + 1)) {
        const int warp = threadIdx.x >> 5;
        for (int v = warp; v < 2 + nw; v += kUpdThreads / 32) {
            const int d = nw - (v - 2);   // Gram distance of slot v - 2
            if (v >= 2 && (d < 1 || d > ng)) continue;
            const double r = warp_reduce_partials(c.p2 + v, G, kP2, v == 1);
            if ((threadIdx.x & 31) == 0) {
                if (v < 2) c.fin_w[2 * (size_t)(j + 1) + v] = r;
                else c.gram[(size_t)(j + 1) * kMaxK + d] = r;
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
        info->breakdown = (c.iscal[0] != 0 && me > 0) ? 1 : 0;
        info->beta = me > 0 ? 1.0 / c.vscale[0] : 0.0;
        info->eps_est = eps;
    }
}

template <int KW, int ZCAP, typename TB>
void launch_steps(const LpCtx &c, size_t smem_spmv, size_t smem_upd, cudaStream_t st) {
    auto spmv = k_arnoldi_spmv_lp<KW, ZCAP, TB>;
    auto update = k_arnoldi_update_lp<KW, ZCAP, TB>;
    if (smem_spmv > 48 * 1024)
        cudaFuncSetAttribute(spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_spmv);
    if (smem_upd > 48 * 1024)
        cudaFuncSetAttribute(update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_upd);
    for (int j = 0; j < c.m; ++j) {
        spmv<<<c.G_spmv, kSpmvThreads, smem_spmv, st>>>(c, j);
        update<<<c.G_upd, kUpdThreads, smem_upd, st>>>(c, j);
    }
}

template <int ZCAP, typename TB>
void launch_steps_k(const LpCtx &c, size_t s1, size_t s2, cudaStream_t st) {
    if (c.k <= 2) launch_steps<2, ZCAP, TB>(c, s1, s2, st);
    else if (c.k <= 4) launch_steps<4, ZCAP, TB>(c, s1, s2, st);
    else if (c.k <= 8) launch_steps<8, ZCAP, TB>(c, s1, s2, st);
    else launch_steps<16, ZCAP, TB>(c, s1, s2, st);
}

// Host driver: init, m x (spmv, update), eps, info on `st`.
template <typename TB>
skf_status arnoldi_run_lp(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, TB *V, int64_t ldv,
                          double *vscale, double *SV, double *SAV, double *H, int *iscal, skf_info *info,
                          cudaStream_t st) {
    LpCtx c{};
    c.n = A->n;
    c.sell_off = A->sell_off;
    c.sell_w = A->sell_w;
    c.sell_val = (const float *)A->sell_val;
    c.sell_col = A->sell_col;
    c.norm_inf = A->norm_inf;
    c.identity = S->kind == SKF_SKETCH_IDENTITY;
    if (!c.identity) {
        c.sp = make_sparse_sign(S);
        c.pattern = S->pattern;
        c.binmax = S->binmax;
        c.binmax_chunk = S->binmax_chunk;
    }
    c.sp.s = S->s;
    c.sp.zeta = c.identity ? 1 : S->zeta;
    c.inv_sqrt_zeta = 1.0 / sqrt((double)c.sp.zeta);
    c.m = m;
    c.k = k;
    c.V = V;
    c.ldv = ldv;
    c.vscale = vscale;
    c.SV = SV;
    c.SAV = SAV;
    c.H = H;
    c.iscal = iscal;
    row_partition(A->n, &c.G_upd, &c.rows_per_cta);
    chunk_partition(A->n, &c.G_spmv);
    const int G = c.G_upd, Gs = c.G_spmv;
    const int s = S->s;

    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t szY = sizeof(float) * A->n;
    const size_t szP1 = sizeof(double) * (size_t)Gs * kP1;
    const size_t szP2 = sizeof(double) * (size_t)G * kP2;
    const size_t szFd = sizeof(double) * (size_t)m * kP1;
    const size_t szFw = sizeof(double) * (size_t)(m + 1) * 2;
    const size_t szSc = sizeof(double) * (size_t)(m + 1) * 4;
    const size_t szGram = sizeof(double) * (size_t)(m + 1) * kMaxK;
    const size_t szCoef = sizeof(double) * (size_t)m * kCoef;
    const size_t szSk = c.identity ? 0 : sizeof(double) * (size_t)m * s;
    const size_t szSkYp = c.identity ? 0 : sizeof(long long) * (size_t)Gs * s;   // also S w_j partials
    const size_t szSkDp = (c.identity || Store<TB>::kExact) ? 0 : sizeof(long long) * (size_t)G * s;
    const size_t szEx = sizeof(int) * (size_t)(2 * m + 1);
    const size_t szEps = sizeof(double) * (size_t)m;
    const size_t szCnt = sizeof(unsigned) * 4;
    const size_t total = al(szY) + al(szP1) + al(szP2) + al(szFd) + al(szFw) + al(szSc) + al(szGram) + al(szCoef) +
                         al(szSk) + 2 * al(szSkYp) + al(szSkDp) + al(szEx) + al(szEps) + al(szCnt);
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
    c.p1 = (double *)take(szP1);
    c.p2 = (double *)take(szP2);
    c.fin_d = (double *)take(szFd);
    c.fin_w = (double *)take(szFw);
    c.stepsc = (double *)take(szSc);
    c.gram = (double *)take(szGram);
    c.coef = (double *)take(szCoef);
    c.skw = (double *)take(szSk);
    c.skWp = (long long *)take(szSkYp);
    c.skYp = (long long *)take(szSkYp);
    c.skDp = (long long *)take(szSkDp);
    c.ex = (int *)take(szEx);
    c.epscol = (double *)take(szEps);
    c.cnt = (unsigned *)take(szCnt);
    cudaMemsetAsync(c.cnt, 0, szCnt, st);

    const size_t smem_spmv = c.identity ? 0 : sizeof(int) * 4 * (size_t)s;
    const size_t smem_upd = (c.identity || Store<TB>::kExact) ? 0 : sizeof(int) * (size_t)s;
    k_arnoldi_init_lp<TB><<<G, kThreads, 0, st>>>(c, b);
    if (c.sp.zeta <= 8) launch_steps_k<8, TB>(c, smem_spmv, smem_upd, st);
    else launch_steps_k<16, TB>(c, smem_spmv, smem_upd, st);
    k_arnoldi_eps_lp<<<(m + (kThreads / 32) - 1) / (kThreads / 32), kThreads, 0, st>>>(c);
    k_arnoldi_info_lp<<<1, kThreads, 0, st>>>(c, info);
    count_launches(3 + 2ll * m);
    cudaError_t e = cudaGetLastError();
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "reduced-precision Arnoldi kernels");
    return SKF_OK;
}

}  // namespace
}  // namespace lp
}  // namespace skf
