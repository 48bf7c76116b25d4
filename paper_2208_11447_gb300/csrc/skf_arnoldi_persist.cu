// Persistent single-launch form of the k-truncated Arnoldi process
// (Algorithm 2, Sec. 2.2) for sparse-sign sketches, with an FP64 basis or
// (k <= 2) an FP32 one: the kernel is instantiated on the value type T of the
// operator, the basis and the on-chip rows; with T = float the SpMV, the
// update and the per-thread sums run in FP32 (block and grid sums, scalars,
// sketches and H stay FP64), and the update applies the FP32 values of sigma_j
// and of its coefficients, which H and the relation for S A v_j then use.
//
// The whole recurrence (all m steps) runs in one cooperative launch of one
// CTA per SM.  CTA g owns R consecutive rows (whole SELL-32 slices) and keeps
// its rows of the k window vectors w_{j-k+1} .. w_j and of y~ = A w_j in
// shared memory for the whole process.  Per step HBM therefore sees the
// operator, the gathered entries of w_j and the store of w_{j+1}: the window
// is never re-read and y~ never leaves the SM.  A step has two phases, each
// closed by a grid-wide barrier:
//   A  y~ = A w_j on the CTA's rows (gathers from V[:, j]), partial window
//      dots <w_i, y~> and max|y~|;
//   B  MGS coefficients from the reduced dots and the window Gram matrix
//      (identical to MGS in exact arithmetic), w_{j+1} = sigma_j y~ -
//      sum_i h_ij sigma_i w_i, partial ||w_{j+1}||^2, Gram entries of the
//      next window and max|w_{j+1}|; exact fixed-point sketch of w_j.
// Storage is that of the two-kernel path: column j of V holds w_j, a
// positive multiple of v_j, and vscale[j] = 1 / ||w_j||.  When the rows of the
// window and of y~ do not fit in shared memory together but the window does
// (FP64, k <= 2), y~ lives in a global array instead, written in phase A and
// read back in phase B by the same CTA (L2-resident).
//
// S A v_j is not scattered row by row.  The update of step j applied
//   w_{j+1} = sigma_j y~_j - sum_i c_i w_i,
// so S A v_j = sigma_j S y~_j = S w_{j+1} + sum_i c_i S w_i, the sketched
// Arnoldi relation S A V_m = S V_{m+1} H, evaluated with the very
// coefficients c_i the update used.  It differs from a direct sketch of
// A v_j only by the sketch of the update's own rounding (about one unit
// roundoff of ||A v_j||).  The last column (and the column at a happy
// breakdown, where no further vector is formed) is sketched directly.
//
// Cross-CTA sums: per-CTA partials of the dots in global memory, reduced
// after the barrier by every CTA in the same fixed order (deterministic);
// integer sketch partials added with 64-bit global atomics (exact, so the
// order does not matter).  Every barrier wait is bounded by a clock64
// budget: past it the kernel records SKF_ERR_TIMEOUT, and every CTA returns
// at its next barrier.
#include <math.h>

#include <algorithm>

#include "skf_internal.cuh"
#include "skf_step.cuh"

namespace skf {

namespace {

constexpr int kPT = 512;                      // threads per CTA
constexpr int kPNW = kPT / 32;                // warps per CTA
constexpr long long kBarrierBudget = 1ll << 31;   // SM cycles (about one second)

struct PCtx {
    int64_t n;
    int R;                     // rows per CTA (multiple of 32)
    const int64_t *sell_off;
    const int32_t *sell_w;
    const void *sell_val;      // T values (T = double, or float for an FP32 basis)
    const int32_t *sell_col;
    SparseSign sp;
    const uint16_t *pattern;   // [n][zeta]
    const uint8_t *pattern8;   // [n][8] or nullptr
    int p8_block;
    int L, frac;               // fixed-point limb width and fraction bits (sketch)
    double sk_scale;           // 1 / sqrt(zeta)
    int m, k;
    const double *b;
    void *V;                   // T [m][ldv]
    int64_t ldv;
    double *vscale, *SV, *SAV, *H;
    int *iscal;
    double *pA;                // [KW + 1][G]: window dots, max|y~|
    double *pB;                // [KW + 1][G]: ||w||^2, max|w|, Gram entries
    unsigned long long *accw;  // [m][2][s]: limb sums of S w_j
    unsigned long long *accy;  // [2][s]: limb sums of the directly sketched y~
    double *Sw;                // s x m: S w_j (unnormalised)
    void *ysg;                 // T y~ in global memory ([G][R]) when the rows do not fit with it on chip
    unsigned *bar;             // barrier arrival counter (zeroed before launch)
    int *flag;                 // 1 once a barrier wait ran out
    long long budget;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    return *(const volatile int *)p;
}

// Grid-wide barrier number `nb` (1, 2, ...) of a co-resident grid: arrive,
// then wait until nb * gridDim.x arrivals are visible.  Returns false (in
// every thread of the CTA) if the wait ran out of budget or another CTA's
// did; the first CTA to give up sets *flag.
__device__ bool grid_barrier(unsigned *bar, int *flag, unsigned nb, long long budget) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = nb * gridDim.x;
        const long long t0 = clock64();
        int good = 1;
        while (ld_acquire_u32(bar) < target) {
            if (ld_volatile_i32(flag) != 0 || clock64() - t0 > budget) {
                good = 0;
                break;
            }
            // spin: one thread per CTA polls one L2 line
        }
        if (!good) atomicExch(flag, 1);
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Exact value of a * 2^L + b for int64 a, b (|a| 2^L < 2^94), rounded to
// double (two roundings at most, as warp_sum_i64_exact).
__device__ __forceinline__ double limbs_to_double(long long a1, long long a0, int L) {
    // 128-bit two's complement: hi:lo = a1 << L, then + a0
    unsigned long long lo = (unsigned long long)a1 << L;
    long long hi = (L == 0) ? (a1 < 0 ? -1 : 0) : (a1 >> (64 - L));
    const unsigned long long nlo = lo + (unsigned long long)a0;
    hi += (a0 < 0 ? -1 : 0) + (nlo < lo ? 1 : 0);
    lo = nlo;
    const bool neg = hi < 0;
    unsigned long long uhi = (unsigned long long)hi;
    if (neg) {
        lo = ~lo + 1ull;
        uhi = ~uhi + (lo == 0ull ? 1ull : 0ull);
    }
    const double r = (double)uhi * 18446744073709551616.0 + (double)lo;
    return neg ? -r : r;
}

constexpr int kMaxG = 160;   // partial-table rows one warp reduces with hoisted loads (G <= SMs)

// Sum (or max) of p[0 .. G) in a fixed order, by one warp: every lane loads
// its (at most five) entries at once, adds them in index order, then a
// butterfly; the result is returned to every lane.  The same order in every
// CTA, so all CTAs obtain bitwise the same total.
__device__ __forceinline__ double reduce_slot(const double *p, int G, bool is_max) {
    const int lane = threadIdx.x & 31;
    double v[kMaxG / 32];
#pragma unroll
    for (int i = 0; i < kMaxG / 32; ++i) v[i] = (lane + 32 * i < G) ? __ldcg(p + lane + 32 * i) : 0.0;
    double acc = v[0];
#pragma unroll
    for (int i = 1; i < kMaxG / 32; ++i) acc = is_max ? fmax(acc, v[i]) : acc + v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = is_max ? fmax(acc, t) : acc + t;
    }
    return acc;
}

// Block sums of NV values (one per thread) and the block max of a magnitude
// key, delivered to thread 0.  The FP64 pipe of this part retires one warp
// instruction per 16 SM cycles whatever the active lanes, so the sums use
// full-width adds: values are parked in shared memory and four warps per
// value (one per SM sub-partition) add 128 of them each (4 per lane in index
// order, then a butterfly); thread 0 adds the four quarter sums in order.
// smem: NV * kPT + 4 * NV doubles + kPNW keys.
template <int NV>
__device__ __forceinline__ unsigned long long block_reduce_t0(double (&v)[NV], unsigned long long key, double *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *qs = smem + NV * kPT;
    unsigned long long *ks = (unsigned long long *)(qs + 4 * NV);
#pragma unroll
    for (int i = 0; i < NV; ++i) smem[i * kPT + tid] = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
    if (lane == 0) ks[warp] = key;
    __syncthreads();
    if (warp < 4 * NV) {
        const double *p = smem + (warp >> 2) * kPT + (warp & 3) * 128 + lane;
        double a = ((p[0] + p[32]) + p[64]) + p[96];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) qs[warp] = a;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = ((qs[4 * i] + qs[4 * i + 1]) + qs[4 * i + 2]) + qs[4 * i + 3];
        key = ks[0];
#pragma unroll
        for (int w = 1; w < kPNW; ++w) key = max(key, ks[w]);
    }
    return key;
}

// Fixed-point limbs of one value into the shared bins of the sparse-sign
// rows of row r (pattern8: one 8-byte entry per row, prefetched).
template <int ZCAP>
__device__ __forceinline__ void scatter_row(const PCtx &c, int64_t r, uint2 pv, bool p8, int *b0, int *b1, int l0,
                                            int l1) {
    if (p8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = (int)__byte_perm(q < 4 ? pv.x : pv.y, 0u, 0x4440u + (q & 3));
            const bool neg = e >= c.p8_block;
            red_limbs(b0, b1, c.sp.start[q] + (neg ? e - c.p8_block : e), l0, l1, neg);
        }
    } else {
        uint16_t e[ZCAP];
        load_pattern<ZCAP>(c.pattern, c.sp.zeta, r, e);
#pragma unroll
        for (int q = 0; q < ZCAP; ++q) {
            if (q < c.sp.zeta) {
                int row;
                bool neg;
                pattern_entry(c.sp, e[q], q, row, neg);
                red_limbs(b0, b1, row, l0, l1, neg);
            }
        }
    }
}

// y~ = A w on this CTA's rows into ys[] by the kSpmvWarps SpMV warps, warp
// w taking slices w, w + kSpmvWarps, ... (a fixed assignment, so every lane
// accumulates the same rows in every run: the dot products are bitwise
// reproducible), with the window dots acc[a] = <w_{i0+a}, y~> (soff: slot
// offsets of the window in win[], nw of them) and the magnitude key of
// max|y~|.  Entries of one row are summed in their SELL (= CSR) order.
constexpr int kSpmvWarps = kPNW - 1;   // the last warp serves the reductions
template <int KW, int W, typename T>
__device__ __forceinline__ void spmv_rows(const PCtx &c, const T *__restrict__ wsrc, const T *win,
                                          const int (&soff)[KW], int nw, T *ys, const long long *meta_o,
                                          const int *meta_w, int nsl, int nr, T (&acc)[KW],
                                          unsigned long long &ykey) {
    const T *sell_val = (const T *)c.sell_val;
    const int lane = threadIdx.x & 31;
    int next_t = threadIdx.x >> 5;
    auto grab = [&]() {
        const int t = next_t;
        next_t += kSpmvWarps;
        return t;
    };
    if constexpr (W > 0) {
        // three-stage pipeline: values and gathers of slice tn and column
        // indices of slice tnn are in flight while slice t is computed
        int t = grab();
        int wt = t < nsl ? meta_w[t] : 0;
        int cv[W];
        {
            const int32_t *pc = c.sell_col + (t < nsl ? meta_o[t] : 0) + lane;
#pragma unroll
            for (int p = 0; p < W; ++p) cv[p] = p < wt ? __ldcs(pc + 32 * p) : 0;
        }
        T av[W], xv[W];
        {
            const T *pv = sell_val + (t < nsl ? meta_o[t] : 0) + lane;
#pragma unroll
            for (int p = 0; p < W; ++p) {
                av[p] = p < wt ? __ldcs(pv + 32 * p) : T(0);
                xv[p] = p < wt ? __ldcg(wsrc + cv[p]) : T(0);
            }
        }
        int tn = t < nsl ? grab() : nsl;
        int wtn = tn < nsl ? meta_w[tn] : 0;
        int cvn[W];
        {
            const int32_t *pc = c.sell_col + (tn < nsl ? meta_o[tn] : 0) + lane;
#pragma unroll
            for (int p = 0; p < W; ++p) cvn[p] = p < wtn ? __ldcs(pc + 32 * p) : 0;
        }
        while (t < nsl) {
            T avn[W], xvn[W];
            {
                const T *pv = sell_val + (tn < nsl ? meta_o[tn] : 0) + lane;
#pragma unroll
                for (int p = 0; p < W; ++p) {
                    avn[p] = p < wtn ? __ldcs(pv + 32 * p) : T(0);
                    xvn[p] = p < wtn ? __ldcg(wsrc + cvn[p]) : T(0);
                }
            }
            const int tnn = tn < nsl ? grab() : nsl;
            const int wtnn = tnn < nsl ? meta_w[tnn] : 0;
            int cvnn[W];
            {
                const int32_t *pc = c.sell_col + (tnn < nsl ? meta_o[tnn] : 0) + lane;
#pragma unroll
                for (int p = 0; p < W; ++p) cvnn[p] = p < wtnn ? __ldcs(pc + 32 * p) : 0;
            }
            const int lr = t * 32 + lane;
            if (lr < nr) {
                T y = T(0);
#pragma unroll
                for (int p = 0; p < W; ++p)
                    if (p < wt) y = fma(av[p], xv[p], y);
                ys[lr] = y;
#pragma unroll
                for (int a = 0; a < KW; ++a)
                    if (a < nw) acc[a] = fma(win[soff[a] + lr], y, acc[a]);
                ykey = max(ykey, abs_key((double)y));
            }
            t = tn;
            wt = wtn;
            tn = tnn;
            wtn = wtnn;
#pragma unroll
            for (int p = 0; p < W; ++p) {
                av[p] = avn[p];
                xv[p] = xvn[p];
                cvn[p] = cvnn[p];
            }
        }
    } else {
        // slices wider than 8: one row per lane, entries in a loop
        for (int t = grab(); t < nsl; t = grab()) {
            const int lr = t * 32 + lane;
            const int wt = meta_w[t];
            const long long o = meta_o[t] + lane;
            T y = T(0);
            for (int p = 0; p < wt; ++p)
                y = fma(__ldcs(sell_val + o + 32 * p), __ldcg(wsrc + __ldcs(c.sell_col + o + 32 * p)), y);
            if (lr < nr) {
                ys[lr] = y;
#pragma unroll
                for (int a = 0; a < KW; ++a)
                    if (a < nw) acc[a] = fma(win[soff[a] + lr], y, acc[a]);
                ykey = max(ykey, abs_key((double)y));
            }
        }
    }
}

// T = double: the FP64 basis; T = float: an FP32 basis with FP32 SpMV,
// orthogonalisation and accumulation, the update applying the FP32 values of
// sigma_j and of the MGS coefficients (H and S A v_j are those of the relation
// with the applied values), everything else FP64.
template <int KW, int W, int ZCAP, bool YG, typename T>
__global__ void __launch_bounds__(kPT, 1) k_arnoldi_persist(PCtx c) {
    constexpr bool F32 = sizeof(T) == 4;
    extern __shared__ __align__(16) unsigned char psm[];
    constexpr int kRed = KW * kPT + 4 * KW + kPNW;   // block_reduce_t0<KW>
    constexpr int kSvc = kPNW - 1;                   // the service warp
    const int G = gridDim.x, g = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = c.R, k = c.k, m = c.m, s = c.sp.s;
    const int64_t r0 = (int64_t)g * R;
    const int nr = (int)min((int64_t)R, c.n - r0);          // rows of this CTA (>= 1)
    const int nsl = (nr + 31) >> 5;                          // slices of this CTA
    T *win = (T *)psm;                                       // [k][R]: w_i at slot i % k
    T *Vb = (T *)c.V;
    // [R] y~ of this CTA's rows: shared memory, or (YG) this CTA's slice of a
    // global array, read back by the same CTA after a block barrier (L2)
    T *ys = YG ? (T *)c.ysg + r0 : win + (size_t)k * R;
    double *red = (double *)(YG ? win + (size_t)k * R : ys + R);   // block reductions (R: multiple of 32)
    double *tp = red + kRed;                                 // [KW][kPT] per-thread norm / Gram partials
    unsigned long long *tk = (unsigned long long *)(tp + KW * kPT);   // [kPT] per-thread max|w| keys
    long long *meta_o = (long long *)(tk + kPT);             // [nsl] slice offsets
    int *meta_w = (int *)(meta_o + R / 32);                  // [nsl] slice widths
    int *bins = meta_w + R / 32;                             // [3][2][s]: S w limbs (two buffers), S y limbs
    int *by0 = bins + 4 * s, *by1 = bins + 5 * s;
    const bool p8 = ZCAP == 8 && c.pattern8 != nullptr;
    const long long lmask = (1ll << c.L) - 1;

    // per-step scalars, in rings indexed by step & 3 (k <= 4)
    __shared__ double sig[4];                // sigma_i = 1 / ||w_i||
    __shared__ double sap[4];                // the sigma_i the update of step i applied (FP32: rounded)
    __shared__ double grm[4][kMaxK];         // grm[i & 3][d] = <w_i, w_{i-d}>
    __shared__ double coef[4][kMaxK];        // c_b for w_{i-b} (newest first) of the update of step i
    __shared__ int cnw[4];                   // window length of step i
    __shared__ int ews[4];                   // exponent bound of max|w_i| (its sketch)
    __shared__ int eys[4];                   // exponent bound of max|y~_i|
    __shared__ double sh[kMaxK];             // MGS coefficients h_ij of the current step
    __shared__ double sd[KW + 1];            // reduced dots and max|y~| of the current step
    __shared__ double sb[KW + 1];            // reduced ||w_j||^2, max|w_j|, Gram entries
    __shared__ int sbreak;                   // w_j is a happy breakdown
    unsigned nb = 0;                         // barriers passed

    // Column i of S V and column i-1 of S A V from the integer sums of S w_i
    // (rows is = g + G t of S): S w_i, S v_i = sigma_i S w_i and, by the
    // relation, S A v_{i-1} = S w_i + sum_b c_b S w_{i-1-b}.
    auto finalize_col = [&](int i, int t) {
        const int is = g + G * t;
        if (is >= s) return;
        const unsigned long long *aw = c.accw + (size_t)i * 2 * s;
        const int ew = ews[i & 3];
        double swv = 0.0;
        if (ew != kNoExp)
            swv = scale_pow2(limbs_to_double((long long)__ldcg(aw + s + is), (long long)__ldcg(aw + is), c.L),
                             ew - c.frac) * c.sk_scale;
        c.Sw[is + (size_t)i * s] = swv;
        c.SV[is + (size_t)i * s] = sig[i & 3] * swv;
        if (i >= 1) {
            const int pn = cnw[(i - 1) & 3];
            double v = swv;
            for (int b2 = pn - 1; b2 >= 0; --b2)
                v = fma(coef[(i - 1) & 3][b2], __ldcg(c.Sw + is + (size_t)(i - 1 - b2) * s), v);
            // the update applied sap y~ (= sigma y~ in FP64): S A v = (sigma / sap) (...)
            if constexpr (F32) v *= sig[(i - 1) & 3] / sap[(i - 1) & 3];
            c.SAV[is + (size_t)(i - 1) * s] = v;
        }
    };
    // S A v_i sketched directly from y~_i (limb sums in accy)
    auto finalize_direct = [&](int i, int t) {
        const int is = g + G * t;
        if (is >= s) return;
        const int ey = eys[i & 3];
        double v = 0.0;
        if (ey != kNoExp)
            v = scale_pow2(limbs_to_double((long long)__ldcg(c.accy + s + is), (long long)__ldcg(c.accy + is), c.L),
                           ey - c.frac) * c.sk_scale * sig[i & 3];
        c.SAV[is + (size_t)i * s] = v;
    };
    // add this CTA's S w_i limb bins (buffer i & 1) to accw[i], then clear them
    auto flush_w = [&](int i, int t0, int dt) {
        int *b0 = bins + (i & 1) * 2 * s, *b1 = b0 + s;
        unsigned long long *aw = c.accw + (size_t)i * 2 * s;
        for (int x = t0; x < s; x += dt) {
            atomicAdd(aw + x, (unsigned long long)(long long)b0[x]);
            atomicAdd(aw + s + x, (unsigned long long)(long long)b1[x]);
            b0[x] = 0;
            b1[x] = 0;
        }
    };
    auto flush_y = [&](int t0, int dt) {
        for (int x = t0; x < s; x += dt) {
            atomicAdd(c.accy + x, (unsigned long long)(long long)by0[x]);
            atomicAdd(c.accy + s + x, (unsigned long long)(long long)by1[x]);
        }
    };

    // ---- set-up: slice metadata, bins, H = 0, iscal, w_0 = b
    for (int t = tid; t < nsl; t += kPT) {
        meta_o[t] = c.sell_off[r0 / 32 + t];
        meta_w[t] = c.sell_w[r0 / 32 + t];
    }
    for (int i = tid; i < 6 * s; i += kPT) bins[i] = 0;
    for (int64_t i = (int64_t)g * kPT + tid; i < (int64_t)(m + 1) * m; i += (int64_t)G * kPT) c.H[i] = 0.0;
    if (g == 0 && tid == 0) {
        c.iscal[0] = 0;
        c.iscal[1] = m;
        c.iscal[2] = SKF_OK;
        c.iscal[3] = m;
    }
    if (tid == 0) sbreak = 0;
    {
        double nrm[1] = {0.0};
        unsigned long long key = 0;
        for (int lr = tid; lr < nr; lr += kPT) {
            const T xt = (T)c.b[r0 + lr];
            const double x = (double)xt;
            Vb[r0 + lr] = xt;
            win[lr] = xt;    // slot 0
            nrm[0] = fma(x, x, nrm[0]);
            key = max(key, abs_key(x));
        }
        key = block_reduce_t0<1>(nrm, key, red);
        if (tid == 0) {
            c.pB[g] = nrm[0];
            c.pB[G + g] = key_to_abs(key);
        }
    }
    if (!grid_barrier(c.bar, c.flag, ++nb, c.budget)) goto timeout;
    if (warp < 2) {
        const double v = reduce_slot(c.pB + (size_t)warp * G, G, warp == 1);
        if (lane == 0) sb[warp] = v;
    }
    __syncthreads();
    if (!(sb[0] > 0.0)) {   // zero right-hand side: x = 0
        if (g == 0 && tid == 0) {
            c.iscal[0] = 1;
            c.iscal[1] = 0;
            c.iscal[2] = SKF_ERR_ZERO_RHS;
            c.iscal[3] = 0;
        }
        return;
    }
    if (tid == 0) {
        sig[0] = rsqrt(sb[0]);
        sap[0] = F32 ? (double)(float)sig[0] : sig[0];
        ews[0] = positive_finite(sb[1]) ? bound_exponent(sb[1]) : kNoExp;
        if (g == 0) c.vscale[0] = sig[0];
    }
    __syncthreads();

    for (int j = 0; j < m; ++j) {
        const int i0 = max(0, j - k + 1);
        const int nw = j - i0 + 1;
        const bool last = j == m - 1;
        const int ngj = min(j, k - 1);       // Gram distances of w_j
        // ---- phase A: y~ = A w_j and the window dots (kSpmvWarps warps).
        // Meanwhile the service warp reduces this CTA's partial norms of w_j
        // (left by phase B of the previous step), adds the CTA's S w_{j-1}
        // bins to the global sums and finalises the sketch columns of step
        // j - 2: none of it is needed before the barrier, and phase A does not
        // need the norm of w_j (stored unnormalised).
        T acc[KW];
#pragma unroll
        for (int a = 0; a < KW; ++a) acc[a] = T(0);
        unsigned long long ykey = 0;
        if (warp == kSvc && j >= 1) {
            double v[KW];
#pragma unroll
            for (int q = 0; q < KW; ++q) {
                v[q] = 0.0;
                if (q <= ngj) {
#pragma unroll 4
                    for (int t = lane; t < kPT; t += 32) v[q] += tp[q * kPT + t];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
                }
            }
            unsigned long long kk = 0;
            for (int t = lane; t < kPT; t += 32) kk = max(kk, tk[t]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) kk = max(kk, __shfl_xor_sync(0xffffffffu, kk, o));
            if (lane == 0) {
                c.pB[g] = v[0];
                c.pB[G + g] = key_to_abs(kk);
#pragma unroll
                for (int d = 1; d < KW; ++d)
                    if (d <= ngj) c.pB[(size_t)(1 + d) * G + g] = v[d];
            }
            flush_w(j - 1, lane, 32);
            if (j >= 2)
                for (int t = lane; g + G * t < s; t += 32) finalize_col(j - 2, t);
            __syncwarp();
        }
        {
            int soff[KW];   // window slot offsets, oldest first
#pragma unroll
            for (int a = 0; a < KW; ++a) soff[a] = a < nw ? ((i0 + a) % k) * R : 0;
            if (warp < kSpmvWarps)
                spmv_rows<KW, W, T>(c, Vb + (size_t)j * c.ldv, win, soff, nw, ys, meta_o, meta_w, nsl, nr, acc, ykey);
        }
        double accd[KW];
#pragma unroll
        for (int a = 0; a < KW; ++a) accd[a] = (double)acc[a];
        ykey = block_reduce_t0<KW>(accd, ykey, red);
        if (tid == 0) {
#pragma unroll
            for (int a = 0; a < KW; ++a)
                if (a < nw) c.pA[(size_t)a * G + g] = accd[a];
            c.pA[(size_t)KW * G + g] = key_to_abs(ykey);
        }
        if (!grid_barrier(c.bar, c.flag, ++nb, c.budget)) goto timeout;

        // ---- totals: dots and max|y~| of this step; ||w_j||, max|w_j| and the
        // Gram entries of w_j (every CTA, identically)
        if (warp <= nw) {
            const int slot = warp < nw ? warp : KW;
            const double v = reduce_slot(c.pA + (size_t)slot * G, G, slot == KW);
            if (lane == 0) sd[slot] = v;
        } else if (j >= 1 && warp - nw - 1 < 2 + ngj) {
            const int q = warp - nw - 1;
            const double v = reduce_slot(c.pB + (size_t)q * G, G, q == 1);
            if (lane == 0) sb[q] = v;
        }
        __syncthreads();
        if (tid == 0) {
            if (j >= 1) {
                // ||A v_{j-1}||^2 = sum_i h_i^2 + ||w_j||^2 for the orthonormal window;
                // happy breakdown when ||w_j|| <= 1e-12 ||A v_{j-1}||
                // (compared in squares, and sigma = 1/||w_j|| from one rsqrt: an FP64
                // square root or division is ~650 dependent cycles on this part)
                const double n2 = sb[0];
                double hs = 0.0;
                for (int a = 0; a < cnw[(j - 1) & 3]; ++a) hs = fma(sh[a], sh[a], hs);
                // (FP32: ||w_j|| <= 2^-17 ||A v_{j-1}||, 64 FP32 unit roundoffs)
                sbreak = (n2 > (F32 ? 5.820766091346741e-11 : 1e-24) * (hs + n2)) ? 0 : 1;
                const double sgm = n2 > 0.0 ? rsqrt(n2) : 0.0;
                const double hn = n2 * sgm;
                if (!sbreak) {   // w_j enters the window
                    sig[j & 3] = sgm;
                    sap[j & 3] = F32 ? (double)(float)sgm : sgm;
                    for (int d = 1; d <= ngj; ++d) grm[j & 3][d] = sb[1 + d];
                    ews[j & 3] = positive_finite(sb[1]) ? bound_exponent(sb[1]) : kNoExp;
                }
                if (g == 0) {
                    // FP32: the coefficient of v_j in A v_{j-1} with the applied sigma_{j-1}
                    c.H[j + (size_t)(j - 1) * (m + 1)] =
                        F32 ? sig[(j - 1) & 3] * hn / sap[(j - 1) & 3] : hn;
                    if (!sbreak) c.vscale[j] = sgm;
                }
            }
            if (!sbreak) {
                // MGS in the window, ascending, from the dots and the Gram matrix:
                // h_i = <v_i, y> - sum_{i' < i} h_i' <v_i, v_i'>
                const double sj = sig[j & 3];
                for (int a = 0; a < nw; ++a) {
                    const int ia = i0 + a;
                    const double sa = sig[ia & 3];
                    double h = sa * sj * sd[a];
                    for (int b2 = 0; b2 < a; ++b2) {
                        const int ib = i0 + b2;
                        h -= sh[b2] * sa * sig[ib & 3] * grm[ia & 3][ia - ib];
                    }
                    sh[a] = h;
                    coef[j & 3][nw - 1 - a] = F32 ? (double)(float)(h * sa) : h * sa;
                }
                cnw[j & 3] = nw;
                eys[j & 3] = positive_finite(sd[KW]) ? bound_exponent(sd[KW]) : kNoExp;
                // FP32: the relation with the applied (rounded) sigma_j and coefficients
                if (g == 0 && !last)
                    for (int a = 0; a < nw; ++a) {
                        const int ia = i0 + a;
                        c.H[ia + (size_t)j * (m + 1)] =
                            F32 ? sj * coef[j & 3][nw - 1 - a] / (sap[j & 3] * sig[ia & 3]) : sh[a];
                    }
            }
        }
        __syncthreads();

        if (sbreak) {
            // happy breakdown: w_j is rounding noise, the basis ends at m_eff = j.
            // S A v_{j-1} is sketched directly from y~_{j-1} = A w_{j-1}, computed
            // again (bitwise the same: fixed per-row order) into ys[].
            const int jb = j - 1, i0b = max(0, jb - k + 1), nwb = jb - i0b + 1;
            int soff[KW];
#pragma unroll
            for (int a = 0; a < KW; ++a) soff[a] = a < nwb ? ((i0b + a) % k) * R : 0;
            T accb[KW];
#pragma unroll
            for (int a = 0; a < KW; ++a) accb[a] = T(0);
            unsigned long long kb = 0;
            if (warp < kSpmvWarps)
                spmv_rows<KW, W, T>(c, Vb + (size_t)jb * c.ldv, win, soff, 0, ys, meta_o, meta_w, nsl, nr, accb, kb);
            __syncthreads();
            const int ey = eys[jb & 3];
            const int shift_y = c.frac - (ey == kNoExp ? 0 : ey);
            for (int lr = tid; lr < nr; lr += kPT) {
                const int64_t r = r0 + lr;
                const long long vy = ey == kNoExp ? 0 : fixed_point(ys[lr], shift_y);
                const uint2 pv = p8 ? __ldg((const uint2 *)(c.pattern8 + r * 8)) : make_uint2(0u, 0u);
                scatter_row<ZCAP>(c, r, pv, p8, by0, by1, (int)(vy & lmask), (int)(vy >> c.L));
            }
            __syncthreads();
            flush_y(tid, kPT);
            if (!grid_barrier(c.bar, c.flag, ++nb, c.budget)) goto timeout;
            // S v_{j-1}, S A v_{j-2} (S w_{j-1} was added up before the last barrier) and S A v_{j-1}
            for (int t = tid; g + G * t < s; t += kPT) {
                finalize_col(jb, t);
                finalize_direct(jb, t);
            }
            if (g == 0 && tid == 0) {
                c.iscal[0] = 1;
                c.iscal[1] = j;
                c.iscal[3] = j;
            }
            return;
        }

        // ---- phase B: w_{j+1} and this thread's partials of its norm, Gram
        // entries and max; sketch of w_j (and of y~ in the last step)
        {
            const T sj = (T)sap[j & 3];   // sigma_j as applied
            const int ew = ews[j & 3], ey = eys[j & 3];
            const int shift_w = c.frac - (ew == kNoExp ? 0 : ew);
            const int shift_y = c.frac - (ey == kNoExp ? 0 : ey);
            const int ng = min(j + 1, k - 1);
            int *bw0 = bins + (j & 1) * 2 * s, *bw1 = bw0 + s;
            T cf[KW];        // c_b for w_{j-b} (as applied)
            int soffr[KW];   // slot offsets, newest first
#pragma unroll
            for (int b2 = 0; b2 < KW; ++b2) {
                cf[b2] = b2 < nw ? (T)coef[j & 3][b2] : T(0);
                soffr[b2] = b2 < nw ? ((j - b2) % k) * R : 0;
            }
            const int snew = ((j + 1) % k) * R;
            T *wn = Vb + (size_t)(j + 1) * c.ldv;
            T part[KW];
#pragma unroll
            for (int a = 0; a < KW; ++a) part[a] = T(0);
            unsigned long long nkey = 0;
            uint2 pv_next = make_uint2(0u, 0u);
            if (p8 && tid < nr) pv_next = __ldg((const uint2 *)(c.pattern8 + (r0 + tid) * 8));
            for (int lr = tid; lr < nr; lr += kPT) {
                const int64_t r = r0 + lr;
                const uint2 pv = pv_next;
                if (p8 && lr + kPT < nr) pv_next = __ldg((const uint2 *)(c.pattern8 + (r + kPT) * 8));
                const T y = ys[lr];
                T wv[KW];
#pragma unroll
                for (int b2 = 0; b2 < KW; ++b2) wv[b2] = b2 < nw ? win[soffr[b2] + lr] : T(0);
                if (!last) {
                    T w = sj * y;
#pragma unroll
                    for (int b2 = KW - 1; b2 >= 0; --b2)
                        if (b2 < nw) w = fma(-cf[b2], wv[b2], w);   // oldest first
                    wn[r] = w;
                    win[snew + lr] = w;
                    part[0] = fma(w, w, part[0]);
                    nkey = max(nkey, abs_key((double)w));
#pragma unroll
                    for (int d = 1; d < KW; ++d)
                        if (d <= ng) part[d] = fma(w, wv[d - 1], part[d]);
                }
                const long long vw = ew == kNoExp ? 0 : fixed_point(wv[0], shift_w);
                scatter_row<ZCAP>(c, r, pv, p8, bw0, bw1, (int)(vw & lmask), (int)(vw >> c.L));
                if (last) {
                    const long long vy = ey == kNoExp ? 0 : fixed_point(y, shift_y);
                    scatter_row<ZCAP>(c, r, pv, p8, by0, by1, (int)(vy & lmask), (int)(vy >> c.L));
                }
            }
            if (!last) {
#pragma unroll
                for (int a = 0; a < KW; ++a) tp[a * kPT + tid] = (double)part[a];
                tk[tid] = nkey;
            } else {
                __syncthreads();
                flush_w(j, tid, kPT);
                flush_y(tid, kPT);
            }
        }
        if (!grid_barrier(c.bar, c.flag, ++nb, c.budget)) goto timeout;
        if (last) {
            // S v_{m-2}, S v_{m-1}, S A v_{m-3}, S A v_{m-2} (relation), S A v_{m-1} (direct)
            for (int t = tid; g + G * t < s; t += kPT) {
                if (j >= 1) finalize_col(j - 1, t);
                finalize_col(j, t);
                finalize_direct(j, t);
            }
        }
    }
    return;
timeout:
    if (g == 0 && tid == 0) {
        c.iscal[0] = 1;
        c.iscal[1] = 0;
        c.iscal[2] = SKF_ERR_TIMEOUT;
        c.iscal[3] = 0;
    }
}

// | ||S v_j||^2 - 1 | for column j (one CTA per column), folded into a
// maximum with an integer atomic on the bit pattern (non-negative doubles
// order like their bits, so the result does not depend on the order).
__global__ void __launch_bounds__(128) k_persist_eps(const double *__restrict__ SV, int s,
                                                    const int *__restrict__ iscal, unsigned long long *epsmax) {
    __shared__ double red[4];
    const int j = blockIdx.x;
    if (j >= iscal[1]) return;
    double a = 0.0;
    for (int i = threadIdx.x; i < s; i += 128) a = fma(SV[i + (size_t)j * s], SV[i + (size_t)j * s], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double e = fabs(((red[0] + red[1]) + red[2]) + red[3] - 1.0);
        atomicMax(epsmax, (unsigned long long)__double_as_longlong(e));
    }
}

__global__ void k_persist_info(const double *__restrict__ vscale, const int *__restrict__ iscal,
                               const unsigned long long *epsmax, skf_info *info) {
    if (threadIdx.x != 0 || info == nullptr) return;
    const int me = iscal[1];
    info->status = iscal[2];
    info->m_eff = me;
    info->breakdown = (iscal[0] == 1 && me > 0) ? 1 : 0;
    info->beta = me > 0 ? 1.0 / vscale[0] : 0.0;
    info->eps_est = __longlong_as_double((long long)*epsmax);
}

// A barrier that can never complete (it waits for one CTA more than the
// grid has), with the given budget: the self-test of the bounded wait.
__global__ void __launch_bounds__(32) k_barrier_selftest(unsigned *bar, int *flag, long long budget, int *status) {
    // barrier number 2 needs 2 G arrivals; the grid makes G
    const bool ok = grid_barrier(bar, flag, 2, budget);
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = ok ? SKF_OK : SKF_ERR_TIMEOUT;
}

template <int KW, int W, int ZCAP, bool YG, typename T>
cudaError_t launch_persist(const PCtx &c, int G, size_t smem, cudaStream_t st) {
    auto kern = k_arnoldi_persist<KW, W, ZCAP, YG, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1 || G > per_sm * num_sms()) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kPT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, c);
}

template <int KW, int W, bool YG, typename T>
cudaError_t launch_persist_z(const PCtx &c, int G, size_t smem, cudaStream_t st) {
    return c.sp.zeta <= 8 ? launch_persist<KW, W, 8, YG, T>(c, G, smem, st)
                          : launch_persist<KW, W, 16, YG, T>(c, G, smem, st);
}

template <int KW>
cudaError_t launch_persist_w(const PCtx &c, int maxw, int G, size_t smem, cudaStream_t st) {
    if (maxw <= 5) return launch_persist_z<KW, 5, false, double>(c, G, smem, st);
    if (maxw <= 7) return launch_persist_z<KW, 7, false, double>(c, G, smem, st);
    if (maxw <= 8) return launch_persist_z<KW, 8, false, double>(c, G, smem, st);
    return launch_persist_z<KW, 0, false, double>(c, G, smem, st);
}

// y~ in global memory: instantiated for k <= 2 and slices at most 7 wide (the
// 5- and 7-point stencils) only
cudaError_t launch_persist_yg(const PCtx &c, int maxw, int G, size_t smem, cudaStream_t st) {
    if (maxw <= 5) return launch_persist_z<2, 5, true, double>(c, G, smem, st);
    return launch_persist_z<2, 7, true, double>(c, G, smem, st);
}

// FP32 basis: k <= 2, slices at most 7 wide, y~ on chip
cudaError_t launch_persist_f32(const PCtx &c, int maxw, int G, size_t smem, cudaStream_t st) {
    if (maxw <= 5) return launch_persist_z<2, 5, false, float>(c, G, smem, st);
    return launch_persist_z<2, 7, false, float>(c, G, smem, st);
}

// Dynamic shared memory of the persistent kernel for R rows per CTA with
// elements of vb bytes (yg: y~ kept in global memory instead).
size_t persist_smem(int R, int k, int KW, int s, bool yg, size_t vb = sizeof(double)) {
    const size_t red = (size_t)KW * kPT + 4 * KW + kPNW;
    const size_t thread_partials = (size_t)(KW + 1) * kPT;
    return vb * (size_t)(k + (yg ? 0 : 1)) * R + sizeof(double) * (red + thread_partials) +
           (sizeof(long long) + sizeof(int)) * (size_t)(R / 32) + sizeof(int) * 6 * (size_t)s;
}

}  // namespace

// Persistent partition: G = min(SMs, ceil(n / 1024)) CTAs of R rows (whole
// slices).  The sketch tables record the bin-load maximum of this partition.
void persist_partition(int64_t n, int *G, int64_t *rows) {
    int64_t g = (n + 1023) / 1024;
    if (g > num_sms()) g = num_sms();
    if (g < 1) g = 1;
    const int64_t R = ((n + g - 1) / g + 31) / 32 * 32;
    *rows = R;
    *G = (int)((n + R - 1) / R);
}

static int g_step_mode = 0;   // 0 auto, 1 two-kernel path only, 2 persistent path required
void set_step_mode(int mode) { g_step_mode = mode; }
int step_mode() { return g_step_mode; }

// The persistent form for an FP64 basis (f32 = false) or an FP32 one (f32:
// FP32 values, k <= 2, slices at most 7 wide, the window and y~ both on chip:
// N up to about 2e6).
static skf_status run_persistent(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, void *V,
                                 int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                                 skf_info *info, cudaStream_t st, bool f32) {
    if (S->kind != SKF_SKETCH_SPARSE_SIGN || S->binmax_persist == nullptr || k > 4 ||
        A->vdtype != (f32 ? SKF_F32 : SKF_F64) || A->nlong > 0 ||
        A->perm != nullptr)   // a row split or sorted slices take the two-kernel form
        return SKF_ERR_NOT_SUPPORTED;
    if (f32 && (k > 2 || A->max_width > 7)) return SKF_ERR_NOT_SUPPORTED;
    const size_t vb = f32 ? sizeof(float) : sizeof(double);
    int G;
    int64_t R64;
    persist_partition(A->n, &G, &R64);
    if (G > kMaxG) return SKF_ERR_NOT_SUPPORTED;
    const int R = (int)R64;
    const int KW = k <= 2 ? 2 : 4;
    const int s = S->s;
    size_t smem = persist_smem(R, k, KW, s, false, vb);
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return SKF_ERR_NOT_SUPPORTED;
    }
    // static shared arrays of the kernel take about 3 KB; past the per-CTA
    // shared memory the window alone may still fit, with y~ in global memory
    bool yg = false;
    if (smem + 4096 > (size_t)optin) {
        if (f32) return SKF_ERR_NOT_SUPPORTED;   // an FP32 basis keeps y~ on chip
        yg = true;
        smem = persist_smem(R, k, KW, s, true, vb);
        if (KW != 2 || A->max_width > 7 || smem + 4096 > (size_t)optin) return SKF_ERR_NOT_SUPPORTED;
    }
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return SKF_ERR_NOT_SUPPORTED;
    }

    PCtx c{};
    c.n = A->n;
    c.R = R;
    c.sell_off = A->sell_off;
    c.sell_w = A->sell_w;
    c.sell_val = A->sell_val;
    c.sell_col = A->sell_col;
    c.sp = make_sparse_sign(S);
    c.pattern = S->pattern;
    if (S->zeta == 8 && S->pattern8 != nullptr) {
        c.pattern8 = S->pattern8;
        c.p8_block = S->p8_block;
    }
    c.L = limb_bits(S->binmax_persist_host);
    c.frac = sketch_fraction_bits_from_limb(c.L);
    c.sk_scale = 1.0 / sqrt((double)S->zeta);
    c.m = m;
    c.k = k;
    c.b = b;
    c.V = V;
    c.ldv = ldv;
    c.vscale = vscale;
    c.SV = SV;
    c.SAV = SAV;
    c.H = H;
    c.iscal = iscal;
    c.budget = kBarrierBudget;

    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t szP = sizeof(double) * (size_t)(KW + 1) * G;
    const size_t szAw = sizeof(unsigned long long) * (size_t)m * 2 * s;
    const size_t szAy = sizeof(unsigned long long) * 2 * (size_t)s;
    const size_t szSw = sizeof(double) * (size_t)s * m;
    const size_t szBar = 2 * sizeof(int) + sizeof(unsigned long long);   // counter, flag, eps maximum
    const size_t szYs = yg ? vb * (size_t)G * R : 0;
    const size_t total = 2 * al(szP) + al(szAw) + al(szAy) + al(szSw) + al(szBar) + al(szYs);
    char *ws = nullptr;
    skf_status stt = dalloc((void **)&ws, total, st);
    if (stt != SKF_OK) return stt;
    size_t off = 0;
    auto take = [&](size_t sz) {
        char *p = ws + off;
        off += al(sz);
        return p;
    };
    c.pA = (double *)take(szP);
    c.pB = (double *)take(szP);
    c.accw = (unsigned long long *)take(szAw);
    c.accy = (unsigned long long *)take(szAy);
    c.Sw = (double *)take(szSw);
    c.bar = (unsigned *)take(szBar);
    c.ysg = yg ? (void *)take(szYs) : nullptr;
    c.flag = (int *)(c.bar + 1);
    unsigned long long *epsmax = (unsigned long long *)(c.bar + 2);
    // accumulators and the barrier start at zero (one memset: they are adjacent)
    cudaMemsetAsync(c.accw, 0, (size_t)((char *)c.Sw - (char *)c.accw), st);
    cudaMemsetAsync(c.bar, 0, szBar, st);
    cudaError_t e;
    if (f32) e = launch_persist_f32(c, A->max_width, G, smem, st);
    else if (yg) e = launch_persist_yg(c, A->max_width, G, smem, st);
    else if (KW == 2) e = launch_persist_w<2>(c, A->max_width, G, smem, st);
    else e = launch_persist_w<4>(c, A->max_width, G, smem, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        dfree(ws, st);
        if (e == cudaErrorCooperativeLaunchTooLarge) return SKF_ERR_NOT_SUPPORTED;
        return cuda_fail(e, "persistent Arnoldi launch");
    }
    k_persist_eps<<<m, 128, 0, st>>>(SV, s, iscal, epsmax);
    k_persist_info<<<1, 32, 0, st>>>(vscale, iscal, epsmax, info);
    count_launches(3);
    e = cudaGetLastError();
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "persistent Arnoldi kernels");
    return SKF_OK;
}

skf_status arnoldi_run_persistent(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, double *V,
                                  int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                                  skf_info *info, cudaStream_t st) {
    return run_persistent(A, S, b, m, k, V, ldv, vscale, SV, SAV, H, iscal, info, st, false);
}

skf_status arnoldi_run_persistent_f32(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, float *V,
                                      int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                                      skf_info *info, cudaStream_t st) {
    return run_persistent(A, S, b, m, k, V, ldv, vscale, SV, SAV, H, iscal, info, st, true);
}

// Self-test of the bounded barrier wait: a grid of `ctas` co-resident CTAs
// waits at a barrier that can never complete; the wait must give up after
// `budget` SM cycles and report SKF_ERR_TIMEOUT in *status_out (device int).
skf_status barrier_selftest(int ctas, long long budget, int *status_out, cudaStream_t st) {
    char *ws = nullptr;
    skf_status stt = dalloc((void **)&ws, 256, st);
    if (stt != SKF_OK) return stt;
    unsigned *bar = (unsigned *)ws;
    int *flag = (int *)(ws + 4);
    cudaMemsetAsync(ws, 0, 8, st);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_barrier_selftest, bar, flag, budget, status_out);
    count_launches(1);
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "barrier self-test launch");
    return SKF_OK;
}

}  // namespace skf
