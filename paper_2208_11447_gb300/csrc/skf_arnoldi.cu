// k-truncated Arnoldi with on-the-fly sketching (Algorithm 2, Sec. 2.2).
//
// Storage: column j of V holds w_j, a positive multiple of the basis vector
// v_j = sigma_j w_j with sigma_j = 1/||w_j||.  Keeping w_j unnormalised lets
// one step run as two kernels (two grid-wide dependencies per step: the dot
// products before the update, and the new vector before the next SpMV):
//
//   spmv   (step j): y~ = A w_j on the CTA's rows -> Y; partial dots
//                    <w_i, y~> (i in the window) and max|y~|; in its
//                    prologue, S v_{j-1} and S A v_{j-1} from the update's
//                    integer partials.
//   update (step j): MGS coefficients from the reduced dots and the window
//                    Gram matrix (identical to MGS in exact arithmetic),
//                    w_{j+1} = sigma_j y~ - sum_i h_ij sigma_i w_i, partial
//                    ||w_{j+1}||^2, max|w_{j+1}| and the Gram entries
//                    <w_{j+1}, w_i> of the next window; fixed-point sketches
//                    of w_j (-> S v_j) and of y~ (-> S A v_j).
//
// Cross-CTA reductions: every CTA writes its partials; the CTA that arrives
// last (atomic ticket, no waiting) reduces them in a fixed order and publishes
// the totals for the next launch.  Sketch partial sums are integers, reduced
// exactly.  Results therefore do not depend on scheduling.
#include <math.h>

#include <algorithm>

#include "skf_internal.cuh"
#include "skf_step.cuh"

namespace skf {

constexpr int kP1 = kMaxK + 1;    // slots of one spmv partial: d[kMaxK], ymax
constexpr int kP2 = kMaxK + 2;    // slots of one update partial: ||w||^2, max|w|, g[kMaxK]
constexpr int kSpmvThreads = 1024; // threads per CTA of the SpMV kernel: one CTA per SM
constexpr int kUpdThreads = 512;  // threads per CTA of the update kernel

struct ArnCtx {
    int64_t n;
    const int64_t *sell_off;   // SELL-32 operator (see skf_csr)
    const int32_t *sell_w;
    const double *sell_val;
    const int32_t *sell_col;
    int max_width;             // widest SELL slice
    SparseSign sp;
    const uint16_t *pattern;   // expanded sparse-sign pattern [n][zeta]
    const uint8_t *pattern8;   // compact pattern [n][8] when zeta = 8 (row in stripe + p8_block * sign), or nullptr
    int p8_block;              // its sign offset: 64 or 128
    const int *binmax;         // bin-load maximum of the row partition
    int identity;      // S = I
    int sparse;        // sparse-sign S (scattered by the update kernel)
    int srht;          // SRHT S (separate block-transform kernels after each update)
    int direct;        // SRDCT S: S v_j, S A v_j written directly by a kernel after each update
    int sk_parts;      // integer partials per sketch column (update CTAs or SRHT blocks)
    int srht_frac;     // SRHT fixed-point fraction bits
    double sk_scale;   // scale of the integer sums: 1/sqrt(zeta) or 1/sqrt(s)
    int m, k;
    double *V;
    int64_t ldv;
    int vring;         // 0: V holds all m columns; > 0: a ring of vring slots (two-pass)
    int64_t woff[kMaxK];   // element offsets of the window columns i0 .. j of this launch's step (host-filled)
    double *vscale;    // [m]
    double *SV, *SAV;  // s x m
    double *H;         // (m+1) x m
    double *Y;         // [n]
    double *p1;        // [G][kP1] spmv partials
    double *p2;        // [G][kP2] update partials: ||w||^2, max|w|, <w_{j+1}, w_{j+1-d}>
    double *fin_d;     // [m][kP1] reduced spmv partials of step j
    double *fin_w;     // [m+1][2] ||w_j||^2, max|w_j|
    double *stepsc;    // [m+1][4] per-step scalars, computed once: 1/||w_j||, ||w_j||, stop flag
    double inv_sqrt_zeta;
    unsigned *cnt;     // [2] arrival tickets of the spmv / update launches
    long long *skSV;   // [G][s]
    long long *skSAV;  // [G][s]
    double *gram;      // [m][kMaxK]: <w_j, w_{j-d}>, d = 1..k-1 (reduced by the update kernel of step j-1)
    int *eys;          // [m] exponent of max|y~_j| (kNoExp if zero)
    int *ews;          // [m] exponent of max|w_j|
    double *epscol;    // [m] | ||S v_j||^2 - 1 |
    int *iscal;        // [0] stopped, [1] m_eff, [2] status, [3] step that stopped
    int64_t rows_per_cta;      // row partition of the update kernel (sized the sketch tables)
    int64_t spmv_rows;         // rows per CTA of the SpMV kernel (multiple of 32)
    int G_upd;                 // CTAs of the update kernel = number of sketch partials
    RowSplit rs;               // long rows of a skewed operator (row split)
    double *seg_part;          // [rs.nseg] partial sums of the long rows' segments
};

namespace {

// Finalise a sketch column from the integer partials, for this CTA's slice of
// the s rows: one warp per row of S.
__device__ __forceinline__ void finalize_sketch(const long long *part, int G, int s, int E, int frac, double scale,
                                                double *out_col) {
    const int per = (s + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per;
    const int i1 = min(s, i0 + per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = i0 + warp; i < i1; i += blockDim.x / 32) {
        double v = 0.0;
        if (E != kNoExp) v = scale_pow2(warp_sum_i64_exact(part + i, G, (size_t)s), E - frac) * scale;
        if (lane == 0) out_col[i] = v;
    }
}

__global__ void __launch_bounds__(kThreads) k_arnoldi_init(ArnCtx c, const double *__restrict__ b) {
    __shared__ double red[64];
    const int64_t r0 = (int64_t)blockIdx.x * c.rows_per_cta;
    const int64_t r1 = min(c.n, r0 + c.rows_per_cta);
    double nrm[1] = {0.0};
    double mx = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) {
        const double x = b[r];
        c.V[r] = x;
        nrm[0] = fma(x, x, nrm[0]);
        mx = fmax(mx, fabs(x));
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

// Row split: one warp per segment of a long row, lane-strided products over
// its CSR entries, then a butterfly whose lane-0 result (a fixed order) is the
// segment's partial sum of A w_j.
__global__ void __launch_bounds__(256) k_spmv_long(ArnCtx c, int j) {
    if (c.iscal[0] && c.iscal[3] < j) return;
    const double *x = c.V + vcol(c, j);
    const double *vals = (const double *)c.rs.values;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < c.rs.nseg; g += nwarps) {
        const int b = __ldg(c.rs.seg_beg + g), e = __ldg(c.rs.seg_end + g);
        double acc = 0.0;
        for (int p = b + lane; p < e; p += 32) acc = fma(__ldg(vals + p), x[__ldg(c.rs.colind + p)], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) c.seg_part[g] = acc;
    }
}

template <int KW, int WMAX>
__global__ void __launch_bounds__(kSpmvThreads, 1) k_arnoldi_spmv(ArnCtx c, int j) {
    __shared__ double red[BlockSumTraits<KW, kSpmvThreads>::kSmem];
    // a stop decided by an earlier launch; a stop decided in this launch is
    // recomputed identically by every CTA below
    if (c.iscal[0] && c.iscal[3] < j) return;
    const int G = gridDim.x;
    const int s = c.sp.s;

    // S v_{j-1} and S A v_{j-1} from the integer partials of the previous step
    if (j >= 1 && !c.identity && !c.direct) {
        const int frac = c.srht ? c.srht_frac : sketch_fraction_bits_from_limb(limb_bits(*c.binmax));
        const double sc = c.vscale[j - 1] * c.sk_scale;
        finalize_sketch(c.skSV, c.sk_parts, s, c.ews[j - 1], frac, sc, c.SV + (size_t)(j - 1) * s);
        finalize_sketch(c.skSAV, c.sk_parts, s, c.eys[j - 1], frac, sc, c.SAV + (size_t)(j - 1) * s);
    }

    // zero right-hand side (j = 0) or happy breakdown ||w_j|| <= 1e-12 ||A v_{j-1}||,
    // decided once by the previous launch
    const double *sc_j = c.stepsc + 4 * (size_t)j;
    if (j >= 1 && blockIdx.x == 0 && threadIdx.x == 0) c.H[j + (size_t)(j - 1) * (c.m + 1)] = sc_j[1];
    if (sc_j[2] != 0.0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c.iscal[0] = 1;
            c.iscal[1] = j;
            c.iscal[3] = j;
            if (j == 0) c.iscal[2] = SKF_ERR_ZERO_RHS;
        }
        return;
    }

    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;
    // acc[a] = <w_{i0+a}, y~>
    double acc[KW];
#pragma unroll
    for (int i = 0; i < KW; ++i) acc[i] = 0.0;
    double ymax = 0.0;
    const double *wj = c.V + vcol(c, j);
    const int64_t r0 = (int64_t)blockIdx.x * c.spmv_rows;
    const int64_t r1 = min(c.n, r0 + c.spmv_rows);
    unsigned long long ykey = 0;
    // rows_per_cta is a multiple of 32, so each warp works on whole slices;
    // the slice width and offset are loaded once per warp, and for slices up
    // to WMAX wide all value/column loads of a row are issued together
    const int lane = threadIdx.x & 31;
    for (int64_t rw = r0 + (threadIdx.x & ~31); rw < r1; rw += kSpmvThreads) {
        const int64_t t = rw >> 5;
        int wt = 0;
        long long so = 0;
        uint2 sl = make_uint2(0u, 0u);
        if (lane == 0) {
            wt = __ldg(c.sell_w + t);
            so = __ldg(c.sell_off + t);
            if (c.rs.sell_long) sl = __ldg(c.rs.sell_long + t);
        }
        wt = __shfl_sync(0xffffffffu, wt, 0);
        so = __shfl_sync(0xffffffffu, so, 0);
        sl.x = __shfl_sync(0xffffffffu, sl.x, 0);
        sl.y = __shfl_sync(0xffffffffu, sl.y, 0);
        const int64_t slot = rw + lane;
        if (slot >= r1) continue;
        const int64_t r = c.rs.perm ? (int64_t)__ldg(c.rs.perm + slot) : slot;   // the lane's row
        const int64_t base = so + lane;
        double y = 0.0;
        if (wt <= WMAX) {
            double av[WMAX], xv[WMAX];
#pragma unroll
            for (int p = 0; p < WMAX; ++p) {
                if (p < wt) {
                    const int64_t o = base + 32ll * p;
                    av[p] = __ldg(c.sell_val + o);
                    xv[p] = wj[__ldg(c.sell_col + o)];
                }
            }
#pragma unroll
            for (int p = 0; p < WMAX; ++p)
                if (p < wt) y = fma(av[p], xv[p], y);
        } else {
            for (int p = 0; p < wt; ++p) {
                const int64_t o = base + 32ll * p;
                y = fma(__ldg(c.sell_val + o), wj[__ldg(c.sell_col + o)], y);
            }
        }
        if (sl.x) y = add_long_row(c.rs, c.seg_part, sl, lane, y);
        c.Y[r] = y;
#pragma unroll
        for (int a = 0; a < KW; ++a)
            if (a < nw) acc[a] = fma(c.V[r + c.woff[a]], y, acc[a]);
        ykey = max(ykey, abs_key(y));
    }
    block_sum_auto<KW, kSpmvThreads>(acc, red);
    ymax = key_to_abs(block_max_key<kSpmvThreads>(ykey, (unsigned long long *)red));
    if (threadIdx.x == 0) {
        double *o = c.p1 + (size_t)blockIdx.x * kP1;
        for (int i = 0; i < KW; ++i) o[i] = acc[i];
        o[kP1 - 1] = ymax;
    }
    if (last_to_arrive(c.cnt)) {
        // reduce only the slots in use: d[0..nw-1], ymax
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int v = warp; v <= nw; v += kSpmvThreads / 32) {
            const int slot = (v < nw) ? v : kP1 - 1;
            const double r = warp_reduce_partials(c.p1 + slot, G, kP1, slot == kP1 - 1);
            if (lane == 0) c.fin_d[(size_t)j * kP1 + slot] = r;
        }
        if (threadIdx.x == 0) c.cnt[0] = 0u;
    }
}

// Pipelined variant of k_arnoldi_spmv for operators whose SELL slices are at
// most W <= 8 wide (W product slots per row, so that no predicated-off DFMA
// takes FP64 pipe time on narrow stencils).  Rows are dealt out in chunks of kPipeRows (one row per
// thread), chunk c to CTA c mod gridDim.x, so all CTAs sweep the rows
// together and the stencil gathers of neighbouring chunks meet in L2.  Within
// a CTA the loads are software-pipelined four deep: while the FP64 products
// of chunk i run, the values, gathers and window entries of chunk i + 1, the
// column indices of chunk i + 2 and the slice metadata of chunk i + 3 are in
// flight, so a chunk costs the longer of its arithmetic and one memory round
// trip rather than their sum.  Prologue and epilogue are those of
// k_arnoldi_spmv.
constexpr int kPipeRows = 512;

// CTAs of the pipelined SpMV: one per SM, at most one per chunk.
inline int pipe_ctas(int64_t n) {
    const int64_t chunks = (n + kPipeRows - 1) / kPipeRows;
    return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, num_sms()));
}

template <int KW, int W>
__global__ void __launch_bounds__(kPipeRows, 1) k_arnoldi_spmv_pipe(ArnCtx c, int j) {
    __shared__ double red[BlockSumTraits<KW, kPipeRows>::kSmem];
    // programmatic dependent of the previous launch: every CTA waits for it
    // before reading anything (and before any exit), then releases the next
    // launch so that its placement overlaps this one
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (c.iscal[0] && c.iscal[3] < j) return;
    const int G = gridDim.x;
    const int s = c.sp.s;
    if (j >= 1 && !c.identity && !c.direct) {
        const int frac = c.srht ? c.srht_frac : sketch_fraction_bits_from_limb(limb_bits(*c.binmax));
        const double sc = c.vscale[j - 1] * c.sk_scale;
        finalize_sketch(c.skSV, c.sk_parts, s, c.ews[j - 1], frac, sc, c.SV + (size_t)(j - 1) * s);
        finalize_sketch(c.skSAV, c.sk_parts, s, c.eys[j - 1], frac, sc, c.SAV + (size_t)(j - 1) * s);
    }
    const double *sc_j = c.stepsc + 4 * (size_t)j;
    if (j >= 1 && blockIdx.x == 0 && threadIdx.x == 0) c.H[j + (size_t)(j - 1) * (c.m + 1)] = sc_j[1];
    if (sc_j[2] != 0.0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c.iscal[0] = 1;
            c.iscal[1] = j;
            c.iscal[3] = j;
            if (j == 0) c.iscal[2] = SKF_ERR_ZERO_RHS;
        }
        return;
    }
    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;
    double acc[KW];
#pragma unroll
    for (int a = 0; a < KW; ++a) acc[a] = 0.0;
    unsigned long long ykey = 0;
    const double *wj = c.V + vcol(c, j);
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (c.n + kPipeRows - 1) / kPipeRows;
    const int64_t nc = nchunks > blockIdx.x ? (nchunks - 1 - blockIdx.x) / G + 1 : 0;
    const int64_t step = (int64_t)G * kPipeRows;
    const int64_t rw0 = (int64_t)blockIdx.x * kPipeRows + (threadIdx.x & ~31);   // warp's slice in chunk 0

    // Stage state at the top of iteration i: values, gathers and window of
    // chunk i (in flight since iteration i - 1), slice metadata and column
    // indices of chunk i + 1, lane 0's raw metadata of chunk i + 2.  Wide
    // windows (KW > 4) are loaded in their own iteration: two sets of them
    // would not fit in the registers.
    constexpr bool kWinAhead = KW <= 4;
    int wr0 = 0, wr1 = 0;
    long long or0 = 0, or1 = 0;
    if (lane == 0) {
        if (nc > 0 && rw0 < c.n) {
            wr0 = __ldg(c.sell_w + (rw0 >> 5));
            or0 = __ldg(c.sell_off + (rw0 >> 5));
        }
        if (nc > 1 && rw0 + step < c.n) {
            wr1 = __ldg(c.sell_w + ((rw0 + step) >> 5));
            or1 = __ldg(c.sell_off + ((rw0 + step) >> 5));
        }
    }
    int wt_c = __shfl_sync(0xffffffffu, wr0, 0);
    const long long so_c = __shfl_sync(0xffffffffu, or0, 0);
    int wt_n = __shfl_sync(0xffffffffu, wr1, 0);
    long long so_n = __shfl_sync(0xffffffffu, or1, 0);
    int cv[W], cvn[W];
#pragma unroll
    for (int p = 0; p < W; ++p) cv[p] = cvn[p] = 0;
    {
        const int32_t *pc = c.sell_col + so_c + lane;
        const int32_t *pn = c.sell_col + so_n + lane;
#pragma unroll
        for (int p = 0; p < W; ++p) {
            if (p < wt_c) cv[p] = __ldcs(pc + 32 * p);
            if (p < wt_n) cvn[p] = __ldcs(pn + 32 * p);
        }
    }
    int mw_raw = 0;
    long long mo_raw = 0;
    if (lane == 0 && nc > 2 && rw0 + 2 * step < c.n) {
        mw_raw = __ldg(c.sell_w + ((rw0 + 2 * step) >> 5));
        mo_raw = __ldg(c.sell_off + ((rw0 + 2 * step) >> 5));
    }
    double av[W], xv[W], wv[KW];
    {
        const double *pv = c.sell_val + so_c + lane;
        const bool ok = nc > 0 && rw0 < c.n && rw0 + lane < c.n;
#pragma unroll
        for (int p = 0; p < W; ++p) {
            av[p] = 0.0;
            xv[p] = 0.0;
            if (p < wt_c) {
                av[p] = __ldcs(pv + 32 * p);
                xv[p] = wj[cv[p]];
            }
        }
#pragma unroll
        for (int a = 0; a < KW; ++a) wv[a] = (kWinAhead && ok && a < nw) ? c.V[rw0 + lane + c.woff[a]] : 0.0;
    }
    for (int64_t i = 0; i < nc; ++i) {
        const int64_t rw = rw0 + i * step;
        const int64_t r = rw + lane;
        const bool ok = rw < c.n && r < c.n;   // padded rows of the last slice do no work
        // (1) values, gathers and window of chunk i + 1 (wt_n = 0 past the end)
        double avn[W], xvn[W], wvn[KW];
        {
            const double *pv = c.sell_val + so_n + lane;
            const int64_t rn = r + step;
            const bool okn = i + 1 < nc && rw + step < c.n && rn < c.n;
#pragma unroll
            for (int p = 0; p < W; ++p) {
                avn[p] = 0.0;
                xvn[p] = 0.0;
                if (p < wt_n) {
                    avn[p] = __ldcs(pv + 32 * p);
                    xvn[p] = wj[cvn[p]];
                }
            }
#pragma unroll
            for (int a = 0; a < KW; ++a) wvn[a] = (kWinAhead && okn && a < nw) ? c.V[rn + c.woff[a]] : 0.0;
        }
        if constexpr (!kWinAhead) {
#pragma unroll
            for (int a = 0; a < KW; ++a) wv[a] = (ok && a < nw) ? c.V[r + c.woff[a]] : 0.0;
        }
        // (2) metadata of chunk i + 2 (loaded one iteration ago) and its column indices
        const int wt_nn = __shfl_sync(0xffffffffu, mw_raw, 0);
        const long long so_nn = __shfl_sync(0xffffffffu, mo_raw, 0);
        int cvnn[W];
        {
            const int32_t *pc = c.sell_col + so_nn + lane;
#pragma unroll
            for (int p = 0; p < W; ++p) {
                cvnn[p] = 0;
                if (p < wt_nn) cvnn[p] = __ldcs(pc + 32 * p);
            }
        }
        // (3) metadata of chunk i + 3
        mw_raw = 0;
        mo_raw = 0;
        if (lane == 0 && i + 3 < nc && rw + 3 * step < c.n) {
            mw_raw = __ldg(c.sell_w + ((rw + 3 * step) >> 5));
            mo_raw = __ldg(c.sell_off + ((rw + 3 * step) >> 5));
        }
        // (4) y~ of chunk i, from the loads issued one iteration ago
        if (ok) {
            double y = 0.0;
#pragma unroll
            for (int p = 0; p < W; ++p)
                if (p < wt_c) y = fma(av[p], xv[p], y);
            c.Y[r] = y;
#pragma unroll
            for (int a = 0; a < KW; ++a)
                if (a < nw) acc[a] = fma(wv[a], y, acc[a]);
            ykey = max(ykey, abs_key(y));
        }
        wt_c = wt_n;
        wt_n = wt_nn;
        so_n = so_nn;
#pragma unroll
        for (int p = 0; p < W; ++p) {
            av[p] = avn[p];
            xv[p] = xvn[p];
            cvn[p] = cvnn[p];
        }
#pragma unroll
        for (int a = 0; a < KW; ++a) wv[a] = wvn[a];
    }
    block_sum_auto<KW, kPipeRows>(acc, red);
    const double ymax = key_to_abs(block_max_key<kPipeRows>(ykey, (unsigned long long *)red));
    if (threadIdx.x == 0) {
        double *o = c.p1 + (size_t)blockIdx.x * kP1;
        for (int i = 0; i < KW; ++i) o[i] = acc[i];
        o[kP1 - 1] = ymax;
    }
    if (last_to_arrive(c.cnt)) {
        const int warp = threadIdx.x >> 5;
        for (int v = warp; v <= nw; v += kPipeRows / 32) {
            const int slot = (v < nw) ? v : kP1 - 1;
            const double r = warp_reduce_partials(c.p1 + slot, G, kP1, slot == kP1 - 1);
            if (lane == 0) c.fin_d[(size_t)j * kP1 + slot] = r;
        }
        if (threadIdx.x == 0) c.cnt[0] = 0u;
    }
}

template <int KW, int ZCAP>
__global__ void __launch_bounds__(kUpdThreads, KW <= 2 ? 2 : 1) k_arnoldi_update(ArnCtx c, int j) {
    extern __shared__ int bins[];
    __shared__ double red[BlockSumTraits<KW, kUpdThreads>::kSmem];
    __shared__ double sh[kMaxK];     // MGS coefficients h_ij
    __shared__ double scoef[kMaxK];  // h_ij * sigma_i, newest window vector first: scoef[b] for w_{j-b}
    // programmatic dependent of the SpMV launch (see k_arnoldi_spmv_pipe)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (c.iscal[0] && c.iscal[3] <= j) return;   // stopped at this step (set by its spmv launch) or earlier
    const int G = gridDim.x;
    const double *fd = c.fin_d + (size_t)j * kP1;
    const double sigma = c.stepsc[4 * (size_t)j];
    const double wmax = c.fin_w[2 * j + 1];
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
            scoef[nw - 1 - a] = h * sa;
        }
    }
    __syncthreads();
    const int ey = positive_finite(ymax) ? bound_exponent(ymax) : kNoExp;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c.vscale[j] = sigma;
        c.eys[j] = ey;
        if (j < c.m - 1)
            for (int a = 0; a < nw; ++a) c.H[(i0 + a) + (size_t)j * (c.m + 1)] = sh[a];
    }
    // fixed-point sketches of w_j (-> S v_j) and y~ (-> S A v_j), two limbs each
    int *aw0 = bins, *aw1 = bins + s, *ay0 = bins + 2 * s, *ay1 = bins + 3 * s;
    if (c.sparse)
        for (int i = threadIdx.x; i < 4 * s; i += kUpdThreads) bins[i] = 0;
    __syncthreads();
    const int L = c.sparse ? limb_bits(*c.binmax) : 0;
    const int frac = sketch_fraction_bits_from_limb(L);
    const long long lmask = (1ll << L) - 1;
    const int ew = positive_finite(wmax) ? bound_exponent(wmax) : kNoExp;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.ews[j] = ew;
    const int shift_w = frac - (ew == kNoExp ? 0 : ew);
    const int shift_y = frac - (ey == kNoExp ? 0 : ey);
    const bool do_update = j < c.m - 1;
    // part[0] = ||w_{j+1}||^2, part[d] = <w_{j+1}, w_{j+1-d}> for the Gram
    // distances d = 1 .. ng of the next window (ng <= KW - 1): only the live
    // products are issued (a predicated-off DFMA still takes FP64 pipe time)
    const int ng = min(j + 1, c.k - 1);
    double part[KW];
#pragma unroll
    for (int i = 0; i < KW; ++i) part[i] = 0.0;
    unsigned long long nkey = 0;
    const int64_t r0 = (int64_t)blockIdx.x * c.rows_per_cta;
    const int64_t r1 = min(c.n, r0 + c.rows_per_cta);
    double *wn = c.V + vcol(c, j + 1);
    // window offsets newest first: woffr[b] locates w_{j-b}
    int64_t woffr[KW];
#pragma unroll
    for (int b = 0; b < KW; ++b) woffr[b] = b < nw ? c.woff[nw - 1 - b] : 0;
    // four rows per thread per iteration, all loads (with the compact sketch
    // pattern, where there is one) issued before the arithmetic
    constexpr int U = 4;
    const bool p8 = ZCAP == 8 && c.sparse && c.pattern8 != nullptr;
    for (int64_t rb = r0 + threadIdx.x; rb < r1; rb += U * kUpdThreads) {
        double yv[U], wv[U][KW];   // wv[u][b] = w_{j-b}: newest first
        uint2 pvu[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = rb + (int64_t)u * kUpdThreads;
            const bool ok = r < r1;
            yv[u] = ok ? c.Y[r] : 0.0;
#pragma unroll
            for (int a = 0; a < KW; ++a)
                wv[u][a] = (ok && a < nw) ? c.V[r + woffr[a]] : 0.0;
            pvu[u] = (ok && p8) ? __ldg((const uint2 *)(c.pattern8 + r * 8)) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = rb + (int64_t)u * kUpdThreads;
            if (r < r1) {
                const double y = yv[u];
                const double wjr = wv[u][0];
                if (do_update) {
                    double w = sigma * y;
#pragma unroll
                    for (int a = 0; a < KW; ++a)
                        if (KW - 1 - a < nw) w = fma(-scoef[KW - 1 - a], wv[u][KW - 1 - a], w);   // oldest first
                    wn[r] = w;
                    part[0] = fma(w, w, part[0]);
                    nkey = max(nkey, abs_key(w));
#pragma unroll
                    for (int d = 1; d < KW; ++d) {
                        if (d <= ng) part[d] = fma(w, wv[u][d - 1], part[d]);   // w_{j+1-d}
                    }
                }
                if (c.identity) {
                    c.SV[r + (size_t)j * s] = sigma * wjr;
                    c.SAV[r + (size_t)j * s] = sigma * y;
                } else if (c.sparse) {
                    const long long vw = fixed_point(wjr, shift_w);
                    const long long vy = ey == kNoExp ? 0 : fixed_point(y, shift_y);
                    const int w0 = (int)(vw & lmask), w1 = (int)(vw >> L);
                    const int y0 = (int)(vy & lmask), y1 = (int)(vy >> L);
                    if (p8) {
                        const uint2 pv = pvu[u];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int e = (int)__byte_perm(q < 4 ? pv.x : pv.y, 0u, 0x4440u + (q & 3));
                            const bool neg = e >= c.p8_block;
                            const int row = c.sp.start[q] + (neg ? e - c.p8_block : e);
                            red_limbs(aw0, aw1, row, w0, w1, neg);
                            red_limbs(ay0, ay1, row, y0, y1, neg);
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
                                red_limbs(aw0, aw1, row, w0, w1, neg);
                                red_limbs(ay0, ay1, row, y0, y1, neg);
                            }
                        }
                    }
                }
            }
        }
    }
    block_sum_auto<KW, kUpdThreads>(part, red);
    const double nmax = key_to_abs(block_max_key<kUpdThreads>(nkey, (unsigned long long *)red));
    if (threadIdx.x == 0) {
        // partial layout: slot 2 + a holds the Gram entry at distance d = nw - a
        double *o = c.p2 + (size_t)blockIdx.x * kP2;
        o[0] = part[0];
        o[1] = nmax;
#pragma unroll
        for (int d = 1; d < KW; ++d)
            if (d <= ng) o[2 + nw - d] = part[d];
    }
    if (c.sparse) {
        __syncthreads();
        long long *ow = c.skSV + (size_t)blockIdx.x * s, *oy = c.skSAV + (size_t)blockIdx.x * s;
        for (int i = threadIdx.x; i < s; i += kUpdThreads) {
            ow[i] = combine_limbs(aw0[i], aw1[i], L);
            oy[i] = combine_limbs(ay0[i], ay1[i], L);
        }
    }
    if (last_to_arrive(c.cnt + 1)) {
        const int warp = threadIdx.x >> 5;
        if (do_update)
            for (int v = warp; v < 2 + nw; v += kUpdThreads / 32) {
                const int d = nw - (v - 2);   // Gram distance of slot v - 2
                if (v >= 2 && (d < 1 || d > ng)) continue;
                const double r = warp_reduce_partials(c.p2 + v, G, kP2, v == 1);
                if ((threadIdx.x & 31) == 0) {
                    if (v < 2) c.fin_w[2 * (j + 1) + v] = r;
                    else c.gram[(size_t)(j + 1) * kMaxK + d] = r;
                }
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (do_update) {
                // ||A v_j||^2 = sum_i h_ij^2 + ||w_{j+1}||^2 for the orthonormal window
                const double n2 = c.fin_w[2 * (j + 1)];
                double hs = 0.0;
                for (int a = 0; a < nw; ++a) hs += sh[a] * sh[a];
                const double hn = sqrt(n2);
                double *o = c.stepsc + 4 * (size_t)(j + 1);
                o[0] = hn > 0.0 ? 1.0 / hn : 0.0;
                o[1] = hn;
                o[2] = (hn > 1e-12 * sqrt(hs + n2)) ? 0.0 : 1.0;
            }
            c.cnt[1] = 0u;
        }
    }
}

// After the loop: S v_{m-1} and S A v_{m-1}.
__global__ void __launch_bounds__(kThreads) k_arnoldi_finish(ArnCtx c) {
    if (c.iscal[0] == 0 && !c.identity && !c.direct) {
        const int frac = c.srht ? c.srht_frac : sketch_fraction_bits_from_limb(limb_bits(*c.binmax));
        const double sc = c.vscale[c.m - 1] * c.sk_scale;
        finalize_sketch(c.skSV, c.sk_parts, c.sp.s, c.ews[c.m - 1], frac, sc, c.SV + (size_t)(c.m - 1) * c.sp.s);
        finalize_sketch(c.skSAV, c.sk_parts, c.sp.s, c.eys[c.m - 1], frac, sc, c.SAV + (size_t)(c.m - 1) * c.sp.s);
    }
}

// | ||S v_j||^2 - 1 | per column (the embedding-quality estimate of Sec. 4.3),
// one warp per column.
__global__ void __launch_bounds__(kThreads) k_arnoldi_eps(ArnCtx c) {
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

__global__ void __launch_bounds__(kThreads) k_arnoldi_info(ArnCtx c, skf_info *info) {
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

template <int KW, int ZCAP>
void launch_steps(const ArnCtx &c, int G, int Gs, size_t smem, const SrhtDev *sd, const SrdctDev *dd,
                  cudaStream_t st, const StepHook *hook) {
    // slices up to 8 wide take the pipelined SpMV; wider ones the generic
    // kernel (16 unrolled product slots, an entry loop past 16)
    auto spmv = k_arnoldi_spmv<KW, 16>;
    // a row split or a sorted slice layout takes the generic SpMV
    const bool pipe = c.max_width <= 8 && c.rs.sell_long == nullptr && c.rs.perm == nullptr;
    // product slots of the pipelined SpMV: the widest slice rounded up to 5, 7
    // or 8 (a slot past a slice's width is a predicated-off FP64 instruction)
    auto spmv_pipe = c.max_width <= 5 ? k_arnoldi_spmv_pipe<KW, 5>
                   : c.max_width <= 7 ? k_arnoldi_spmv_pipe<KW, 7> : k_arnoldi_spmv_pipe<KW, 8>;
    const int Gp = pipe_ctas(c.n);
    auto update = k_arnoldi_update<KW, ZCAP>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // the pipelined SpMV and the update are launched as programmatic
    // dependents of the launch before them (each waits for it in full)
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg_s = {}, cfg_u = {};
    cfg_s.gridDim = dim3((unsigned)Gp);
    cfg_s.blockDim = dim3(kPipeRows);
    cfg_s.stream = st;
    cfg_s.attrs = pdl;
    cfg_s.numAttrs = 1;
    cfg_u.gridDim = dim3((unsigned)G);
    cfg_u.blockDim = dim3(kUpdThreads);
    cfg_u.dynamicSmemBytes = smem;
    cfg_u.stream = st;
    cfg_u.attrs = pdl;
    cfg_u.numAttrs = 1;
    for (int j = 0; j < c.m; ++j) {
        ArnCtx cj = c;
        window_offsets(cj, j);
        if (c.rs.sell_long) k_spmv_long<<<long_ctas(c.rs.nseg, num_sms()), 256, 0, st>>>(cj, j);
        if (pipe) cudaLaunchKernelEx(&cfg_s, spmv_pipe, cj, j);
        else spmv<<<Gs, kSpmvThreads, 0, st>>>(cj, j);
        call_hook(hook, j, st);   // S v_i, S A v_i final for i < j
        cudaLaunchKernelEx(&cfg_u, update, cj, j);
        if (j + 1 < c.m) call_col_hook(hook, j + 1, st);
        if (dd) {   // SV[:, j] = sigma_j S w_j, SAV[:, j] = sigma_j S y_j
            SrdctCols cols{};
            cols.ncols = 2;
            cols.x[0] = c.V + (size_t)(c.vring ? j % c.vring : j) * c.ldv;
            cols.x[1] = c.Y;
            cols.out[0] = c.SV + (size_t)j * c.sp.s;
            cols.out[1] = c.SAV + (size_t)j * c.sp.s;
            cols.colscale = c.stepsc + 4 * (size_t)j;
            cols.iscal = c.iscal;
            cols.step = j;
            srdct_launch(*dd, cols, st);
        }
        if (sd) {   // S w_j and S y_j (exponents written by the update kernel)
            SrhtCols cols{};
            cols.ncols = 2;
            cols.x[0] = c.V + (size_t)(c.vring ? j % c.vring : j) * c.ldv;
            cols.e[0] = c.ews + j;
            cols.part[0] = c.skSV;
            cols.x[1] = c.Y;
            cols.e[1] = c.eys + j;
            cols.part[1] = c.skSAV;
            cols.iscal = c.iscal;
            cols.step = j;
            srht_launch(*sd, cols, st);
        }
    }
}

template <int ZCAP>
void launch_steps_k(const ArnCtx &c, int G, int Gs, size_t smem, const SrhtDev *sd, const SrdctDev *dd,
                    cudaStream_t st, const StepHook *hook) {
    if (c.k <= 2) launch_steps<2, ZCAP>(c, G, Gs, smem, sd, dd, st, hook);
    else if (c.k <= 4) launch_steps<4, ZCAP>(c, G, Gs, smem, sd, dd, st, hook);
    else if (c.k <= 8) launch_steps<8, ZCAP>(c, G, Gs, smem, sd, dd, st, hook);
    else launch_steps<16, ZCAP>(c, G, Gs, smem, sd, dd, st, hook);
}

}  // namespace

// Host driver: launches init, m x (spmv, update), finish on `st`.
skf_status arnoldi_run(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, double *V, int64_t ldv,
                       double *vscale, double *SV, double *SAV, double *H, int *iscal, skf_info *info,
                       cudaStream_t st, const StepHook *hook, int vring) {
    // the persistent single-launch form where it applies (no per-step host
    // hooks, one-pass storage, sparse-sign S, k <= 4, rows fit in shared memory)
    if (step_mode() != 1 && hook == nullptr && vring == 0) {
        const skf_status ps = arnoldi_run_persistent(A, S, b, m, k, V, ldv, vscale, SV, SAV, H, iscal, info, st);
        if (ps != SKF_ERR_NOT_SUPPORTED) return ps;
        if (step_mode() == 2) return fail(SKF_ERR_NOT_SUPPORTED, "persistent Arnoldi form does not apply here");
    }
    ArnCtx c{};
    c.n = A->n;
    c.sell_off = A->sell_off;
    c.sell_w = A->sell_w;
    c.sell_val = (const double *)A->sell_val;
    c.sell_col = A->sell_col;
    c.max_width = A->max_width;
    c.identity = S->kind == SKF_SKETCH_IDENTITY;
    c.sparse = S->kind == SKF_SKETCH_SPARSE_SIGN;
    c.srht = S->kind == SKF_SKETCH_SRHT;
    c.direct = S->kind == SKF_SKETCH_SRDCT;
    SrhtDev sd{};
    SrdctDev dd{};
    if (c.direct) dd = make_srdct(S);
    if (c.sparse) {
        c.sp = make_sparse_sign(S);
        c.pattern = S->pattern;
        c.binmax = S->binmax;
        if (S->zeta == 8 && S->pattern8 != nullptr) {
            c.pattern8 = S->pattern8;
            c.p8_block = S->p8_block;
        }
    }
    if (c.srht) {
        sd = make_srht(S);
        c.srht_frac = sd.frac;
    }
    c.sp.s = S->s;
    c.sp.zeta = c.sparse ? S->zeta : 1;
    c.inv_sqrt_zeta = 1.0 / sqrt((double)c.sp.zeta);
    c.sk_scale = c.srht ? 1.0 / sqrt((double)S->s) : c.inv_sqrt_zeta;
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
    int G;
    row_partition(A->n, &G, &c.rows_per_cta);   // the partition the sketch tables were sized for
    int Gs = num_sms();
    if ((A->n + 1023) / 1024 < Gs) Gs = (int)((A->n + 1023) / 1024);
    if (Gs < 1) Gs = 1;
    c.spmv_rows = ((A->n + Gs - 1) / Gs + 31) / 32 * 32;
    c.G_upd = G;
    c.sk_parts = c.srht ? sd.nblk : G;

    char *ws = nullptr;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t szY = sizeof(double) * A->n;
    const size_t szP1 = sizeof(double) * (size_t)std::max(std::max(G, Gs), pipe_ctas(A->n)) * kP1;
    const size_t szP2 = sizeof(double) * (size_t)G * kP2;
    const size_t szFd = sizeof(double) * (size_t)m * kP1;
    const size_t szFw = sizeof(double) * (size_t)(m + 1) * 2;
    const size_t szSc = sizeof(double) * (size_t)(m + 1) * 4;
    const size_t szCnt = sizeof(unsigned) * 4;
    const size_t szSk = c.identity ? 0 : sizeof(long long) * (size_t)c.sk_parts * S->s;
    const size_t szGram = sizeof(double) * (size_t)m * kMaxK;
    const size_t szE = sizeof(int) * (size_t)m;
    const size_t szEps = sizeof(double) * (size_t)m;
    c.rs = row_split_of(A);
    const size_t szSeg = sizeof(double) * (size_t)std::max<int64_t>(c.rs.nseg, 1);
    const size_t szDct = c.direct ? srdct_work_bytes(S) : 0;   // FFT form of the SRDCT: its complex buffers
    const size_t total = al(szY) + al(szP1) + al(szP2) + al(szFd) + al(szFw) + al(szSc) + al(szCnt) + 2 * al(szSk) +
                         al(szGram) + 2 * al(szE) + al(szEps) + al(szSeg) + al(szDct);
    skf_status stt = dalloc((void **)&ws, total, st);
    if (stt != SKF_OK) return stt;
    size_t off = 0;
    auto take = [&](size_t sz) {
        char *p = ws + off;
        off += al(sz);
        return p;
    };
    c.Y = (double *)take(szY);
    c.p1 = (double *)take(szP1);
    c.p2 = (double *)take(szP2);
    c.fin_d = (double *)take(szFd);
    c.fin_w = (double *)take(szFw);
    c.stepsc = (double *)take(szSc);
    c.cnt = (unsigned *)take(szCnt);
    c.skSV = (long long *)take(szSk);
    c.skSAV = (long long *)take(szSk);
    c.gram = (double *)take(szGram);
    c.eys = (int *)take(szE);
    c.ews = (int *)take(szE);
    c.epscol = (double *)take(szEps);
    c.seg_part = (double *)take(szSeg);
    if (szDct) dd.work = (double2 *)take(szDct);
    cudaMemsetAsync(c.cnt, 0, szCnt, st);

    const size_t smem = c.sparse ? sizeof(int) * 4 * S->s : 0;   // two limbs for each of S v_j, S A v_j
    k_arnoldi_init<<<G, kThreads, 0, st>>>(c, b);
    call_col_hook(hook, 0, st);
    const SrhtDev *sdp = c.srht ? &sd : nullptr;
    const SrdctDev *ddp = c.direct ? &dd : nullptr;
    if (c.sp.zeta <= 8) launch_steps_k<8>(c, G, Gs, smem, sdp, ddp, st, hook);
    else launch_steps_k<16>(c, G, Gs, smem, sdp, ddp, st, hook);
    k_arnoldi_finish<<<G, kThreads, 0, st>>>(c);
    call_hook(hook, m, st);
    k_arnoldi_eps<<<(m + (kThreads / 32) - 1) / (kThreads / 32), kThreads, 0, st>>>(c);
    k_arnoldi_info<<<1, kThreads, 0, st>>>(c, info);
    count_launches(4 + (c.rs.sell_long ? 3ll : 2ll) * m);
    cudaError_t e = cudaGetLastError();
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "arnoldi kernels");
    return SKF_OK;
}

}  // namespace skf
