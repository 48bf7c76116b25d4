// k-truncated Arnoldi with on-the-fly sketching (Algorithm 2, Sec. 2.2).
//
// Storage: column j of V holds w_j, a positive multiple of the basis vector
// v_j = sigma_j w_j with sigma_j = 1/||w_j||.  Keeping w_j unnormalised lets
// one step run as two kernels (two grid-wide dependencies per step: the dot
// products before the update, and the new vector before the next SpMV):
//
//   spmv   (step j): y~ = A w_j on the CTA's rows -> Y; partial dots
//                    <w_i, y~> (i in the window), Gram <w_j, w_i>, max|y~|;
//                    fixed-point sketch of w_j (-> S v_j).
//   update (step j): every CTA reduces the partials in a fixed order, forms
//                    the MGS coefficients from the dots and the window Gram
//                    matrix (identical to MGS in exact arithmetic), writes
//                    w_{j+1} = sigma_j y~ - sum_i h_ij sigma_i w_i, partial
//                    ||w_{j+1}||^2 and max|w_{j+1}|; fixed-point sketch of y~
//                    (-> S A v_j).
//
// Cross-CTA reductions always run in CTA order, so the results do not depend
// on scheduling.  Sketch partial sums are integers (exact), see skf_internal.
#include <math.h>

#include "skf_internal.cuh"

namespace skf {

struct ArnCtx {
    int64_t n;
    const int32_t *rowptr;
    const int32_t *colind;
    const double *vals;
    SparseSign sp;
    int frac;          // fixed-point fraction bits
    int identity;      // S = I
    int m, k;
    double *V;
    int64_t ldv;
    double *vscale;    // [m]
    double *SV, *SAV;  // s x m
    double *H;         // (m+1) x m
    double *Y;         // [n]
    double *p1;        // [G][2*kMaxK]: d[0..k-1], g[0..k-2], ymax at slot 2*kMaxK-1
    double *p2;        // [2][G][2]: ||w||^2, max|w|
    long long *skSV;   // [G][s]
    long long *skSAV;  // [G][s]
    double *gram;      // [m][kMaxK]: <w_j, w_{j-d}>, d = 1..k-1
    int *eys;          // [m] exponent of max|y~_j| (INT_MIN if zero)
    int *iscal;        // [0] stopped, [1] m_eff, [2] status, [3] step that stopped
    int64_t rows_per_cta;
};

namespace {

constexpr int kP1 = 2 * kMaxK;
constexpr int kNoExp = -100000;

// Sums (or maxes) of G per-CTA partials, computed by one warp in a fixed order.
__device__ __forceinline__ double warp_reduce_partials(const double *p, int G, int stride, bool is_max) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int g = lane; g < G; g += 32) {
        const double v = p[(size_t)g * stride];
        acc = is_max ? fmax(acc, v) : acc + v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = is_max ? fmax(acc, t) : acc + t;
    }
    return acc;
}

__device__ __forceinline__ void sketch_scatter(const SparseSign &sp, uint32_t *lo, uint32_t *hi, int64_t r,
                                               long long v) {
    if (v == 0) return;
    uint64_t word = 0;
    for (int q = 0; q < sp.zeta; ++q) {
        if ((q & 3) == 0) word = splitmix_word(sp.seed, (uint64_t)r * sp.words + (q >> 2));
        int row;
        bool neg;
        sparse_sign_entry(sp, word, q, row, neg);
        atomic_add_i64_split(lo + row, hi + row, neg ? -v : v);
    }
}

// Finalise sketch column `col` from the integer partials for this CTA's
// slice of the s rows.
__device__ __forceinline__ void finalize_sketch(const long long *part, int G, int s, int E, int frac, double scale,
                                                double *out_col) {
    const int per = (s + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per;
    const int i1 = min(s, i0 + per);
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        if (E == kNoExp) {
            out_col[i] = 0.0;
        } else {
            const double tot = sum_i64_exact(part + i, G, (size_t)s);
            out_col[i] = ldexp(tot, E - frac) * scale;
        }
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
        nrm[0] += x * x;
        mx = fmax(mx, fabs(x));
    }
    block_sum<1>(nrm, red);
    mx = block_max(mx, red);
    if (threadIdx.x == 0) {
        c.p2[(size_t)blockIdx.x * 2 + 0] = nrm[0];
        c.p2[(size_t)blockIdx.x * 2 + 1] = mx;
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
}

template <int KW>
__global__ void __launch_bounds__(kThreads) k_arnoldi_spmv(ArnCtx c, int j) {
    extern __shared__ uint32_t bins[];
    __shared__ double red[32 * kP1];
    __shared__ double sv[4];
    // a stop decided by an earlier launch; a stop decided in this launch is
    // recomputed identically by every CTA below
    if (c.iscal[0] && c.iscal[3] < j) return;
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double *p2 = c.p2 + (size_t)(j & 1) * G * 2;
    if (warp < 2) {
        const double v = warp_reduce_partials(p2 + warp, G, 2, warp == 1);
        if (lane == 0) sv[warp] = v;
    }
    __syncthreads();
    const double wnorm2 = sv[0], wmax = sv[1];
    const int s = c.sp.s;

    // S A v_{j-1} from the integer partials the previous update kernel wrote
    if (j >= 1 && !c.identity)
        finalize_sketch(c.skSAV, G, s, c.eys[j - 1], c.frac, c.vscale[j - 1] / sqrt((double)c.sp.zeta),
                        c.SAV + (size_t)(j - 1) * s);

    // zero right-hand side / happy breakdown: ||w_j|| <= 1e-12 ||A v_{j-1}||
    if (j == 0) {
        if (!(wnorm2 > 0.0)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                c.iscal[0] = 1;
                c.iscal[1] = 0;
                c.iscal[2] = SKF_ERR_ZERO_RHS;
                c.iscal[3] = 0;
            }
            return;
        }
    } else {
        const int i0p = max(0, j - c.k);
        double hs = 0.0;
        for (int i = i0p; i <= j - 1; ++i) {
            const double h = c.H[i + (size_t)(j - 1) * (c.m + 1)];
            hs += h * h;
        }
        const double hn = sqrt(wnorm2);
        if (blockIdx.x == 0 && threadIdx.x == 0) c.H[j + (size_t)(j - 1) * (c.m + 1)] = hn;
        if (!(hn > 1e-12 * sqrt(hs + wnorm2))) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                c.iscal[0] = 1;
                c.iscal[1] = j;
                c.iscal[3] = j;
            }
            return;
        }
    }

    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;
    uint32_t *lo = bins, *hi = bins + s;
    if (!c.identity) {
        for (int i = threadIdx.x; i < 2 * s; i += kThreads) bins[i] = 0u;
    }
    __syncthreads();
    const int shift = c.frac - bound_exponent(wmax);

    // acc[0..KW-1]: <w_i, y~>; acc[KW..2KW-2]: <w_j, w_i>
    double acc[2 * KW];
#pragma unroll
    for (int i = 0; i < 2 * KW; ++i) acc[i] = 0.0;
    double ymax = 0.0;
    const double *wj = c.V + (size_t)j * c.ldv;
    const int64_t r0 = (int64_t)blockIdx.x * c.rows_per_cta;
    const int64_t r1 = min(c.n, r0 + c.rows_per_cta);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) {
        const int p0 = c.rowptr[r], pe = c.rowptr[r + 1];
        double y = 0.0;
        for (int p = p0; p < pe; ++p) y = fma(c.vals[p], wj[c.colind[p]], y);
        c.Y[r] = y;
        const double wjr = wj[r];
#pragma unroll
        for (int sl = 0; sl < KW; ++sl) {
            if (sl < nw) {
                const double wi = (sl == nw - 1) ? wjr : c.V[r + (size_t)(i0 + sl) * c.ldv];
                acc[sl] = fma(wi, y, acc[sl]);
                if (sl < nw - 1) acc[KW + sl] = fma(wjr, wi, acc[KW + sl]);
            }
        }
        ymax = fmax(ymax, fabs(y));
        if (!c.identity) sketch_scatter(c.sp, lo, hi, r, fixed_point(wjr, shift));
    }
    block_sum<2 * KW>(acc, red);
    ymax = block_max(ymax, red);
    if (threadIdx.x == 0) {
        double *o = c.p1 + (size_t)blockIdx.x * kP1;
        for (int i = 0; i < kP1 - 1; ++i) o[i] = 0.0;
        for (int i = 0; i < KW; ++i) o[i] = acc[i];
        for (int i = 0; i < KW - 1; ++i) o[kMaxK + i] = acc[KW + i];
        o[kP1 - 1] = ymax;
    }
    if (!c.identity) {
        long long *o = c.skSV + (size_t)blockIdx.x * s;
        for (int i = threadIdx.x; i < s; i += kThreads)
            o[i] = (long long)(((unsigned long long)hi[i] << 32) | lo[i]);
    }
}

template <int KW>
__global__ void __launch_bounds__(kThreads) k_arnoldi_update(ArnCtx c, int j) {
    extern __shared__ uint32_t bins[];
    __shared__ double red[64];
    __shared__ double sd[kP1 + 2];
    __shared__ double sh[kMaxK];     // MGS coefficients h_ij
    __shared__ double scoef[kMaxK];  // h_ij * sigma_i
    if (c.iscal[0]) return;          // set at the latest by the spmv launch of this step
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double *p2 = c.p2 + (size_t)(j & 1) * G * 2;
    for (int v = warp; v < kP1 + 2; v += kThreads / 32) {
        double r;
        if (v < kP1) r = warp_reduce_partials(c.p1 + v, G, kP1, v == kP1 - 1);
        else r = warp_reduce_partials(p2 + (v - kP1), G, 2, v == kP1 + 1);
        if (lane == 0) sd[v] = r;
    }
    __syncthreads();
    const double sigma = 1.0 / sqrt(sd[kP1]);
    const double wmax = sd[kP1 + 1];
    const double ymax = sd[kP1 - 1];
    const int s = c.sp.s;
    const int i0 = max(0, j - c.k + 1);
    const int nw = j - i0 + 1;

    if (threadIdx.x == 0) {
        // MGS in the window, ascending, from the dots and the Gram matrix:
        // h_i = <v_i, y> - sum_{i' < i} h_i' <v_i, v_i'>.
        for (int a = 0; a < nw; ++a) {
            const int ia = i0 + a;
            const double sa = (ia == j) ? sigma : c.vscale[ia];
            double h = sa * sigma * sd[a];
            for (int b2 = 0; b2 < a; ++b2) {
                const int ib = i0 + b2;
                const double sb = c.vscale[ib];
                const double gab = (ia == j) ? sd[kMaxK + b2] : c.gram[(size_t)ia * kMaxK + (ia - ib)];
                h -= sh[b2] * sa * sb * gab;
            }
            sh[a] = h;
            scoef[a] = h * sa;
        }
    }
    __syncthreads();
    const int ey = ymax > 0.0 ? bound_exponent(ymax) : kNoExp;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c.vscale[j] = sigma;
        c.eys[j] = ey;
        if (j < c.m - 1)
            for (int a = 0; a < nw; ++a) c.H[(i0 + a) + (size_t)j * (c.m + 1)] = sh[a];
        for (int d = 1; d < nw; ++d) c.gram[(size_t)j * kMaxK + d] = sd[kMaxK + (nw - 1 - d)];
    }
    // S v_j from the integer partials of the spmv kernel
    if (!c.identity)
        finalize_sketch(c.skSV, G, s, wmax > 0.0 ? bound_exponent(wmax) : kNoExp, c.frac,
                        sigma / sqrt((double)c.sp.zeta), c.SV + (size_t)j * s);

    uint32_t *lo = bins, *hi = bins + s;
    if (!c.identity)
        for (int i = threadIdx.x; i < 2 * s; i += kThreads) bins[i] = 0u;
    __syncthreads();
    const int shift = c.frac - (ey == kNoExp ? 0 : ey);
    const bool do_update = j < c.m - 1;
    double nrm[1] = {0.0};
    double nmax = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * c.rows_per_cta;
    const int64_t r1 = min(c.n, r0 + c.rows_per_cta);
    double *wn = c.V + (size_t)(j + 1) * c.ldv;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) {
        const double y = c.Y[r];
        if (do_update) {
            double w = sigma * y;
#pragma unroll
            for (int a = 0; a < KW; ++a)
                if (a < nw) w = fma(-scoef[a], c.V[r + (size_t)(i0 + a) * c.ldv], w);
            wn[r] = w;
            nrm[0] = fma(w, w, nrm[0]);
            nmax = fmax(nmax, fabs(w));
        }
        if (c.identity) {
            c.SV[r + (size_t)j * s] = sigma * c.V[r + (size_t)j * c.ldv];
            c.SAV[r + (size_t)j * s] = sigma * y;
        } else if (ey != kNoExp) {
            sketch_scatter(c.sp, lo, hi, r, fixed_point(y, shift));
        }
    }
    block_sum<1>(nrm, red);
    nmax = block_max(nmax, red);
    if (do_update && threadIdx.x == 0) {
        double *o = c.p2 + (size_t)((j + 1) & 1) * G * 2 + (size_t)blockIdx.x * 2;
        o[0] = nrm[0];
        o[1] = nmax;
    }
    if (!c.identity) {
        long long *o = c.skSAV + (size_t)blockIdx.x * s;
        for (int i = threadIdx.x; i < s; i += kThreads)
            o[i] = (long long)(((unsigned long long)hi[i] << 32) | lo[i]);
    }
}

// After the loop: S A v_{m-1}, and the embedding-quality estimate of Sec. 4.3.
__global__ void __launch_bounds__(kThreads) k_arnoldi_finish(ArnCtx c, skf_info *info) {
    __shared__ double red[64];
    const int G = gridDim.x;
    const int s = c.sp.s;
    const bool stopped = c.iscal[0] != 0;
    if (!stopped && !c.identity)
        finalize_sketch(c.skSAV, G, s, c.eys[c.m - 1], c.frac, c.vscale[c.m - 1] / sqrt((double)c.sp.zeta),
                        c.SAV + (size_t)(c.m - 1) * s);
    if (blockIdx.x != 0 || info == nullptr) return;
    // block 0 finishes after its own slice; other slices are complete only
    // after this kernel, so eps_est is computed by k_arnoldi_info below.
}

__global__ void __launch_bounds__(kThreads) k_arnoldi_info(ArnCtx c, skf_info *info) {
    __shared__ double red[64];
    const int me = c.iscal[1];
    const int s = c.sp.s;
    double eps = 0.0;
    for (int j = 0; j < me; ++j) {
        double acc[1] = {0.0};
        for (int i = threadIdx.x; i < s; i += kThreads) acc[0] = fma(c.SV[i + (size_t)j * s], c.SV[i + (size_t)j * s], acc[0]);
        block_sum<1>(acc, red);
        eps = fmax(eps, fabs(acc[0] - 1.0));
    }
    if (threadIdx.x == 0 && info != nullptr) {
        info->status = c.iscal[2];
        info->m_eff = me;
        info->breakdown = (c.iscal[0] != 0 && me > 0) ? 1 : 0;
        info->beta = me > 0 ? 1.0 / c.vscale[0] : 0.0;
        info->eps_est = eps;
    }
}

}  // namespace

// Host driver: launches init, m x (spmv, update), finish on `st`.
skf_status arnoldi_run(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, double *V, int64_t ldv,
                       double *vscale, double *SV, double *SAV, double *H, int *iscal, skf_info *info,
                       cudaStream_t st) {
    ArnCtx c{};
    c.n = A->n;
    c.rowptr = A->rowptr;
    c.colind = A->colind;
    c.vals = (const double *)A->values;
    c.identity = S->kind == SKF_SKETCH_IDENTITY;
    if (!c.identity) c.sp = make_sparse_sign(S);
    c.sp.s = S->s;
    c.sp.zeta = c.identity ? 1 : S->zeta;
    c.m = m;
    c.k = k;
    c.V = V;
    c.ldv = ldv;
    c.vscale = vscale;
    c.SV = SV;
    c.SAV = SAV;
    c.H = H;
    c.iscal = iscal;
    int G = 2 * num_sms();
    const int64_t min_rows = 512;
    if ((A->n + min_rows - 1) / min_rows < G) G = (int)((A->n + min_rows - 1) / min_rows);
    if (G < 1) G = 1;
    c.rows_per_cta = (A->n + G - 1) / G;
    c.frac = sketch_fraction_bits(c.rows_per_cta);

    char *ws = nullptr;
    const size_t szY = sizeof(double) * A->n;
    const size_t szP1 = sizeof(double) * (size_t)G * kP1;
    const size_t szP2 = sizeof(double) * 2 * (size_t)G * 2;
    const size_t szSk = c.identity ? 0 : sizeof(long long) * (size_t)G * S->s;
    const size_t szGram = sizeof(double) * (size_t)m * kMaxK;
    const size_t szE = sizeof(int) * (size_t)m;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t total = al(szY) + al(szP1) + al(szP2) + 2 * al(szSk) + al(szGram) + al(szE);
    skf_status stt = dalloc((void **)&ws, total, st);
    if (stt != SKF_OK) return stt;
    size_t off = 0;
    c.Y = (double *)(ws + off); off += al(szY);
    c.p1 = (double *)(ws + off); off += al(szP1);
    c.p2 = (double *)(ws + off); off += al(szP2);
    c.skSV = (long long *)(ws + off); off += al(szSk);
    c.skSAV = (long long *)(ws + off); off += al(szSk);
    c.gram = (double *)(ws + off); off += al(szGram);
    c.eys = (int *)(ws + off); off += al(szE);

    const size_t smem = c.identity ? 0 : sizeof(uint32_t) * 2 * S->s;
    k_arnoldi_init<<<G, kThreads, 0, st>>>(c, b);
    auto loop = [&](auto spmv, auto update) {
        if (smem > 48 * 1024) {
            cudaFuncSetAttribute(spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        }
        for (int j = 0; j < m; ++j) {
            spmv<<<G, kThreads, smem, st>>>(c, j);
            update<<<G, kThreads, smem, st>>>(c, j);
        }
    };
    if (k <= 2) loop(k_arnoldi_spmv<2>, k_arnoldi_update<2>);
    else if (k <= 4) loop(k_arnoldi_spmv<4>, k_arnoldi_update<4>);
    else if (k <= 8) loop(k_arnoldi_spmv<8>, k_arnoldi_update<8>);
    else loop(k_arnoldi_spmv<16>, k_arnoldi_update<16>);
    k_arnoldi_finish<<<G, kThreads, 0, st>>>(c, info);
    k_arnoldi_info<<<1, kThreads, 0, st>>>(c, info);
    cudaError_t e = cudaGetLastError();
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "arnoldi kernels");
    return SKF_OK;
}

}  // namespace skf
