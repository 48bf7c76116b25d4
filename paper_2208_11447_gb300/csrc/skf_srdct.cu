// Subsampled randomized discrete cosine transform (the sketch of the paper's
// experiments, Sec. 5.1: S = P F E with F a DCT):
//   (S x)_i = sqrt(N/s) (F E x)_{P_i},  F the orthonormal DCT-II,
//   (F y)_k = a_k sum_n y_n cos(pi k (2n + 1) / (2N)),  a_0 = 1/sqrt(N), a_k = sqrt(2/N),
// E the signs of the SRHT definition and P the first s entries of its partial
// Fisher-Yates shuffle, of [0, N).
//
// Fast form (N with no prime factor above 7).  Makhoul's reordering (IEEE
// Trans. ASSP 28, 1980) turns the DCT-II into one DFT of length N: with
// v_n = y_{2n} for n < ceil(N/2) and v_{N-1-n} = y_{2n+1} for n < N/2,
// V = DFT_N(v) and (F y)_k = a_k Re(e^{-i pi k / (2N)} V_k), for any N.  v is
// real, so for even N it is packed two to a complex entry, z_n = v_{2n} +
// i v_{2n+1} (n < M = N/2), and only Z = DFT_M(z) is computed: the DFTs of
// the even and odd entries are E_k = (Z_k + conj Z_{M-k}) / 2 and
// O_k = (Z_k - conj Z_{M-k}) / (2i) (indices mod M), V_k = E_k +
// e^{-2 pi i k / N} O_k.  The DFT runs as Stockham autosort passes (one
// launch each, radices 4, 2, 3, 5, 7): pass with radix R and span Ns (the
// product of the earlier radices) reads x_{j + r L/R}, multiplies by
// e^{-2 pi i (j mod Ns) r / (Ns R)}, takes the R-point DFT (radix 3 and 5 in
// the symmetric form: sums and differences of the entries r and R - r) and
// writes it to (j div Ns) Ns R + (j mod Ns) + r Ns, so the output comes out
// in natural order.  Only the s sampled V_k are then formed.  Work per
// vector about 2.5 N log2 N flops instead of 2 s N; the complex buffers
// (2 per column) are the caller's scratch.
//
// Direct form (any other N): each output is a dot product of length N
// against a cosine table of period 4N (cos(pi j / (2N)), j = k (2n + 1) mod
// 4N, advanced by additions): O(s N) work per vector, one CTA per sampled
// row, fixed summation order.
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "skf_internal.cuh"

namespace skf {

namespace {

constexpr int kSrdctThreads = 256;
constexpr int kFftThreads = 256;

__device__ __forceinline__ bool srdct_stopped(const SrdctCols &cols) {
    return cols.iscal && cols.iscal[0] && cols.iscal[3] <= cols.step;   // the Arnoldi process stopped
}

// entry r of column q, widened exactly from F32 where the columns are F32
__device__ __forceinline__ double srdct_ld(const SrdctCols &cols, int q, int64_t r) {
    return cols.f32 ? (double)((const float *)cols.x[q])[r] : ((const double *)cols.x[q])[r];
}

__global__ void __launch_bounds__(kSrdctThreads) k_srdct(SrdctDev d, SrdctCols cols) {
    __shared__ double red[64];
    if (srdct_stopped(cols)) return;
    const int i = blockIdx.x;
    const int64_t k = d.P[i];
    const int64_t M4 = 4 * d.n;
    int64_t idx = (k * (2 * (int64_t)threadIdx.x + 1)) % M4;
    const int64_t stp = (2 * k * (int64_t)blockDim.x) % M4;
    double acc[2] = {0.0, 0.0};
    for (int64_t n = threadIdx.x; n < d.n; n += blockDim.x) {
        const double cs = d.costab[idx] * d.E[n];
        acc[0] = fma(srdct_ld(cols, 0, n), cs, acc[0]);
        if (cols.ncols > 1) acc[1] = fma(srdct_ld(cols, 1, n), cs, acc[1]);
        idx += stp;
        if (idx >= M4) idx -= M4;
    }
    block_sum<2>(acc, red);
    if (threadIdx.x == 0) {
        const double sk = sqrt((k == 0 ? 1.0 : 2.0) / (double)d.s);
        const double cscale = cols.colscale ? *cols.colscale : 1.0;
        for (int q = 0; q < cols.ncols; ++q) cols.out[q][i] = acc[q] * sk * cscale;
    }
}

// entry t of Makhoul's reordering v of E x (column q)
__device__ __forceinline__ double makhoul(const SrdctDev &d, const SrdctCols &cols, int q, int64_t t) {
    const int64_t src = t < (d.n + 1) / 2 ? 2 * t : 2 * (d.n - 1 - t) + 1;
    return d.E[src] * srdct_ld(cols, q, src);
}

// the FFT input of column blockIdx.y: z_t = v_{2t} + i v_{2t+1} (even n) or
// v_t (odd n)
__global__ void __launch_bounds__(kFftThreads) k_dct_permute(SrdctDev d, SrdctCols cols, double2 *dst) {
    if (srdct_stopped(cols)) return;
    const int q = blockIdx.y;
    const int64_t L = d.fft_len;
    const bool packed = 2 * L == d.n;
    double2 *z = dst + (size_t)q * L;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < L; t += (int64_t)gridDim.x * blockDim.x)
        z[t] = packed ? make_double2(makhoul(d, cols, q, 2 * t), makhoul(d, cols, q, 2 * t + 1))
                      : make_double2(makhoul(d, cols, q, t), 0.0);
}

// cos and sin of 2 pi k / R, k < R (host-computed)
struct RootTable {
    double c[8], s[8];
};

// one Stockham pass of radix R over each column (blockIdx.y)
// (length n; the twiddle table holds e^{-2 pi i t / (n twstride)})
template <int R>
__global__ void __launch_bounds__(kFftThreads) k_fft_pass(int64_t n, int64_t ns, const double2 *__restrict__ tw,
                                                         int64_t twstride, RootTable rt,
                                                         const double2 *__restrict__ src, double2 *__restrict__ dst,
                                                         SrdctCols cols) {
    if (srdct_stopped(cols)) return;
    src += (size_t)blockIdx.y * n;
    dst += (size_t)blockIdx.y * n;
    const int64_t nr = n / R;
    // twiddle index step: e^{-2 pi i k r / (ns R)} = tw[k r tstep]
    const int64_t tstep = n / (ns * R) * twstride;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += (int64_t)gridDim.x * blockDim.x) {
        double2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * nr];
        const int64_t k = j % ns;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const double2 w = tw[k * r * tstep];   // k r < ns R: the index stays below n twstride
            const double re = fma(v[r].x, w.x, -v[r].y * w.y);
            const double im = fma(v[r].x, w.y, v[r].y * w.x);
            v[r] = make_double2(re, im);
        }
        double2 o[R];
        if constexpr (R == 2) {
            o[0] = make_double2(v[0].x + v[1].x, v[0].y + v[1].y);
            o[1] = make_double2(v[0].x - v[1].x, v[0].y - v[1].y);
        } else if constexpr (R == 4) {
            const double2 t0 = make_double2(v[0].x + v[2].x, v[0].y + v[2].y);
            const double2 t1 = make_double2(v[0].x - v[2].x, v[0].y - v[2].y);
            const double2 t2 = make_double2(v[1].x + v[3].x, v[1].y + v[3].y);
            const double2 t3 = make_double2(v[1].x - v[3].x, v[1].y - v[3].y);
            o[0] = make_double2(t0.x + t2.x, t0.y + t2.y);
            o[2] = make_double2(t0.x - t2.x, t0.y - t2.y);
            o[1] = make_double2(t1.x + t3.y, t1.y - t3.x);   // t1 - i t3
            o[3] = make_double2(t1.x - t3.y, t1.y + t3.x);   // t1 + i t3
        } else if constexpr (R == 3) {
            // o_0 = v0 + t1, o_{1,2} = (v0 - t1 / 2) -/+ i sin(2 pi / 3) t2, t1 = v1 + v2, t2 = v1 - v2
            const double2 t1 = make_double2(v[1].x + v[2].x, v[1].y + v[2].y);
            const double2 t2 = make_double2(v[1].x - v[2].x, v[1].y - v[2].y);
            const double2 a = make_double2(fma(-0.5, t1.x, v[0].x), fma(-0.5, t1.y, v[0].y));
            const double2 b = make_double2(rt.s[1] * t2.x, rt.s[1] * t2.y);
            o[0] = make_double2(v[0].x + t1.x, v[0].y + t1.y);
            o[1] = make_double2(a.x + b.y, a.y - b.x);   // a - i b
            o[2] = make_double2(a.x - b.y, a.y + b.x);   // a + i b
        } else if constexpr (R == 5) {
            // t1 = v1 + v4, t2 = v2 + v3, t3 = v1 - v4, t4 = v2 - v3;
            // o_{1,4} = v0 + c1 t1 + c2 t2 -/+ i (s1 t3 + s2 t4),
            // o_{2,3} = v0 + c2 t1 + c1 t2 -/+ i (s2 t3 - s1 t4)  (c_k, s_k: cos, sin of 2 pi k / 5)
            const double2 t1 = make_double2(v[1].x + v[4].x, v[1].y + v[4].y);
            const double2 t2 = make_double2(v[2].x + v[3].x, v[2].y + v[3].y);
            const double2 t3 = make_double2(v[1].x - v[4].x, v[1].y - v[4].y);
            const double2 t4 = make_double2(v[2].x - v[3].x, v[2].y - v[3].y);
            const double c1 = rt.c[1], c2 = rt.c[2], s1 = rt.s[1], s2 = rt.s[2];
            const double2 a1 = make_double2(fma(c2, t2.x, fma(c1, t1.x, v[0].x)), fma(c2, t2.y, fma(c1, t1.y, v[0].y)));
            const double2 a2 = make_double2(fma(c1, t2.x, fma(c2, t1.x, v[0].x)), fma(c1, t2.y, fma(c2, t1.y, v[0].y)));
            const double2 b1 = make_double2(fma(s2, t4.x, s1 * t3.x), fma(s2, t4.y, s1 * t3.y));
            const double2 b2 = make_double2(fma(-s1, t4.x, s2 * t3.x), fma(-s1, t4.y, s2 * t3.y));
            o[0] = make_double2(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
            o[1] = make_double2(a1.x + b1.y, a1.y - b1.x);
            o[4] = make_double2(a1.x - b1.y, a1.y + b1.x);
            o[2] = make_double2(a2.x + b2.y, a2.y - b2.x);
            o[3] = make_double2(a2.x - b2.y, a2.y + b2.x);
        } else {
            // direct R-point DFT: o_t = sum_q v_q e^{-2 pi i q t / R}
#pragma unroll
            for (int t = 0; t < R; ++t) {
                double re = v[0].x, im = v[0].y;
#pragma unroll
                for (int q = 1; q < R; ++q) {
                    const int e = (q * t) % R;
                    re = fma(v[q].x, rt.c[e], fma(v[q].y, rt.s[e], re));
                    im = fma(v[q].y, rt.c[e], fma(-v[q].x, rt.s[e], im));
                }
                o[t] = make_double2(re, im);
            }
        }
        const int64_t base = (j / ns) * ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + r * ns] = o[r];
    }
}

// out[q][i] = colscale Re(twist_i V_k), k = P_i; V_k from the FFT output Z
// (even n: V_k = E_k + e^{-2 pi i k / n} O_k from Z_{k mod M} and Z_{M - k mod M})
__global__ void __launch_bounds__(kFftThreads) k_dct_gather(SrdctDev d, SrdctCols cols, const double2 *Zall) {
    if (srdct_stopped(cols)) return;
    const int q = blockIdx.y;
    const int64_t L = d.fft_len;
    const double2 *Z = Zall + (size_t)q * L;
    const double cscale = cols.colscale ? *cols.colscale : 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.s; i += gridDim.x * blockDim.x) {
        const int64_t k = d.P[i];
        double2 V;
        if (2 * L == d.n) {
            const int64_t kk = k % L, kc = (L - kk) % L;
            const double2 z1 = Z[kk], z2 = Z[kc];          // z2 enters conjugated
            const double2 e = make_double2(0.5 * (z1.x + z2.x), 0.5 * (z1.y - z2.y));
            const double2 o = make_double2(0.5 * (z1.y + z2.y), -0.5 * (z1.x - z2.x));   // (z1 - conj z2) / (2i)
            const double2 w = d.tw[k];
            V = make_double2(e.x + fma(w.x, o.x, -w.y * o.y), e.y + fma(w.x, o.y, w.y * o.x));
        } else {
            V = Z[k];
        }
        const double2 t = d.twist[i];
        cols.out[q][i] = fma(t.x, V.x, -t.y * V.y) * cscale;
    }
}

RootTable root_table(int R) {
    RootTable rt{};
    for (int k = 0; k < R; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)R;
        rt.c[k] = cos(a);
        rt.s[k] = sin(a);
    }
    return rt;
}

void fft_launch(const SrdctDev &d, const SrdctCols &cols, cudaStream_t st) {
    const int64_t n = d.fft_len;
    const int64_t twstride = d.n / n;
    double2 *a = d.work, *b = d.work + 2 * (size_t)n;
    const unsigned ny = (unsigned)cols.ncols;
    auto grid = [&](int64_t items) {
        return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((items + kFftThreads - 1) / kFftThreads,
                                                                       8ll * num_sms())), ny);
    };
    k_dct_permute<<<grid(n), kFftThreads, 0, st>>>(d, cols, a);
    int64_t ns = 1;
    for (int p = 0; p < d.nrad; ++p) {
        const int R = d.rad[p];
        const RootTable rt = root_table(R);
        const dim3 g = grid(n / R);
        switch (R) {
            case 2: k_fft_pass<2><<<g, kFftThreads, 0, st>>>(n, ns, d.tw, twstride, rt, a, b, cols); break;
            case 3: k_fft_pass<3><<<g, kFftThreads, 0, st>>>(n, ns, d.tw, twstride, rt, a, b, cols); break;
            case 4: k_fft_pass<4><<<g, kFftThreads, 0, st>>>(n, ns, d.tw, twstride, rt, a, b, cols); break;
            case 5: k_fft_pass<5><<<g, kFftThreads, 0, st>>>(n, ns, d.tw, twstride, rt, a, b, cols); break;
            default: k_fft_pass<7><<<g, kFftThreads, 0, st>>>(n, ns, d.tw, twstride, rt, a, b, cols); break;
        }
        ns *= R;
        std::swap(a, b);
    }
    k_dct_gather<<<grid(d.s), kFftThreads, 0, st>>>(d, cols, a);
    count_launches(2 + d.nrad);
}

}  // namespace

size_t srdct_work_bytes(const skf_sketch *S) {
    return S->fft_len > 0 ? sizeof(double2) * 4 * (size_t)S->fft_len : 0;
}

SrdctDev make_srdct(const skf_sketch *S) {
    SrdctDev d{};
    d.n = S->n;
    d.s = S->s;
    d.P = S->P;
    d.E = S->E;
    d.costab = S->costab;
    d.fft_len = S->fft_len;
    d.nrad = S->nrad;
    for (int i = 0; i < S->nrad; ++i) d.rad[i] = S->rad[i];
    d.tw = S->tw;
    d.twist = S->twist;
    d.work = nullptr;
    return d;
}

skf_status build_srdct_tables(skf_sketch *S) {
    if ((int64_t)S->s > S->n) return fail(SKF_ERR_INVALID_ARG, "SRDCT needs s <= N");
    S->np = S->n;
    skf_status st = build_sampled_rows(S, S->n);
    if (st != SKF_OK) return st;
    const int64_t n = S->n;
    std::vector<double> E((size_t)n);
    for (int64_t c = 0; c < n; ++c) E[c] = (splitmix_word(S->seed, (uint64_t)c) & 1ull) ? -1.0 : 1.0;
    if (cudaMalloc(&S->E, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(SKF_ERR_OOM, "SRDCT table allocation");
    }
    if (cudaMemcpy(S->E, E.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "SRDCT table upload");
    // FFT length (real input packed two to an entry for even n); radices 4
    // first, then 2, 3, 5, 7; the FFT form if nothing is left over
    const int64_t len = (n % 2 == 0) ? n / 2 : n;
    int64_t rest = len;
    int nrad = 0;
    int rad[64];
    for (int p : {4, 2, 3, 5, 7})
        while (rest % p == 0 && rest > 1 && nrad < 64) {
            rad[nrad++] = p;
            rest /= p;
        }
    if (rest == 1 && n >= 2) {
        S->fft_len = len;
        S->nrad = nrad;
        for (int i = 0; i < nrad; ++i) S->rad[i] = rad[i];
        std::vector<double2> tw((size_t)n), twist((size_t)S->s);
        for (int64_t t = 0; t < n; ++t) {
            const double a = 2.0 * M_PI * ((double)t / (double)n);
            tw[t] = make_double2(cos(a), -sin(a));
        }
        std::vector<int32_t> P((size_t)S->s);
        if (cudaMemcpy(P.data(), S->P, sizeof(int32_t) * S->s, cudaMemcpyDeviceToHost) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "SRDCT sampled rows");
        for (int i = 0; i < S->s; ++i) {
            const int64_t k = P[i];
            const double a = M_PI * (double)k / (2.0 * (double)n);
            const double sc = sqrt((k == 0 ? 1.0 : 2.0) / (double)S->s);   // a_k sqrt(N / s)
            twist[i] = make_double2(cos(a) * sc, -sin(a) * sc);
        }
        if (cudaMalloc(&S->tw, sizeof(double2) * n) != cudaSuccess ||
            cudaMalloc(&S->twist, sizeof(double2) * S->s) != cudaSuccess) {
            cudaGetLastError();
            return fail(SKF_ERR_OOM, "SRDCT FFT table allocation");
        }
        if (cudaMemcpy(S->tw, tw.data(), sizeof(double2) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(S->twist, twist.data(), sizeof(double2) * S->s, cudaMemcpyHostToDevice) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "SRDCT FFT table upload");
        return SKF_OK;
    }
    std::vector<double> tab((size_t)(4 * n));
    for (int64_t j = 0; j < 4 * n; ++j) tab[j] = cos(M_PI * (double)j / (2.0 * (double)n));
    if (cudaMalloc(&S->costab, sizeof(double) * 4 * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(SKF_ERR_OOM, "SRDCT table allocation");
    }
    if (cudaMemcpy(S->costab, tab.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "SRDCT table upload");
    return SKF_OK;
}

void srdct_launch(const SrdctDev &d, const SrdctCols &cols, cudaStream_t st) {
    if (d.fft_len > 0 && d.work != nullptr) {
        fft_launch(d, cols, st);
        return;
    }
    k_srdct<<<d.s, kSrdctThreads, 0, st>>>(d, cols);
    count_launches(1);
}

skf_status srdct_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                           cudaStream_t st) {
    SrdctDev d = make_srdct(S);
    const size_t wb = srdct_work_bytes(S);
    if (wb > 0) {
        skf_status e = dalloc((void **)&d.work, wb, st);
        if (e != SKF_OK) return e;
    }
    for (int c0 = 0; c0 < ncols; c0 += 2) {
        SrdctCols cols{};
        cols.ncols = ncols - c0 < 2 ? ncols - c0 : 2;
        for (int q = 0; q < cols.ncols; ++q) {
            cols.x[q] = X + (size_t)(c0 + q) * ldx;
            cols.out[q] = SX + (size_t)(c0 + q) * S->s;
        }
        srdct_launch(d, cols, st);
    }
    if (d.work) dfree(d.work, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "SRDCT kernels");
    return SKF_OK;
}

}  // namespace skf
