// Subsampled randomized discrete cosine transform (the sketch of the paper's
// experiments, Sec. 5.1: S = P F E with F a DCT):
//   (S x)_i = sqrt(N/s) (F E x)_{P_i},  F the orthonormal DCT-II,
//   (F y)_k = a_k sum_n y_n cos(pi k (2n + 1) / (2N)),  a_0 = 1/sqrt(N), a_k = sqrt(2/N),
// E the signs of the SRHT definition and P the first s entries of its partial
// Fisher-Yates shuffle, of [0, N).  Only the s sampled rows of F are needed,
// so each output is a direct dot product of length N against a cosine table
// of period 4N (cos(pi j / (2N)), j = k (2n + 1) mod 4N, advanced by additions):
// O(s N) work per vector, one CTA per sampled row, fixed summation order.
#include <math.h>

#include <vector>

#include "skf_internal.cuh"

namespace skf {

namespace {

constexpr int kSrdctThreads = 256;

__global__ void __launch_bounds__(kSrdctThreads) k_srdct(SrdctDev d, SrdctCols cols) {
    __shared__ double red[64];
    if (cols.iscal && cols.iscal[0] && cols.iscal[3] <= cols.step) return;   // the Arnoldi process stopped
    const int i = blockIdx.x;
    const int64_t k = d.P[i];
    const int64_t M4 = 4 * d.n;
    int64_t idx = (k * (2 * (int64_t)threadIdx.x + 1)) % M4;
    const int64_t stp = (2 * k * (int64_t)blockDim.x) % M4;
    double acc[2] = {0.0, 0.0};
    for (int64_t n = threadIdx.x; n < d.n; n += blockDim.x) {
        const double cs = d.costab[idx] * d.E[n];
        acc[0] = fma(cols.x[0][n], cs, acc[0]);
        if (cols.ncols > 1) acc[1] = fma(cols.x[1][n], cs, acc[1]);
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

}  // namespace

SrdctDev make_srdct(const skf_sketch *S) {
    SrdctDev d{};
    d.n = S->n;
    d.s = S->s;
    d.P = S->P;
    d.E = S->E;
    d.costab = S->costab;
    return d;
}

skf_status build_srdct_tables(skf_sketch *S) {
    if ((int64_t)S->s > S->n) return fail(SKF_ERR_INVALID_ARG, "SRDCT needs s <= N");
    S->np = S->n;
    skf_status st = build_sampled_rows(S, S->n);
    if (st != SKF_OK) return st;
    const int64_t n = S->n;
    std::vector<double> E((size_t)n), tab((size_t)(4 * n));
    for (int64_t c = 0; c < n; ++c) E[c] = (splitmix_word(S->seed, (uint64_t)c) & 1ull) ? -1.0 : 1.0;
    for (int64_t j = 0; j < 4 * n; ++j) tab[j] = cos(M_PI * (double)j / (2.0 * (double)n));
    if (cudaMalloc(&S->E, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&S->costab, sizeof(double) * 4 * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(SKF_ERR_OOM, "SRDCT table allocation");
    }
    if (cudaMemcpy(S->E, E.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(S->costab, tab.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "SRDCT table upload");
    return SKF_OK;
}

void srdct_launch(const SrdctDev &d, const SrdctCols &cols, cudaStream_t st) {
    k_srdct<<<d.s, kSrdctThreads, 0, st>>>(d, cols);
    count_launches(1);
}

skf_status srdct_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                           cudaStream_t st) {
    const SrdctDev d = make_srdct(S);
    for (int c0 = 0; c0 < ncols; c0 += 2) {
        SrdctCols cols{};
        cols.ncols = ncols - c0 < 2 ? ncols - c0 : 2;
        for (int q = 0; q < cols.ncols; ++q) {
            cols.x[q] = X + (size_t)(c0 + q) * ldx;
            cols.out[q] = SX + (size_t)(c0 + q) * S->s;
        }
        srdct_launch(d, cols, st);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "SRDCT kernel");
    return SKF_OK;
}

}  // namespace skf
