// Application of the subspace embedding S (eq. (1.1)) to general vectors:
// column maxima, fixed-point scatter into per-CTA shared-memory bins, and an
// exact cross-CTA reduction.  The same device routines are used inside the
// Arnoldi kernels.
#include <math.h>

#include "skf_internal.cuh"

namespace skf {

SparseSign make_sparse_sign(const skf_sketch *S) {
    SparseSign sp{};
    sp.s = S->s;
    sp.zeta = S->zeta;
    sp.words = (S->zeta + 3) / 4;
    sp.seed = S->seed;
    for (int q = 0; q < S->zeta; ++q) {
        const int a = (int)(((long long)q * S->s) / S->zeta);
        const int b = (int)(((long long)(q + 1) * S->s) / S->zeta);
        sp.start[q] = a;
        sp.size[q] = b - a;
    }
    return sp;
}

namespace {

// Per-CTA partial max |X[:, col]| for every column.
__global__ void k_colmax(const double *__restrict__ X, int64_t ldx, int64_t n, int ncols, int64_t rows_per_cta,
                         double *__restrict__ part /* [ncols][G] */) {
    __shared__ double red[32];
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    for (int c = 0; c < ncols; ++c) {
        double mx = 0.0;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) mx = fmax(mx, fabs(X[r + c * ldx]));
        mx = block_max(mx, red);
        if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = mx;
    }
}

// Scatter of the rows of this CTA into fixed-point bins; writes the int64
// partial sums [ncols][G][s].
__global__ void k_sparse_sign_scatter(const double *__restrict__ X, int64_t ldx, int64_t n, int ncols,
                                      int64_t rows_per_cta, SparseSign sp, int frac_bits,
                                      const double *__restrict__ maxpart, long long *__restrict__ out) {
    extern __shared__ uint32_t bins[];   // lo[s], hi[s]
    __shared__ double red[32];
    uint32_t *lo = bins, *hi = bins + sp.s;
    const int G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    for (int c = 0; c < ncols; ++c) {
        double mx = 0.0;
        for (int g = threadIdx.x; g < G; g += kThreads) mx = fmax(mx, maxpart[(size_t)c * G + g]);
        mx = block_max(mx, red);
        for (int i = threadIdx.x; i < 2 * sp.s; i += kThreads) bins[i] = 0u;
        __syncthreads();
        if (mx > 0.0) {
            const int shift = frac_bits - bound_exponent(mx);
            for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) {
                const long long v = fixed_point(X[r + c * ldx], shift);
                if (v == 0) continue;
                uint64_t word = 0;
                for (int q = 0; q < sp.zeta; ++q) {
                    if ((q & 3) == 0) word = splitmix_word(sp.seed, (uint64_t)r * sp.words + (q >> 2));
                    int row;
                    bool neg;
                    sparse_sign_entry(sp, word, q, row, neg);
                    atomic_add_i64_split(lo + row, hi + row, neg ? -v : v);
                }
            }
        }
        __syncthreads();
        long long *o = out + ((size_t)c * G + blockIdx.x) * sp.s;
        for (int i = threadIdx.x; i < sp.s; i += kThreads)
            o[i] = (long long)(((unsigned long long)hi[i] << 32) | lo[i]);
        __syncthreads();
    }
}

// SX[i, c] = 2^-frac * 2^E_c * zeta^-1/2 * sum_g partial[c][g][i].
__global__ void k_sparse_sign_reduce(const long long *__restrict__ part, const double *__restrict__ maxpart, int G,
                                     int s, int ncols, int zeta, int frac_bits, double *__restrict__ SX) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)s * ncols) return;
    const int c = (int)(idx / s), i = (int)(idx % s);
    double mx = 0.0;
    for (int g = 0; g < G; ++g) mx = fmax(mx, maxpart[(size_t)c * G + g]);
    if (mx == 0.0) {
        SX[idx] = 0.0;
        return;
    }
    const double tot = sum_i64_exact(part + (size_t)c * G * s + i, G, (size_t)s);
    SX[idx] = ldexp(tot, bound_exponent(mx) - frac_bits) / sqrt((double)zeta);
}

__global__ void k_copy_cols(const double *__restrict__ X, int64_t ldx, int64_t n, int ncols, double *__restrict__ Y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * ncols) return;
    const int64_t c = idx / n, r = idx % n;
    Y[idx] = X[r + c * ldx];
}

}  // namespace

skf_status sketch_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                            cudaStream_t st) {
    const int64_t n = S->n;
    if (ncols <= 0) return SKF_OK;
    if (S->kind == SKF_SKETCH_IDENTITY) {
        const int64_t tot = n * ncols;
        k_copy_cols<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, ldx, n, ncols, SX);
        SKF_LAUNCH_CHECK("k_copy_cols");
        return SKF_OK;
    }
    if (S->kind != SKF_SKETCH_SPARSE_SIGN) return fail(SKF_ERR_NOT_SUPPORTED, "sketch kind not implemented");
    const SparseSign sp = make_sparse_sign(S);
    int G = 2 * num_sms();
    const int64_t min_rows = 1024;
    if ((n + min_rows - 1) / min_rows < G) G = (int)((n + min_rows - 1) / min_rows);
    if (G < 1) G = 1;
    const int64_t rows = (n + G - 1) / G;
    const int frac = sketch_fraction_bits(rows);
    double *maxpart = nullptr;
    long long *part = nullptr;
    skf_status stt = dalloc((void **)&maxpart, sizeof(double) * G * ncols, st);
    if (stt != SKF_OK) return stt;
    stt = dalloc((void **)&part, sizeof(long long) * (size_t)G * ncols * S->s, st);
    if (stt != SKF_OK) {
        dfree(maxpart, st);
        return stt;
    }
    k_colmax<<<G, kThreads, 0, st>>>(X, ldx, n, ncols, rows, maxpart);
    const size_t smem = sizeof(uint32_t) * 2 * S->s;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_sparse_sign_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_sparse_sign_scatter<<<G, kThreads, smem, st>>>(X, ldx, n, ncols, rows, sp, frac, maxpart, part);
    const int64_t tot = (int64_t)S->s * ncols;
    k_sparse_sign_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, maxpart, G, S->s, ncols, S->zeta, frac,
                                                                        SX);
    cudaError_t e = cudaGetLastError();
    dfree(part, st);
    dfree(maxpart, st);
    if (e != cudaSuccess) return cuda_fail(e, "sketch_apply kernels");
    return SKF_OK;
}

}  // namespace skf
