// Subsampled randomized Hadamard transform (the SRHT variant of the sketch,
// Sec. 2.2; S = P F E of Sec. 5.1 with F the Walsh-Hadamard transform):
//   S x = s^{-1/2} (H_{N'} (E x, zero-padded to N'))[P],
// H unnormalised in Sylvester order, E = diag of signs from the counter hash
// (bit 0 of word(seed, i)), P the first s entries of a seeded partial
// Fisher-Yates shuffle of 0..N'-1 (words of the hash with seed mix64(seed)).
//
// Computed exactly in integers, in one pass over x: each value becomes a
// fixed-point int64 (62 - b fraction bits below the column's maximum, integer
// bit operations only), and H_{N'} = H_{N'/2^b} (x) H_{2^b} splits the
// transform: every CTA transforms one block of 2^b consecutive entries in
// shared memory (exact integer butterflies), then emits, for each sampled
// row p = p_hi 2^b + p_lo, its contribution (-1)^{popc(p_hi & block)} u[p_lo].
// The per-block contributions are summed exactly (128-bit) in block order.
#include <math.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "skf_internal.cuh"
#include "skf_step.cuh"

namespace skf {

namespace {

constexpr int kSrhtThreads = 512;

// Fixed-point transform of one 2^b block of up to two columns; partials
// part[c][blk * s + o] for the s sampled rows.
__global__ void __launch_bounds__(kSrhtThreads) k_srht_blocks(SrhtDev d, SrhtCols cols) {
    extern __shared__ long long z[];   // [2^b]
    if (cols.iscal && cols.iscal[0] && cols.iscal[3] <= cols.step) return;   // the Arnoldi process stopped
    const int c = blockIdx.y;
    const int blk = blockIdx.x;
    const int B = 1 << d.b;
    const int E = *cols.e[c];
    long long *part = cols.part[c] + (size_t)blk * d.s;
    if (E == kNoExp) {   // zero column
        for (int o = threadIdx.x; o < d.s; o += blockDim.x) part[o] = 0;
        return;
    }
    const int shift = d.frac - E;
    const int64_t r0 = (int64_t)blk * B;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const int64_t r = r0 + i;
        long long v = 0;
        if (r < d.n) {
            const double xr = cols.f32 ? (double)((const float *)cols.x[c])[r] : ((const double *)cols.x[c])[r];
            v = fixed_point(xr, shift);
            if (splitmix_word(d.seed, (uint64_t)r) & 1ull) v = -v;
        }
        z[i] = v;
    }
    __syncthreads();
    // Sylvester-ordered butterflies, stride h = 1, 2, ..., B / 2
    for (int h = 1; h < B; h <<= 1) {
        for (int t = threadIdx.x; t < B / 2; t += blockDim.x) {
            const int i = (t / h) * 2 * h + (t % h);
            const long long a = z[i], bb = z[i + h];
            z[i] = a + bb;
            z[i + h] = a - bb;
        }
        __syncthreads();
    }
    for (int o = threadIdx.x; o < d.s; o += blockDim.x) {
        const int64_t p = d.P[o];
        const long long u = z[p & (B - 1)];
        part[o] = (__popcll((unsigned long long)((p >> d.b) & (int64_t)blk)) & 1) ? -u : u;
    }
}

// Exponent bound of each column's maximum (kNoExp for a zero column).
__global__ void k_col_exponent(const double *__restrict__ maxpart, int G, int ncols, int *__restrict__ E) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double mx = 0.0;
    for (int g = 0; g < G; ++g) mx = fmax(mx, maxpart[(size_t)c * G + g]);
    E[c] = mx > 0.0 ? bound_exponent(mx) : kNoExp;
}

// SX[:, c] from the block partials, one thread per output (blocks summed
// exactly in block order).
__global__ void k_srht_reduce(SrhtDev d, const long long *__restrict__ part, const int *__restrict__ E, int ncols,
                              double scale, double *__restrict__ SX) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)d.s * ncols) return;
    const int c = (int)(idx / d.s), o = (int)(idx % d.s);
    if (E[c] == kNoExp) {
        SX[idx] = 0.0;
        return;
    }
    const double tot = sum_i64_exact(part + (size_t)c * d.nblk * d.s + o, d.nblk, (size_t)d.s);
    SX[idx] = scale_pow2(tot, E[c] - d.frac) * scale;
}

// Per-CTA partial max |X[:, c]| (rows of CTA g: g, g + G, ...).
__global__ void k_colmax_srht(const double *__restrict__ X, int64_t ldx, int64_t n, int ncols,
                              double *__restrict__ part) {
    __shared__ double red[32];
    for (int c = 0; c < ncols; ++c) {
        double mx = 0.0;
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
            mx = fmax(mx, fabs(X[r + c * ldx]));
        mx = block_max(mx, red);
        if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = mx;
    }
}

// Per-CTA partial max |x| of up to two F32 columns (rows g, g + G, ...),
// nothing once the Arnoldi process stopped.
__global__ void k_colmax_f32(DenseCols cols, int64_t n, double *__restrict__ part) {
    __shared__ double red[32];
    if (cols.iscal && cols.iscal[0] && cols.iscal[3] <= cols.step) return;
    for (int c = 0; c < cols.ncols; ++c) {
        double mx = 0.0;
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
            mx = fmax(mx, fabs((double)cols.x[c][r]));
        mx = block_max(mx, red);
        if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = mx;
    }
}

// out[c][o] = colscale s^{-1/2} (sum of the block partials), as k_srht_reduce
__global__ void k_srht_reduce_cols(SrhtDev d, DenseCols cols, const long long *__restrict__ part,
                                   const int *__restrict__ E) {
    if (cols.iscal && cols.iscal[0] && cols.iscal[3] <= cols.step) return;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)d.s * cols.ncols) return;
    const int c = (int)(idx / d.s), o = (int)(idx % d.s);
    const double cs = cols.colscale ? *cols.colscale : 1.0;
    if (E[c] == kNoExp) {
        cols.out[c][o] = 0.0;
        return;
    }
    const double tot = sum_i64_exact(part + (size_t)c * d.nblk * d.s + o, d.nblk, (size_t)d.s);
    cols.out[c][o] = scale_pow2(tot, E[c] - d.frac) * (1.0 / sqrt((double)d.s)) * cs;
}

}  // namespace

SrhtDev make_srht(const skf_sketch *S) {
    SrhtDev d{};
    d.n = S->n;
    d.np = S->np;
    d.s = S->s;
    d.seed = S->seed;
    d.P = S->P;
    int lg = 0;
    while ((1ll << lg) < S->np) ++lg;
    d.b = std::min(lg, kSrhtBlockLog2);
    d.nblk = (int)(S->np >> d.b);
    d.frac = 62 - d.b;   // |block transform| < 2^(frac + b) <= 2^62
    return d;
}

skf_status build_srht_tables(skf_sketch *S) {
    int64_t np = 1;
    while (np < S->n) np <<= 1;
    if ((int64_t)S->s > np) return fail(SKF_ERR_INVALID_ARG, "SRHT needs s <= N' = 2^ceil(log2 N)");
    S->np = np;
    return build_sampled_rows(S, np);
}

skf_status build_sampled_rows(skf_sketch *S, int64_t np) {
    // P: first s entries of a partial Fisher-Yates shuffle of 0..np-1
    const uint64_t seed2 = mix64(S->seed);
    std::unordered_map<int64_t, int64_t> swapped;
    std::vector<int32_t> P(S->s);
    for (int i = 0; i < S->s; ++i) {
        const uint64_t word = splitmix_word(seed2, (uint64_t)i);
        const int64_t j = i + (int64_t)(word % (uint64_t)(np - i));
        auto gi = swapped.find(i);
        auto gj = swapped.find(j);
        const int64_t vi = gi == swapped.end() ? i : gi->second;
        const int64_t vj = gj == swapped.end() ? j : gj->second;
        swapped[i] = vj;
        swapped[j] = vi;
        P[i] = (int32_t)vj;
    }
    if (cudaMalloc(&S->P, sizeof(int32_t) * S->s) != cudaSuccess) {
        cudaGetLastError();
        S->P = nullptr;
        return fail(SKF_ERR_OOM, "SRHT row table allocation");
    }
    if (cudaMemcpy(S->P, P.data(), sizeof(int32_t) * S->s, cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "SRHT row table upload");
    return SKF_OK;
}

void srht_launch(const SrhtDev &d, const SrhtCols &cols, cudaStream_t st) {
    const size_t smem = sizeof(long long) << d.b;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_srht_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_srht_blocks<<<dim3((unsigned)d.nblk, (unsigned)cols.ncols), kSrhtThreads, smem, st>>>(d, cols);
    count_launches(1);
}

skf_status srht_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX, cudaStream_t st) {
    if (ncols <= 0) return SKF_OK;
    const SrhtDev d = make_srht(S);
    const int G = std::max(1, std::min(2 * num_sms(), (int)((S->n + kThreads - 1) / kThreads)));
    double *maxpart = nullptr;
    int *E = nullptr;
    long long *part = nullptr;
    skf_status stt = dalloc((void **)&maxpart, sizeof(double) * G * ncols, st);
    if (stt == SKF_OK) stt = dalloc((void **)&E, sizeof(int) * ncols, st);
    if (stt == SKF_OK) stt = dalloc((void **)&part, sizeof(long long) * (size_t)ncols * d.nblk * d.s, st);
    if (stt == SKF_OK) {
        k_colmax_srht<<<G, kThreads, 0, st>>>(X, ldx, S->n, ncols, maxpart);
        k_col_exponent<<<(ncols + 127) / 128, 128, 0, st>>>(maxpart, G, ncols, E);
        count_launches(2);
        for (int c0 = 0; c0 < ncols; c0 += 2) {
            SrhtCols cols{};
            cols.ncols = std::min(2, ncols - c0);
            for (int q = 0; q < cols.ncols; ++q) {
                cols.x[q] = X + (size_t)(c0 + q) * ldx;
                cols.e[q] = E + c0 + q;
                cols.part[q] = part + (size_t)(c0 + q) * d.nblk * d.s;
            }
            srht_launch(d, cols, st);
        }
        const int64_t tot = (int64_t)d.s * ncols;
        k_srht_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(d, part, E, ncols, 1.0 / sqrt((double)d.s), SX);
        count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (part) dfree(part, st);
    if (E) dfree(E, st);
    if (maxpart) dfree(maxpart, st);
    if (stt != SKF_OK) return stt;
    if (e != cudaSuccess) return cuda_fail(e, "SRHT kernels");
    return SKF_OK;
}

size_t dense_sketch_work_bytes(const skf_sketch *S) {
    if (S->kind == SKF_SKETCH_SRDCT) return srdct_work_bytes(S);
    if (S->kind != SKF_SKETCH_SRHT) return 0;
    const SrhtDev d = make_srht(S);
    const int G = std::max(1, std::min(2 * num_sms(), (int)((S->n + kThreads - 1) / kThreads)));
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return al(sizeof(double) * 2 * G) + al(sizeof(int) * 2) + al(sizeof(long long) * 2 * (size_t)d.nblk * d.s);
}

void dense_sketch_f32(const skf_sketch *S, const DenseCols &cols, void *work, cudaStream_t st) {
    if (S->kind == SKF_SKETCH_SRDCT) {
        SrdctDev d = make_srdct(S);
        d.work = (double2 *)work;
        SrdctCols sc{};
        sc.ncols = cols.ncols;
        for (int q = 0; q < cols.ncols; ++q) {
            sc.x[q] = cols.x[q];
            sc.out[q] = cols.out[q];
        }
        sc.colscale = cols.colscale;
        sc.iscal = cols.iscal;
        sc.step = cols.step;
        sc.f32 = 1;
        srdct_launch(d, sc, st);
        return;
    }
    // SRHT: column maxima, exponent bounds, exact block transforms, reduction
    const SrhtDev d = make_srht(S);
    const int G = std::max(1, std::min(2 * num_sms(), (int)((S->n + kThreads - 1) / kThreads)));
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    double *maxpart = (double *)work;
    int *E = (int *)((char *)work + al(sizeof(double) * 2 * G));
    long long *part = (long long *)((char *)E + al(sizeof(int) * 2));
    k_colmax_f32<<<G, kThreads, 0, st>>>(cols, S->n, maxpart);
    k_col_exponent<<<1, 128, 0, st>>>(maxpart, G, cols.ncols, E);
    SrhtCols hc{};
    hc.ncols = cols.ncols;
    for (int q = 0; q < cols.ncols; ++q) {
        hc.x[q] = cols.x[q];
        hc.e[q] = E + q;
        hc.part[q] = part + (size_t)q * d.nblk * d.s;
    }
    hc.iscal = cols.iscal;
    hc.step = cols.step;
    hc.f32 = 1;
    srht_launch(d, hc, st);
    const int64_t tot = (int64_t)d.s * cols.ncols;
    k_srht_reduce_cols<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(d, cols, part, E);
    count_launches(3);
}

}  // namespace skf
