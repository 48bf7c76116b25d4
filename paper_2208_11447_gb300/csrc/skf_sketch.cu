// The subspace embedding S (eq. (1.1)): expansion of the sparse-sign pattern
// from its SplitMix64 definition, the per-partition bin-load maxima that
// size the fixed-point limbs, and S X for general X (column maxima,
// fixed-point scatter into per-CTA shared-memory bins, exact cross-CTA
// reduction).  The Arnoldi kernels use the same pattern and accumulation.
#include <math.h>

#include <algorithm>
#include <mutex>

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

void row_partition(int64_t n, int *G, int64_t *rows) {
    int g = 2 * num_sms();
    const int64_t min_rows = 512;
    if ((n + min_rows - 1) / min_rows < g) g = (int)((n + min_rows - 1) / min_rows);
    if (g < 1) g = 1;
    *G = g;
    *rows = ((n + g - 1) / g + 31) / 32 * 32;   // whole SELL slices per CTA
}

void chunk_partition(int64_t n, int *G) {
    const int64_t chunks = (n + kChunkRows - 1) / kChunkRows;
    int g = num_sms();
    if (chunks < g) g = (int)chunks;
    *G = g < 1 ? 1 : g;
}

namespace {

// pattern[c * zeta + q] = (row of nonzero q of column c within stripe q) | sign << 15
__global__ void k_build_pattern(SparseSign sp, int64_t n, uint16_t *__restrict__ pattern) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        uint64_t word = 0;
        for (int q = 0; q < sp.zeta; ++q) {
            if ((q & 3) == 0) word = splitmix_word(sp.seed, (uint64_t)c * sp.words + (q >> 2));
            int row;
            bool neg;
            sparse_sign_entry(sp, word, q, row, neg);
            pattern[c * sp.zeta + q] = (uint16_t)((row - sp.start[q]) | (neg ? 0x8000 : 0));
        }
    }
}

// The same pattern in bytes (row within stripe + block * sign, block = 64 or
// 128), eight per column.
__global__ void k_build_pattern8(SparseSign sp, int64_t n, int block, const uint16_t *__restrict__ pattern,
                                 uint8_t *__restrict__ p8) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        for (int q = 0; q < 8; ++q) {
            uint8_t v = 0;
            if (q < sp.zeta) {
                const uint16_t e = pattern[c * sp.zeta + q];
                v = (uint8_t)((e & 0x7FFFu) + ((e >> 15) ? block : 0));
            }
            p8[c * 8 + q] = v;
        }
}

// Largest number of nonzeros that one CTA's rows put into one row of S.  CTA
// g owns the chunks g, g + G, g + 2G, ... of `chunk` rows (one chunk per CTA
// for the contiguous partition).
__global__ void k_bin_max(SparseSign sp, int64_t n, int64_t chunk, const uint16_t *__restrict__ pattern,
                          int *binmax) {
    extern __shared__ int cnt[];
    for (int i = threadIdx.x; i < sp.s; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int64_t r0 = (int64_t)blockIdx.x * chunk; r0 < n; r0 += (int64_t)gridDim.x * chunk) {
        const int64_t r1 = min(n, r0 + chunk);
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
            for (int q = 0; q < sp.zeta; ++q) {
                int row;
                bool neg;
                pattern_entry(sp, pattern[r * sp.zeta + q], q, row, neg);
                atomicAdd(cnt + row, 1);
            }
    }
    __syncthreads();
    int mx = 0;
    for (int i = threadIdx.x; i < sp.s; i += blockDim.x) mx = max(mx, cnt[i]);
    atomicMax(binmax, mx);
}

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

// Scatter of the rows of this CTA into fixed-point limb bins; writes the
// int64 partial sums [ncols][G][s].
__global__ void k_sparse_sign_scatter(const double *__restrict__ X, int64_t ldx, int64_t n, int ncols,
                                      int64_t rows_per_cta, SparseSign sp, const uint16_t *__restrict__ pattern,
                                      const int *__restrict__ binmax, const double *__restrict__ maxpart,
                                      long long *__restrict__ out) {
    extern __shared__ int bins[];   // acc0[s], acc1[s]
    __shared__ double red[32];
    int *acc0 = bins, *acc1 = bins + sp.s;
    const int G = gridDim.x;
    const int L = limb_bits(*binmax);
    const int frac = sketch_fraction_bits_from_limb(L);
    const long long lmask = (1ll << L) - 1;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    for (int c = 0; c < ncols; ++c) {
        double mx = 0.0;
        for (int g = threadIdx.x; g < G; g += kThreads) mx = fmax(mx, maxpart[(size_t)c * G + g]);
        mx = block_max(mx, red);
        for (int i = threadIdx.x; i < 2 * sp.s; i += kThreads) bins[i] = 0;
        __syncthreads();
        if (mx > 0.0) {
            const int shift = frac - bound_exponent(mx);
            for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) {
                const long long v = fixed_point(X[r + c * ldx], shift);
                if (v == 0) continue;
                const int l0 = (int)(v & lmask), l1 = (int)(v >> L);
                for (int q = 0; q < sp.zeta; ++q) {
                    int row;
                    bool neg;
                    pattern_entry(sp, pattern[r * sp.zeta + q], q, row, neg);
                    red_limbs(acc0, acc1, row, l0, l1, neg);
                }
            }
        }
        __syncthreads();
        long long *o = out + ((size_t)c * G + blockIdx.x) * sp.s;
        for (int i = threadIdx.x; i < sp.s; i += kThreads) o[i] = combine_limbs(acc0[i], acc1[i], L);
        __syncthreads();
    }
}

// SX[i, c] = 2^(E_c - frac) zeta^-1/2 sum_g partial[c][g][i].
__global__ void k_sparse_sign_reduce(const long long *__restrict__ part, const double *__restrict__ maxpart, int G,
                                     int s, int ncols, int zeta, const int *__restrict__ binmax,
                                     double *__restrict__ SX) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)s * ncols) return;
    const int c = (int)(idx / s), i = (int)(idx % s);
    const int frac = sketch_fraction_bits_from_limb(limb_bits(*binmax));
    double mx = 0.0;
    for (int g = 0; g < G; ++g) mx = fmax(mx, maxpart[(size_t)c * G + g]);
    if (mx == 0.0) {
        SX[idx] = 0.0;
        return;
    }
    const double tot = sum_i64_exact(part + (size_t)c * G * s + i, G, (size_t)s);
    SX[idx] = scale_pow2(tot, bound_exponent(mx) - frac) / sqrt((double)zeta);
}

__global__ void k_copy_cols(const double *__restrict__ X, int64_t ldx, int64_t n, int ncols, double *__restrict__ Y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * ncols) return;
    const int64_t c = idx / n, r = idx % n;
    Y[idx] = X[r + c * ldx];
}

}  // namespace

// Expand the sparse-sign pattern and its bin-load maximum (once per sketch).
skf_status build_sparse_sign_tables(skf_sketch *S, cudaStream_t st) {
    const SparseSign sp = make_sparse_sign(S);
    const size_t bytes = sizeof(uint16_t) * (size_t)S->n * S->zeta;
    cudaError_t e = cudaMalloc(&S->pattern, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        S->pattern = nullptr;
        return fail(SKF_ERR_OOM, "sketch pattern allocation");
    }
    e = cudaMalloc(&S->binmax, 3 * sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        S->binmax = nullptr;
        return fail(SKF_ERR_OOM, "sketch table allocation");
    }
    S->binmax_chunk = S->binmax + 1;
    S->binmax_persist = S->binmax + 2;
    int G;
    int64_t rows;
    row_partition(S->n, &G, &rows);
    const int blocks = (int)std::min<int64_t>((S->n + 255) / 256, 16ll * num_sms());
    k_build_pattern<<<blocks, 256, 0, st>>>(sp, S->n, S->pattern);
    cudaMemsetAsync(S->binmax, 0, 3 * sizeof(int), st);
    const size_t smem = sizeof(int) * S->s;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_bin_max, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bin_max<<<G, 256, smem, st>>>(sp, S->n, rows, S->pattern, S->binmax);
    int Gc;
    chunk_partition(S->n, &Gc);
    k_bin_max<<<Gc, 256, smem, st>>>(sp, S->n, kChunkRows, S->pattern, S->binmax_chunk);
    int Gp;
    int64_t rows_p;
    persist_partition(S->n, &Gp, &rows_p);
    k_bin_max<<<Gp, 256, smem, st>>>(sp, S->n, rows_p, S->pattern, S->binmax_persist);
    count_launches(4);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sketch table build");
    int hmax[3] = {0, 0, 0};
    cudaMemcpy(hmax, S->binmax, 3 * sizeof(int), cudaMemcpyDeviceToHost);
    if (limb_bits(hmax[0]) < 13 || limb_bits(hmax[1]) < 13)
        return fail(SKF_ERR_NOT_SUPPORTED, "sketch too dense for the fixed-point accumulators");
    // the persistent Arnoldi kernel is simply not used for a denser partition
    S->binmax_persist_host = hmax[2];
    if (limb_bits(hmax[2]) < 13) S->binmax_persist = nullptr;
    int max_stripe = 0;
    for (int q = 0; q < sp.zeta; ++q) max_stripe = std::max(max_stripe, sp.size[q]);
    if (max_stripe <= 128 && S->zeta <= 8) {
        if (cudaMalloc(&S->pattern8, (size_t)S->n * 8) == cudaSuccess) {
            S->p8_block = max_stripe <= 64 ? 64 : 128;
            k_build_pattern8<<<blocks, 256, 0, st>>>(sp, S->n, S->p8_block, S->pattern, S->pattern8);
            count_launches(1);
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "sketch table build");
        } else {
            cudaGetLastError();   // no compact table: the kernels read the 16-bit one
            S->pattern8 = nullptr;
        }
    }
    return SKF_OK;
}

skf_status sketch_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                            cudaStream_t st) {
    const int64_t n = S->n;
    if (ncols <= 0) return SKF_OK;
    if (S->kind == SKF_SKETCH_IDENTITY) {
        const int64_t tot = n * ncols;
        k_copy_cols<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, ldx, n, ncols, SX);
        count_launches(1);
        SKF_LAUNCH_CHECK("k_copy_cols");
        return SKF_OK;
    }
    if (S->kind == SKF_SKETCH_SRHT) return srht_apply_f64(S, X, ldx, ncols, SX, st);
    if (S->kind == SKF_SKETCH_SRDCT) return srdct_apply_f64(S, X, ldx, ncols, SX, st);
    if (S->kind != SKF_SKETCH_SPARSE_SIGN) return fail(SKF_ERR_NOT_SUPPORTED, "sketch kind not implemented");
    const SparseSign sp = make_sparse_sign(S);
    int G;
    int64_t rows;
    row_partition(n, &G, &rows);
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
    const size_t smem = sizeof(int) * 2 * S->s;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_sparse_sign_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_sparse_sign_scatter<<<G, kThreads, smem, st>>>(X, ldx, n, ncols, rows, sp, S->pattern, S->binmax, maxpart,
                                                      part);
    const int64_t tot = (int64_t)S->s * ncols;
    k_sparse_sign_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, maxpart, G, S->s, ncols, S->zeta,
                                                                        S->binmax, SX);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    dfree(part, st);
    dfree(maxpart, st);
    if (e != cudaSuccess) return cuda_fail(e, "sketch_apply kernels");
    return SKF_OK;
}

// ---------------------------------------------------------------------
// Allocation-free variant of sketch_apply_f64.
//
// Some callers cannot allocate device memory at the point where they need a
// sketch: code running inside a memory-budgeted runtime that owns every
// allocation, or code paths that must not touch the allocator or its memory
// pools at all (the allocating path goes through cudaMallocAsync and
// cudaFreeAsync on the library's pool; this one makes no allocator or pool
// call of any kind).  For them the scratch of the column-max / scatter /
// reduce pipeline (per-CTA column maxima and per-CTA integer partial sums)
// lives in the fixed array below instead of coming from cudaMallocAsync.
//
// kNoAllocScratchBytes bounds G * ncols * (s + 1) * 8 bytes, where G is the
// number of CTAs of the row partition (at most 2 per SM).  The array is a
// module global: every GPU that loads this library keeps it for the life of
// the process, and all calls on a device share it, so calls whose kernels
// may overlap on the GPU (different streams, or different host threads)
// race on it.  Every word a call reads is first written by the same call, so
// nothing has to be cleared between calls.
constexpr size_t kNoAllocScratchBytes = 4u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set-up once per
// device; cudaGetSymbolAddress is not valid inside a stream capture).
skf_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SKF_ERR_NOT_SUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SKF_OK;
}

}  // namespace

skf_status sketch_apply_f64_noalloc(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                                    cudaStream_t st) {
    if (S->kind != SKF_SKETCH_SPARSE_SIGN)
        return fail(SKF_ERR_NOT_SUPPORTED, "the allocation-free sketch apply supports the sparse-sign sketch only");
    if (ncols <= 0) return SKF_OK;
    const int64_t n = S->n;
    int G;
    int64_t rows;
    row_partition(n, &G, &rows);
    const size_t need = sizeof(long long) * (size_t)G * ncols * ((size_t)S->s + 1);
    if (need > kNoAllocScratchBytes)
        return fail(SKF_ERR_INVALID_ARG, "allocation-free sketch apply needs " + std::to_string(need) +
                                             " bytes of scratch, more than its fixed " +
                                             std::to_string(kNoAllocScratchBytes) +
                                             " (reduce ncols or s, or use skf_sketch_apply)");
    void *base = nullptr;
    skf_status stt = noalloc_scratch(&base);
    if (stt != SKF_OK) return stt;
    double *maxpart = (double *)base;                                         // [ncols][G]
    long long *part = (long long *)((char *)base + sizeof(double) * (size_t)G * ncols);   // [ncols][G][s]
    const SparseSign sp = make_sparse_sign(S);
    k_colmax<<<G, kThreads, 0, st>>>(X, ldx, n, ncols, rows, maxpart);
    const size_t smem = sizeof(int) * 2 * S->s;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_sparse_sign_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_sparse_sign_scatter<<<G, kThreads, smem, st>>>(X, ldx, n, ncols, rows, sp, S->pattern, S->binmax, maxpart,
                                                      part);
    const int64_t tot = (int64_t)S->s * ncols;
    k_sparse_sign_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, maxpart, G, S->s, ncols, S->zeta,
                                                                        S->binmax, SX);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "allocation-free sketch_apply kernels");
    return SKF_OK;
}

}  // namespace skf
