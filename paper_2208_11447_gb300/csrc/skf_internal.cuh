// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/skf.h"

namespace skf {

constexpr int kThreads = 256;    // threads per CTA of the streaming kernels
constexpr int kMaxK = 16;        // largest supported truncation length k
constexpr int kMaxZeta = 16;     // largest supported sketch sparsity zeta

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
skf_status fail(skf_status st, const std::string &msg);
skf_status cuda_fail(cudaError_t e, const char *what);

#define SKF_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::skf::cuda_fail(e_, #call);       \
    } while (0)

#define SKF_LAUNCH_CHECK(what)                                           \
    do {                                                                 \
        cudaError_t e_ = cudaGetLastError();                             \
        if (e_ != cudaSuccess) return ::skf::cuda_fail(e_, what);        \
    } while (0)

int num_sms();

// ------------------------------------------------------------- handles
}  // namespace skf

struct skf_csr {
    int64_t n = 0, nnz = 0;
    int32_t *rowptr = nullptr;        // device int32[n+1] (owned)
    const int32_t *colind = nullptr;  // device
    const void *values = nullptr;     // device
    skf_dtype vdtype = SKF_F64;
    int32_t *colind_own = nullptr;
    void *values_own = nullptr;
    double norm_inf = 0.0;            // max_i sum_j |a_ij|
};

struct skf_sketch {
    skf_sketch_kind kind = SKF_SKETCH_SPARSE_SIGN;
    int64_t n = 0;
    int32_t s = 0, zeta = 0;
    uint64_t seed = 0;
    int64_t np = 0;                   // SRHT: padded length N'
    int32_t *P = nullptr;             // SRHT: s sampled rows (device)
};

namespace skf {

// ------------------------------------------------------------ device code
// SplitMix64 output function (Steele, Lea & Flood 2014) and its
// counter-based use: word(seed, i) = mix64(seed + (i + 1) * gamma).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}
__host__ __device__ __forceinline__ uint64_t splitmix_word(uint64_t seed, uint64_t i) {
    return mix64(seed + (i + 1ull) * 0x9E3779B97F4A7C15ull);
}

// Description of the sparse-sign pattern: stripe q covers rows
// [start[q], start[q] + size[q]).
struct SparseSign {
    int s, zeta, words;               // words = ceil(zeta / 4)
    uint64_t seed;
    int start[kMaxZeta];
    int size[kMaxZeta];
};
SparseSign make_sparse_sign(const skf_sketch *S);

// Row (within [0, s)) and sign of the q-th nonzero of column c.
__device__ __forceinline__ void sparse_sign_entry(const SparseSign &sp, uint64_t word, int q,
                                                  int &row, bool &neg) {
    const uint32_t u = (uint32_t)(word >> (16 * (q & 3))) & 0xFFFFu;
    neg = (u & 1u) != 0u;
    row = sp.start[q] + (int)(((u >> 1) * (uint32_t)sp.size[q]) >> 15);
}

// Exponent E with |x| < 2^E for all |x| <= xmax (xmax > 0, finite).
__host__ __device__ __forceinline__ int bound_exponent(double xmax) {
    int e;
    (void)frexp(xmax, &e);   // xmax = f 2^e, 0.5 <= f < 1  =>  xmax < 2^e
    return e;
}

// Round x * 2^shift to the nearest integer, using only integer operations
// (keeps the FP64 pipe free).  Requires |x| 2^shift < 2^62.
__device__ __forceinline__ long long fixed_point(double x, int shift) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return 0;   // zero or subnormal: far below any quantum used here
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = e - 1075 + shift;  // x 2^shift = mant 2^sh
    unsigned long long v;
    if (sh >= 0) {
        v = mant << sh;
    } else if (sh > -64) {
        const int r = -sh;
        v = (mant >> r) + ((mant >> (r - 1)) & 1ull);   // round half up on the magnitude
    } else {
        v = 0;
    }
    return (bits >> 63) ? -(long long)v : (long long)v;
}

__device__ __forceinline__ long long fixed_point(float x, int shift) {
    return fixed_point((double)x, shift);
}

// Exact 64-bit two's-complement accumulation into a (lo, hi) pair of 32-bit
// shared-memory words with native 32-bit atomics: the carry out of the low
// word is recovered from the value the atomic returns.
__device__ __forceinline__ void atomic_add_i64_split(uint32_t *lo, uint32_t *hi, long long v) {
    const uint32_t vlo = (uint32_t)(unsigned long long)v;
    const uint32_t vhi = (uint32_t)((unsigned long long)v >> 32);
    const uint32_t old = atomicAdd(lo, vlo);
    const uint32_t carry = (old + vlo < old) ? 1u : 0u;
    const uint32_t add = vhi + carry;
    if (add) atomicAdd(hi, add);
}

// Sum of G int64 values as an exact 128-bit integer, returned as double
// (two roundings at most): the two's-complement total is turned into sign
// and magnitude before conversion so that no cancellation occurs.
__device__ __forceinline__ double sum_i64_exact(const long long *p, int G, size_t stride) {
    unsigned long long lo = 0;
    long long hi = 0;
    for (int g = 0; g < G; ++g) {
        const long long v = p[(size_t)g * stride];
        const unsigned long long nlo = lo + (unsigned long long)v;
        hi += (v < 0 ? -1 : 0) + (nlo < lo ? 1 : 0);
        lo = nlo;
    }
    const bool neg = hi < 0;
    unsigned long long uhi = (unsigned long long)hi;
    if (neg) {
        lo = ~lo + 1ull;
        uhi = ~uhi + (lo == 0ull ? 1ull : 0ull);
    }
    const double r = (double)uhi * 18446744073709551616.0 + (double)lo;
    return neg ? -r : r;
}

// Block-wide reductions (blockDim.x == kThreads); the result is returned to
// every thread of the block.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *smem /* >= NV*32 */) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) smem[i * 32 + warp] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = lane < (kThreads / 32) ? smem[i * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) smem[i * 32] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = smem[i * 32];
    __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double *smem /* >= 32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < (kThreads / 32) ? smem[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) smem[0] = t;
    }
    __syncthreads();
    v = smem[0];
    __syncthreads();
    return v;
}

// Precision (fraction bits below the vector max) of the fixed-point sketch
// accumulators, given the most rows one CTA contributes to a bin.
__host__ __device__ __forceinline__ int sketch_fraction_bits(long long rows_per_cta) {
    int lg = 0;
    while ((1ll << lg) < rows_per_cta + 1) ++lg;
    int p = 62 - lg;
    return p > 52 ? 52 : p;
}

// ------------------------------------------------------ host-side helpers
// Quadrature rule of order ell for f (host); returns false if unsupported.
bool quadrature_rule(const skf_func &f, int ell, double *t, double *w);

// Stream-ordered scratch allocation (capture-safe).
skf_status dalloc(void **p, size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);

// Quadrature levels of the adaptive schedule on the device.
struct RuleDev {
    double *t = nullptr, *w = nullptr;               // all nodes, level after level
    int *lev_start = nullptr, *lev_ell = nullptr;    // device [nlevels+1], [nlevels]
    std::vector<int> h_start, h_ell;                 // host copies
    int nlevels = 0;
};

skf_status arnoldi_run(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, double *V, int64_t ldv,
                       double *vscale, double *SV, double *SAV, double *H, int *iscal, skf_info *info,
                       cudaStream_t st);
skf_status tail_run(skf_method method, int s, int m, int64_t n, const double *V, int64_t ldv, const double *vscale,
                    const double *SV, const double *SAV, int *iscal, const RuleDev &rule, double tol, double *x,
                    skf_info *info, cudaStream_t st);

// Sketch-apply launcher shared by the API and the solvers.
skf_status sketch_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                            cudaStream_t st);

}  // namespace skf
