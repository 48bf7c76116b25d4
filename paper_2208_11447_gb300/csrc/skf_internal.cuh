// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

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

// Number of kernel launches issued by the library (diagnostics).
void count_launches(long long n);

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
    // SELL-32 copy used by the kernels: rows in slices of 32, slice t holds
    // width[t] x 32 entries column-major (entry p of row 32t + l at
    // off[t] + 32 p + l), rows padded with value 0 and their own column.
    // Each row keeps the CSR order of its entries.
    // Values keep the handle's dtype (vdtype: F64 or F32).
    int64_t nslices = 0;
    int64_t *sell_off = nullptr;      // [nslices + 1]
    int32_t *sell_w = nullptr;        // [nslices]
    void *sell_val = nullptr;
    int32_t *sell_col = nullptr;
    int max_width = 0;                // widest slice
    int64_t max_chunk_entries = 0;    // most SELL entries in one chunk of 1024 rows (32 slices)
    // Row split for skewed degree distributions: rows with more than
    // kLongRow entries are left out of the slices (they count as empty there)
    // and cut into segments of at most kSegLen consecutive CSR entries; each
    // segment is reduced by one warp (k_spmv_long) into a partial sum, and the
    // SpMV adds a long row's partials in segment order.  sell_long[t] = (bit
    // mask of the long rows of slice t, index of its first long row); the
    // segments of long row q are long_seg0[q] .. long_seg0[q+1] - 1.
    int64_t nlong = 0, nseg = 0;
    int long_cut = 0;                 // rows longer than this take the row split (kLongRow unless tuned)
    // Sorted slices (irregular row lengths): within aligned windows of
    // kSortWin rows the rows are taken in order of decreasing length, so that
    // a slice holds rows of similar length and pads little; slot i of the
    // slice layout holds row perm[i] (nullptr: slot i holds row i).  Built by
    // skf_csr_set_layout / skf_csr_autotune, not by default.
    int32_t *perm = nullptr;          // [n] or nullptr
    uint2 *sell_long = nullptr;       // [nslices], nullptr without long rows
    int32_t *long_seg0 = nullptr;     // [nlong + 1]
    int32_t *seg_beg = nullptr;       // [nseg] first CSR entry of the segment
    int32_t *seg_end = nullptr;       // [nseg] one past its last entry
};
constexpr int kLongRow = 32;          // longest row kept in the SELL slices
constexpr int kSegLen = 1024;         // entries per segment of a long row (32 per lane)
constexpr int kSortWin = 256;         // rows per sorting window of the sorted slice layout

// The row split of an operator as the step kernels see it (see skf_csr).
struct RowSplit {
    const int32_t *perm = nullptr;        // slot -> row of the sorted slice layout, or nullptr
    const uint2 *sell_long = nullptr;     // nullptr: no long rows
    const int32_t *long_seg0 = nullptr;
    const int32_t *seg_beg = nullptr, *seg_end = nullptr;
    const int32_t *colind = nullptr;      // the operator's CSR
    const void *values = nullptr;
    int64_t nseg = 0;
};

inline RowSplit row_split_of(const skf_csr *A) {
    RowSplit r;
    r.perm = A->perm;
    if (A->nlong > 0) {
        r.sell_long = A->sell_long;
        r.long_seg0 = A->long_seg0;
        r.seg_beg = A->seg_beg;
        r.seg_end = A->seg_end;
        r.colind = A->colind;
        r.values = A->values;
        r.nseg = A->nseg;
    }
    return r;
}

// y of a long row: its segment partials added to y (0 from the empty slice
// row) in segment order.  sl = sell_long of the lane's slice.
template <typename TA>
__device__ __forceinline__ TA add_long_row(const RowSplit &rs, const TA *__restrict__ part, uint2 sl, int lane, TA y) {
    if ((sl.x >> lane) & 1u) {
        const int q = (int)sl.y + __popc(sl.x & ((1u << lane) - 1u));
        const int g1 = rs.long_seg0[q + 1];
        for (int g = rs.long_seg0[q]; g < g1; ++g) y += part[g];
    }
    return y;
}

// CTAs of k_spmv_long: eight segments (warps) per CTA, at most 8 CTAs per SM.
inline unsigned long_ctas(int64_t nseg, int sms) {
    const int64_t c = (nseg + 7) / 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(c, 8ll * sms));
}

struct skf_sketch {
    skf_sketch_kind kind = SKF_SKETCH_SPARSE_SIGN;
    int64_t n = 0;
    int32_t s = 0, zeta = 0;
    uint64_t seed = 0;
    int64_t np = 0;                   // SRHT: padded length N' (SRDCT: N)
    int32_t *P = nullptr;             // SRHT, SRDCT: s sampled rows (device)
    double *E = nullptr;              // SRDCT: the N signs (device)
    double *costab = nullptr;         // SRDCT, direct form: cos(pi j / (2N)), j = 0 .. 4N-1 (device)
    // SRDCT through an FFT (N with no prime factor above 7): the FFT length
    // (N / 2 for even N, the real input packed two to a complex entry; N for
    // odd N; 0: the direct form), the radices of its Stockham passes,
    // e^{-2 pi i t / N} for t < N, and per sampled row k the DCT twist
    // e^{-i pi k / (2N)} times the row's scale (device)
    int64_t fft_len = 0;
    int nrad = 0;
    int rad[64] = {};
    double2 *tw = nullptr;
    double2 *twist = nullptr;
    // Sparse-sign pattern, expanded once from the seed: entry [c * zeta + q]
    // holds the row of nonzero q of column c inside stripe q (bits 0-14) and
    // its sign (bit 15).  2 zeta bytes per column.
    uint16_t *pattern = nullptr;
    int *binmax = nullptr;            // device: most nonzeros one CTA row range puts in one row of S
    int *binmax_chunk = nullptr;      // device: the same for the chunk-interleaved partition
    int *binmax_persist = nullptr;    // device: the same for the persistent partition (persist_partition)
    int binmax_persist_host = 0;      // host copy of *binmax_persist
    // Compact pattern when every stripe has at most 128 rows and zeta <= 8:
    // byte [c * 8 + q] = (row of nonzero q within stripe q) + p8_block * sign,
    // with p8_block = 64 if every stripe has at most 64 rows, else 128; zero
    // bytes beyond zeta; nullptr otherwise.
    uint8_t *pattern8 = nullptr;
    int p8_block = 0;
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

// |x| as an ordered integer: for finite x, larger magnitudes give larger keys,
// so max |x| can be taken with integer instructions.
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ double key_to_abs(unsigned long long k) { return __longlong_as_double((long long)k); }

// Exponent E with |x| < 2^E for all |x| <= xmax (xmax > 0, finite): the
// exponent e of xmax = f 2^e, 0.5 <= f < 1, read from the bit pattern with
// integer instructions (the FP64 pipe retires one warp instruction per 16 SM
// cycles on this part, so per-thread scalar FP64 work is not free).  Normal
// xmax: biased exponent - 1022; subnormal xmax = mant 2^-1074: e = hb - 1073
// with hb the highest set bit of mant.
__host__ __device__ __forceinline__ int bound_exponent(double xmax) {
#ifdef __CUDA_ARCH__
    const unsigned long long bits = (unsigned long long)__double_as_longlong(xmax);
#else
    unsigned long long bits;
    memcpy(&bits, &xmax, sizeof bits);
#endif
    const int be = (int)((bits >> 52) & 0x7FFull);
    if (be != 0) return be - 1022;
    const unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
#ifdef __CUDA_ARCH__
    const int hb = 63 - __clzll((long long)mant);
#else
    const int hb = 63 - __builtin_clzll(mant);
#endif
    return hb - 1073;
}

// x 2^k, equal to ldexp(x, k): one multiplication by the exact power of two
// when 2^k is a normal double (a product with a power of two is rounded once,
// as ldexp rounds), ldexp otherwise.
__host__ __device__ __forceinline__ double scale_pow2(double x, int k) {
    if (k >= -1022 && k <= 1023) {
        const unsigned long long b = (unsigned long long)(k + 1023) << 52;
#ifdef __CUDA_ARCH__
        return x * __longlong_as_double((long long)b);
#else
        double p;
        memcpy(&p, &b, sizeof p);
        return x * p;
#endif
    }
    return ldexp(x, k);
}

// 0 < xmax < inf (false for zero, negative, infinite and NaN xmax), with
// integer instructions.
__host__ __device__ __forceinline__ bool positive_finite(double xmax) {
#ifdef __CUDA_ARCH__
    const long long b = __double_as_longlong(xmax);
#else
    long long b;
    memcpy(&b, &xmax, sizeof b);
#endif
    return b > 0 && b < 0x7FF0000000000000ll;
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

// Block-wide reductions for blocks of NT threads; the result is returned to
// every thread of the block.
template <int NV, int NT = kThreads>
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
            double t = lane < (NT / 32) ? smem[i * 32 + lane] : 0.0;
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

template <int NT = kThreads>
__device__ __forceinline__ double block_max(double v, double *smem /* >= 32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < (NT / 32) ? smem[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) smem[0] = t;
    }
    __syncthreads();
    v = smem[0];
    __syncthreads();
    return v;
}

// Block sum with few FP64 instructions (the FP64 pipe retires one warp
// instruction per 16 SM cycles on this part, whatever the active lanes):
// each thread parks its NV partials in shared memory and warp i alone adds
// up value i (sequential per lane, then one butterfly).  Result in every
// thread.  smem: NV * NT doubles.
template <int NV, int NT>
__device__ __forceinline__ void block_sum_lowflop(double (&v)[NV], double *smem) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) smem[i * NT + threadIdx.x] = v[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < NV; i += NT / 32) {
        double t = 0.0;
#pragma unroll 4
        for (int k = lane; k < NT; k += 32) t += smem[i * NT + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        __syncwarp();
        if (lane == 0) smem[i * NT] = t;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = smem[i * NT];
    __syncthreads();
}

// Shared-memory doubles a block reduction of NV values over NT threads needs,
// and the variant used: the low-FP64 one when its buffer stays within 32 KB.
template <int NV, int NT> struct BlockSumTraits {
    static constexpr bool kLow = (size_t)NV * NT * sizeof(double) <= 32768;
    static constexpr int kSmem = kLow ? NV * NT : 32 * NV;
};
template <int NV, int NT>
__device__ __forceinline__ void block_sum_auto(double (&v)[NV], double *smem) {
    if constexpr (BlockSumTraits<NV, NT>::kLow) block_sum_lowflop<NV, NT>(v, smem);
    else block_sum<NV, NT>(v, smem);
}

// Block max of non-negative magnitude keys (integer instructions only).
template <int NT>
__device__ __forceinline__ unsigned long long block_max_key(unsigned long long k, unsigned long long *smem) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
    __syncthreads();
    if (lane == 0) smem[warp] = k;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = lane < NT / 32 ? smem[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) smem[0] = t;
    }
    __syncthreads();
    k = smem[0];
    __syncthreads();
    return k;
}

// Row partition shared by the streaming kernels and the sketch tables: G
// CTAs, each owning `rows` consecutive rows.
void row_partition(int64_t n, int *G, int64_t *rows);

// Chunk-interleaved row partition of the reduced-precision SpMV kernel: rows
// in chunks of kChunkRows, chunk c handled by CTA c mod G, G = min(SMs,
// number of chunks).  All CTAs sweep the rows together, so the column
// gathers of banded operators stay within a few MB of L2.
constexpr int kChunkRows = 1024;
void chunk_partition(int64_t n, int *G);

// Row partition of the persistent FP64 Arnoldi kernel: G <= SMs CTAs of
// `rows` consecutive rows each (whole SELL slices), every CTA non-empty.
void persist_partition(int64_t n, int *G, int64_t *rows);

// Fixed-point sketch accumulation.  A value x is rounded to the integer
// v = x 2^(P - E) (E: exponent bound of the vector, |v| < 2^P) and split into
// two signed 32-bit limbs v = l1 2^L + l0, 0 <= l0 < 2^L, |l1| < 2^(P-L);
// each limb is added with a native 32-bit shared-memory atomic.  With at most
// `binmax` contributions per bin and CTA, L = 31 - ceil(log2(binmax + 1))
// rules out overflow, and P = min(2L, 52) bits of the vector max are kept.
__host__ __device__ __forceinline__ int limb_bits(int binmax) {
    int lg = 0;
    while ((1 << lg) < binmax + 1) ++lg;
    return 31 - lg;
}
__host__ __device__ __forceinline__ int sketch_fraction_bits_from_limb(int L) { return 2 * L > 52 ? 52 : 2 * L; }

__device__ __forceinline__ void pattern_entry(const SparseSign &sp, uint16_t e, int q, int &row, bool &neg) {
    row = sp.start[q] + (int)(e & 0x7FFFu);
    neg = (e >> 15) != 0;
}

__device__ __forceinline__ void red_limbs(int *acc0, int *acc1, int row, int l0, int l1, bool neg) {
    atomicAdd(acc0 + row, neg ? -l0 : l0);
    atomicAdd(acc1 + row, neg ? -l1 : l1);
}

// int64 partial of one bin from its two limbs.
__device__ __forceinline__ long long combine_limbs(int a0, int a1, int L) {
    return ((long long)a1 << L) + (long long)a0;
}

// ------------------------------------------------------ host-side helpers
// Quadrature rule of order ell for f (host); returns false if unsupported.
bool quadrature_rule(const skf_func &f, int ell, double *t, double *w);

// Stream-ordered scratch allocation (capture-safe).
skf_status dalloc(void **p, size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);

// Quadrature levels of the adaptive schedule on the device.
struct RuleDev {
    double *t = nullptr, *w = nullptr;               // all nodes, level after level (real parts)
    double *t_im = nullptr, *w_im = nullptr;         // imaginary parts (contour rules), else nullptr
    bool cplx = false;
    int *lev_start = nullptr, *lev_ell = nullptr;    // device [nlevels+1], [nlevels]
    std::vector<int> h_start, h_ell;                 // host copies
    int nlevels = 0;
};

// Called by the Arnoldi host drivers while they enqueue the steps: once the
// work enqueued so far has run, columns 0 .. done-1 of S V and S A V are final
// (done = m after the last step).  The stopping criterion enqueues its
// checkpoints from here.  iscal[0] = 2 marks a stop by the criterion (the
// recurrence ends at m_eff = iscal[1] with those columns already final).
// col_fn(ctx, j, st) is called once column j of V (w_j) is written: j = 0
// after the start kernel, j + 1 after the update of step j (the two-pass
// mode accumulates f there before the ring slot is reused).
struct StepHook {
    void (*fn)(void *ctx, int done, cudaStream_t st) = nullptr;
    void *ctx = nullptr;
    void (*col_fn)(void *ctx, int j, cudaStream_t st) = nullptr;
    void *col_ctx = nullptr;
};
inline void call_hook(const StepHook *h, int done, cudaStream_t st) {
    if (h && h->fn) h->fn(h->ctx, done, st);
}
inline void call_col_hook(const StepHook *h, int j, cudaStream_t st) {
    if (h && h->col_fn) h->col_fn(h->col_ctx, j, st);
}

// Persistent single-launch FP64 Arnoldi process (skf_arnoldi_persist.cu):
// SKF_ERR_NOT_SUPPORTED, with nothing left enqueued, when the case does not
// fit it (sketch kind, k > 4, shared memory, cooperative launch).
skf_status arnoldi_run_persistent(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, double *V,
                                  int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                                  skf_info *info, cudaStream_t st);
// the persistent form with an FP32 basis (FP32 values, k <= 2, slices at most 7 wide)
skf_status arnoldi_run_persistent_f32(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, float *V,
                                      int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                                      skf_info *info, cudaStream_t st);
// Which FP64 step form arnoldi_run uses: 0 automatic (persistent where it
// fits), 1 the two-kernel form only, 2 the persistent form or
// SKF_ERR_NOT_SUPPORTED.
void set_step_mode(int mode);
int step_mode();
// Form of the whitening QR in the tail: 0 one cooperative launch where it
// fits, 1 one launch per Householder reflector.
void set_qr_mode(int mode);
int qr_mode();
// what the tail factors (skf_set_tail_form)
void set_tail_form(int form);
int tail_form();
// Bounded-wait self-test: `ctas` co-resident CTAs wait at a barrier that
// cannot complete; *status_out (device) becomes SKF_ERR_TIMEOUT.
skf_status barrier_selftest(int ctas, long long budget, int *status_out, cudaStream_t st);

skf_status arnoldi_run(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, double *V, int64_t ldv,
                       double *vscale, double *SV, double *SAV, double *H, int *iscal, skf_info *info,
                       cudaStream_t st, const StepHook *hook = nullptr, int vring = 0);
// Reduced-precision variants: FP32 matrix values, basis stored in FP32 or
// BF16 (V of that type), FP32 SpMV and orthogonalisation, FP64 sketches.
skf_status arnoldi_run_f32(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, float *V,
                           int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                           skf_info *info, cudaStream_t st, const StepHook *hook = nullptr, int vring = 0);
// nr FP32-basis Arnoldi processes on one operator and one sketch in lockstep
// (one SpMM per step for each group of right-hand sides; skf_arnoldi_lp.cuh)
skf_status arnoldi_run_f32_block(const skf_csr *A, const skf_sketch *S, int nr, const double *const *b, int m, int k,
                                 float *const *V, int64_t ldv, double *const *vscale, double *const *SV,
                                 double *const *SAV, double *const *H, int *const *iscal, skf_info *const *info,
                                 cudaStream_t st);
skf_status arnoldi_run_bf16(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, void *V,
                            int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                            skf_info *info, cudaStream_t st, const StepHook *hook = nullptr, int vring = 0);
// V has type vdt (F64, F32 or BF16).  With sketch_out != nullptr the tail
// writes S f = S V y (s doubles) there instead of recombining x = V y (x
// unused); with x == nullptr and no sketch_out it only forms the
// coefficients.  z_out (nullable, m doubles): the coefficients z_j of the
// stored columns (x = sum_j z_j w_j), zero for j >= m_eff.  stop_state (nullable): [1] last estimate, [2] stop step of the
// stopping criterion, copied into info.  H (nullable; ld ldh, truncation kt):
// the Arnoldi coefficients; with H and an FP64 basis the tail uses the
// relation form (QR of [S V_m, S A v_m], S A v_j = S V_m H(:, j) for j < m).
skf_status tail_run(skf_method method, int s, int m, int64_t n, const void *V, skf_dtype vdt, int64_t ldv,
                    const double *vscale, const double *SV, const double *SAV, int *iscal, const RuleDev &rule,
                    double tol, double *x, skf_info *info, cudaStream_t st, double *sketch_out = nullptr,
                    const double *stop_state = nullptr, double *z_out = nullptr, double cond_max = 0.0,
                    const double *H = nullptr, int ldh = 0, int kt = 0);
// One method's outputs of a tail: the recombined f (nullable), the result
// record (nullable), the coefficients (nullable) and its status words
// (iscal[1] = m_eff is read, iscal[2] written).
struct TailOut {
    skf_method method;
    double *x;
    skf_info *info;
    double *z_out;
    int *iscal;
};
// The tails of one or two methods on the same Arnoldi output: the whitening
// QR, M, cond(R) and gamma once (for the most demanding method), then each
// method's node solves, level sums and coefficients; with two FP64 outputs
// both recombinations share one pass over V.  The iscal of outs[1] must hold
// a copy of outs[0]'s (same m_eff).
skf_status tail_run_multi(int nout, const TailOut *outs, int s, int m, int64_t n, const void *V, skf_dtype vdt,
                          int64_t ldv, const double *vscale, const double *SV, const double *SAV, const RuleDev &rule,
                          double tol, cudaStream_t st, double *sketch_out, const double *stop_state, double cond_max,
                          const double *H, int ldh, int kt);
// Two-pass mode: x (+)= z_j w_j for basis column w_j (type vdt), j < m_eff =
// iscal[1]; j = 0 starts x (x = 0 when m_eff = 0).  The FMA sequence per row
// is that of the one-pass FP64 recombination.
skf_status accumulate_column(const void *w, skf_dtype vdt, const double *z, const int *iscal, int j, int64_t n,
                             double *x, cudaStream_t st);
// One checkpoint of the stopping criterion at prefix p (see skf_params):
// the tail of the leading p columns in sketched form, then the comparison
// with the previous checkpoint; on success sets iscal to stop at m_eff = p.
// Work buffers: iscal_chk[4], sf_prev[s], sf_cur[s], state[4] ([0] previous
// checkpoint valid, [1] last estimate, [2] stop step), zeroed by the caller.
skf_status stop_check(skf_method method, int s, int p, const double *vscale, const double *SV, const double *SAV,
                      int *iscal, int *iscal_chk, double *sf_prev, double *sf_cur, double *state, const RuleDev &rule,
                      double tol_quad, double stop_tol, cudaStream_t st);

// SRHT sketch (see skf_srht.cu): blocks of 2^b entries transformed exactly in
// integers, b = min(kSrhtBlockLog2, log2 N').
constexpr int kSrhtBlockLog2 = 12;
struct SrhtDev {
    int64_t n, np;       // N, N' = 2^ceil(log2 N)
    int s, b, nblk;      // rows, block log2, N' / 2^b
    int frac;            // fraction bits of the fixed-point input, 62 - b
    uint64_t seed;
    const int32_t *P;    // [s] sampled rows
};
// Up to two columns per launch: x[c] (device, N entries), the exponent bound
// of its maximum (device int, kNoExp for a zero column) and its block
// partials part[c][nblk][s]; with iscal non-null the launch does nothing once
// the Arnoldi process has stopped at or before `step`.
struct SrhtCols {
    const void *x[2];    // F64 columns, or F32 with f32 = 1 (widened exactly)
    const int *e[2];
    long long *part[2];
    int ncols;
    const int *iscal;
    int step;
    int f32;
};
SrhtDev make_srht(const skf_sketch *S);
skf_status build_srht_tables(skf_sketch *S);
void srht_launch(const SrhtDev &d, const SrhtCols &cols, cudaStream_t st);
skf_status srht_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX, cudaStream_t st);

// SRDCT sketch (see skf_srdct.cu): the sampled rows of the orthonormal
// DCT-II, through a length-N FFT (O(N log N) per vector) when N has no prime
// factor above 7, else by direct O(sN) evaluation.
struct SrdctDev {
    int64_t n;
    int s;
    const int32_t *P;       // [s] sampled rows
    const double *E;        // [n] signs
    const double *costab;   // [4n] cos(pi j / (2n)) (direct form)
    int64_t fft_len;        // FFT form: n / 2 (even n) or n (odd n); 0: direct form
    int nrad;               // Stockham passes of the FFT
    int rad[64];
    const double2 *tw;      // [n] e^{-2 pi i t / n}
    const double2 *twist;   // [s] e^{-i pi k / (2n)} a_k sqrt(n / s), k = P[i]
    double2 *work;          // FFT form: [2][2][fft_len] scratch of the caller
};
// Up to two columns: out[q][i] = colscale * (S x[q])_i (colscale a device
// scalar or nullptr for 1); iscal/step as for SrhtCols.
struct SrdctCols {
    const void *x[2];    // F64 columns, or F32 with f32 = 1 (widened exactly)
    double *out[2];
    const double *colscale;
    int ncols;
    const int *iscal;
    int step;
    int f32;
};
// bytes of the FFT form's scratch (0 for the direct form)
size_t srdct_work_bytes(const skf_sketch *S);
SrdctDev make_srdct(const skf_sketch *S);
skf_status build_srdct_tables(skf_sketch *S);
void srdct_launch(const SrdctDev &d, const SrdctCols &cols, cudaStream_t st);
skf_status srdct_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX, cudaStream_t st);

// An SRHT or SRDCT applied to up to two F32 columns of a reduced-precision
// Arnoldi step (the stored w_j and y_j = A w_j): out[q] = colscale S x[q],
// computed in FP64 from the exactly widened values (SRHT: exact fixed point);
// nothing is done once the Arnoldi process stopped at or before `step`.
struct DenseCols {
    const float *x[2];
    double *out[2];
    const double *colscale;
    int ncols;
    const int *iscal;
    int step;
};
size_t dense_sketch_work_bytes(const skf_sketch *S);   // scratch of dense_sketch_f32
void dense_sketch_f32(const skf_sketch *S, const DenseCols &cols, void *work, cudaStream_t st);
// P: the first s entries of the partial Fisher-Yates shuffle of [0, np) (device).
skf_status build_sampled_rows(skf_sketch *S, int64_t np);

// Sketch-apply launcher shared by the API and the solvers.
skf_status build_sparse_sign_tables(skf_sketch *S, cudaStream_t st);
skf_status sketch_apply_f64_noalloc(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                                    cudaStream_t st);
skf_status sketch_apply_f64(const skf_sketch *S, const double *X, int64_t ldx, int ncols, double *SX,
                            cudaStream_t st);

}  // namespace skf
