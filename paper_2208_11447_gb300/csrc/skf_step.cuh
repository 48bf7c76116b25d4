// Device helpers shared by the Arnoldi step kernels (FP64 and reduced-precision
// variants): exact and fixed-order cross-CTA reductions, the arrival ticket and
// the sparse-sign pattern load.
#pragma once

#include "skf_internal.cuh"

namespace skf {

constexpr int kNoExp = -100000;

// Exact sum of G int64 partials by one warp (lanes strided over G, 128-bit
// butterfly); every lane returns the same double.
__device__ __forceinline__ double warp_sum_i64_exact(const long long *p, int G, size_t stride) {
    const int lane = threadIdx.x & 31;
    unsigned long long lo = 0;
    long long hi = 0;
    for (int g = lane; g < G; g += 32) {
        const long long v = __ldcg(p + (size_t)g * stride);
        const unsigned long long nlo = lo + (unsigned long long)v;
        hi += (v < 0 ? -1 : 0) + (nlo < lo ? 1 : 0);
        lo = nlo;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, o);
        const long long ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const unsigned long long nlo = lo + olo;
        hi += ohi + (nlo < lo ? 1 : 0);
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

// Fixed-order reduction of G partials by one warp (sum or max).
__device__ __forceinline__ double warp_reduce_partials(const double *p, int G, int stride, bool is_max) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int g = lane; g < G; g += 32) {
        const double v = __ldcg(p + (size_t)g * stride);
        acc = is_max ? fmax(acc, v) : acc + v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = is_max ? fmax(acc, t) : acc + t;
    }
    return acc;
}

// The zeta pattern entries of column r (one 16-byte load for zeta = 8).
template <int ZCAP>
__device__ __forceinline__ void load_pattern(const uint16_t *pattern, int zeta, int64_t r, uint16_t (&e)[ZCAP]) {
    if (ZCAP == 8 && zeta == 8) {
        const uint4 v = __ldg((const uint4 *)(pattern + r * 8));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 8; ++q) e[q] = (uint16_t)(w[q >> 1] >> (16 * (q & 1)));
    } else {
#pragma unroll
        for (int q = 0; q < ZCAP; ++q) e[q] = q < zeta ? __ldg(pattern + r * zeta + q) : (uint16_t)0;
    }
}

// Arrival ticket: true in exactly one CTA, the last to finish its partials.
__device__ __forceinline__ bool last_to_arrive(unsigned *cnt) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Offset of basis column j in V: column-major with leading dimension ldv,
// or, when the basis is kept as a ring of vring slots (two-pass mode, only
// the columns the recurrence still reads are alive), slot j mod vring.
template <class Ctx>
__host__ __device__ __forceinline__ size_t vcol(const Ctx &c, int j) {
    return (size_t)(c.vring ? j % c.vring : j) * (size_t)c.ldv;
}

// Host: the window columns i0 .. j of step j (i0 = max(0, j - k + 1)) as
// element offsets into V, in the launch's copy of the context.
template <class Ctx>
inline void window_offsets(Ctx &c, int j) {
    const int i0 = j - c.k + 1 > 0 ? j - c.k + 1 : 0;
    for (int a = 0; a < kMaxK; ++a) {
        const int col = i0 + a <= j ? i0 + a : j;
        c.woff[a] = (int64_t)(c.vring ? col % c.vring : col) * c.ldv;
    }
}

}  // namespace skf
