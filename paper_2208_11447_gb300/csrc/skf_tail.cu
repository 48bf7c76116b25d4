// Small dense FP64 tail of sFOM / sGMRES (Sec. 2.1, Sec. 3, Sec. 4.1) and the
// recombination f = V_m y.
//
// One Householder QR of the s x 2m matrix [S V_m, S A V_m] gives everything:
// with S V_m = Q R and S A V_m = Q R12 + Q2 R22,
//   Z = S A V_m R^{-1} = Q M + Q2 R2,  M = R12 R^{-1},  R2 = R22 R^{-1},
// and c = Q^T S b = ||b|| R_11 e_1 (S b is ||b|| times the first column of
// S V_m).  Hence, for every quadrature node t,
//   sFOM:   (t I + M) y = c
//   sGMRES: min_y || [t I + M; R2] y - [c; 0] ||      (an m-column problem,
//           independent of s, equal to min ||(t Q + Z) y - S b||).
// Each node is solved from its normal equations by Cholesky with one step of
// FP64 iterative refinement on the original residual.
//
// With an FP64 or FP32 basis the tail factors only the s x (m+1) matrix
// [S V_m, S A v_m] instead (relation form): the Arnoldi relation
// A v_j = sum_i h_ij v_i (i <= j + 1, eq. (2.1)) sketched gives
// S A v_j = S V_m H(1:m, j) for j < m, so with [S V_m, S A v_m] = Q R,
//   Q^T S A V_m = [R_11 H(1:m, 1:m-1), R(1:m, m+1)],
// and the part of S A V_m orthogonal to S V_m is R(m+1, m+1) q_{m+1} e_m^T:
// M = [R_11 H(1:m, 1:m-1), R(1:m, m+1)] R_11^{-1} and R2 is the single row
// gamma e_m^T, gamma = R(m+1, m+1) / R(m, m) (the last row of R_11^{-1} is
// e_m^T / R(m, m)).  Same M and ||R2 y|| as the 2m-column QR (S A V_m enters
// only through the relation, which both Arnoldi forms satisfy to rounding),
// half the reflectors for sGMRES, and rank-one R2 terms in the node solves.
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

#include <cuda_bf16.h>

#include "skf_internal.cuh"

namespace skf {

struct TailCtx {
    int s, m;          // allocation sizes; m_eff = iscal[1] at run time
    int method;        // skf_method
    int *iscal;        // [0] stopped, [1] m_eff, [2] status
    const double *vscale;
    double *Aw;        // s x 2m, ld s
    double *Rdiag;     // [2m]
    double *M, *R2;    // m x m, ld m
    double *MT, *R2T;  // transposes, m x m, ld m
    double *B, *C;     // m x m, ld m (lower triangles used)
    double *cvec, *Mtc;  // [m]
    double *Nw;        // node workspace [batch][m*m]
    double *out;       // [batch][m] weighted node solutions
    int *nodebad;      // [batch] 1 = the mixed-precision solve did not converge
    double *qbuf;      // [levels][m]
    double *qacc;      // [m]
    double *z;         // [m] coefficients for V (scaled by vscale)
    double *qstate;    // [0] converged, [1] ell, [2] quad_err, [3] rdiag_ratio, [4] FP64 node solves, [5] cond(R) estimate,
                       // [6] gamma of the relation form (R2 = gamma e_m^T), [7] 1 if R_11 has a zero pivot
    const double *H;   // relation form: Arnoldi coefficients h_ij = H[i + j ldh]
    int ldh, kt;       // leading dimension of H, truncation length k
    int rel;           // 1: relation form (QR of [S V_m, S A v_m]), 0: QR of [S V_m, S A V_m]
    int hess;          // 1: real node solves by Givens reduction of the Hessenberg node matrix (relation form)
    double *RT, *RTs;  // R_11 row-major, and D^{-1} R_11 row-major (D = diag(R_11)), ld m, from k_r_pack
    double *Rcs;       // R_11 D^{-1} column-major, ld m
    double *rinv;      // [m] 1 / R_jj
    double *cn2;       // [m] squared column norms of R_11
    unsigned *lev_cnt; // CTAs of the current k_levels launch that have finished their level
    double cond_max;   // ILL_CONDITIONED above this cond(R) estimate (0: no test)
    double *hsig;      // [2m] ||x(jj+1:)||^2 of each pivot column, from the previous reflector launch
    const double *t, *w;      // node table
    const double *ti, *wi;    // imaginary parts of complex (contour) nodes and weights, or nullptr
    int nlevels;
};

namespace {

__global__ void k_tail_copy(const double *__restrict__ SV, const double *__restrict__ SAV, TailCtx c) {
    const int me = c.iscal[1];
    const int64_t tot = (int64_t)c.s * (c.rel ? c.m + 1 : 2 * c.m);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(idx / c.s);
        const int64_t r = idx % c.s;
        double v = 0.0;
        if (col < me) v = SV[r + (int64_t)col * c.s];
        else if (c.rel ? col == me : col < 2 * me) v = SAV[r + (int64_t)(c.rel ? me - 1 : col - me) * c.s];
        c.Aw[idx] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x < 8) c.qstate[threadIdx.x] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *c.lev_cnt = 0u;
}

// Householder reflector for column jj (LAPACK convention: beta = -sign(x0)
// ||x||, v = [1; x(jj+1:)/(x0 - beta)], tau = (beta - x0)/beta), applied to
// the trailing columns, one CTA of kHhThreads per trailing column, so a
// launch spreads over all SMs and each column's rows are read by four warps
// at once.  Every CTA forms the reflector from column jj, which no CTA
// modifies (its diagonal goes to Rdiag), so the launch has no intra-launch
// dependencies.  sig = ||x(jj+1:)||^2 comes from the previous launch: the
// CTA that updates column jj+1 sums its squares below the next diagonal right
// after its update (hsig[jj+1]); launch 0 sums it itself.
constexpr int kHhThreads = 128;

__device__ __forceinline__ double hh_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kHhThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kHhThreads) k_householder(TailCtx c, int jj) {
    __shared__ double red[kHhThreads / 32];
    // Launched as a programmatic dependent of the previous reflector: wait for
    // it to finish (every CTA, before any exit, so that no launch can finish
    // ahead of its predecessor), then let the next reflector's CTAs be placed
    // while this one runs.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int me = c.iscal[1];
    const int ncols = c.rel ? me + 1 : 2 * me;
    const int nref = (c.method == SKF_METHOD_SGMRES) ? ncols : me;
    if (jj >= nref || jj >= c.s) return;
    const int tid = threadIdx.x;
    const int gw = blockIdx.x;
    const int ntrail = ncols - jj - 1;
    if (gw >= ntrail && gw != 0) return;
    const double *x = c.Aw + (int64_t)jj * c.s;
    double sig;
    if (jj == 0) {
        double p = 0.0;
        for (int i = jj + 1 + tid; i < c.s; i += kHhThreads) p = fma(x[i], x[i], p);
        sig = hh_sum(p, red);
    } else {
        sig = c.hsig[jj];
    }
    const double x0 = x[jj];
    double tau = 0.0, beta = x0, scale = 0.0;
    if (sig > 0.0 || x0 == 0.0) {
        const double nx = sqrt(x0 * x0 + sig);
        beta = (x0 >= 0.0) ? -nx : nx;
        if (nx > 0.0) {
            tau = (beta - x0) / beta;
            scale = 1.0 / (x0 - beta);
        }
    }
    if (gw == 0 && tid == 0) c.Rdiag[jj] = beta;
    if (gw >= ntrail) return;
    double *y = c.Aw + (int64_t)(jj + 1 + gw) * c.s;
    if (tau != 0.0) {
        double p = (tid == 0) ? y[jj] : 0.0;
        for (int i = jj + 1 + tid; i < c.s; i += kHhThreads) p = fma(x[i] * scale, y[i], p);
        const double f = tau * hh_sum(p, red);
        if (tid == 0) y[jj] -= f;
        for (int i = jj + 1 + tid; i < c.s; i += kHhThreads) y[i] = fma(-f, x[i] * scale, y[i]);
    }
    if (gw == 0 && jj + 1 < nref) {
        // sig of the next pivot column, from the entries the CTA just wrote
        __syncthreads();
        double p = 0.0;
        for (int i = jj + 2 + tid; i < c.s; i += kHhThreads) p = fma(y[i], y[i], p);
        const double sn = hh_sum(p, red);
        if (tid == 0) c.hsig[jj + 1] = sn;
    }
}

// The whole Householder QR of [S V_m, S A V_m] in one cooperative launch.
// Column q belongs to CTA q mod G for the whole factorisation and stays in
// that CTA's shared memory until the end, so a CTA's trailing columns are
// only ever read and updated on chip.  The only data a step needs from
// another CTA is its pivot column: the owner of column jj + 1 updates that
// column first at step jj, writes it to global memory and publishes it (a
// release store of jj + 1 to a step counter); every other CTA starts step
// jj + 1 as soon as the counter reaches jj + 1 (bounded wait), so the updates
// of the remaining columns overlap the next steps instead of meeting at a
// grid barrier.  Each step is one pass over the pivot column per CTA:
// ||x(jj+1:)||^2 and the products x(jj+1:)^T y for the CTA's columns, summed
// in one block reduction; the reflector (LAPACK convention, as
// k_householder) is formed identically by every CTA.
constexpr int kQrThreads = 256;
constexpr int kQrOwn = 7;            // columns per CTA (at most)
constexpr long long kQrBudget = 1ll << 31;

__device__ __forceinline__ unsigned qr_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// sums over the CTA of nv <= kQrOwn + 1 per-thread values, in a fixed order,
// into tot[] (visible to every thread on return)
__device__ __forceinline__ void qr_block_sums(const double (&v)[kQrOwn + 1], int nv, double *sm, double *tot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < kQrOwn + 1; ++k)
        if (k < nv) sm[k * kQrThreads + tid] = v[k];
    __syncthreads();
    if (warp < nv) {
        double a = 0.0;
#pragma unroll
        for (int r = 0; r < kQrThreads / 32; ++r) a += sm[warp * kQrThreads + lane + 32 * r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) tot[warp] = a;
    }
    __syncthreads();
}

size_t qr_smem_bytes(int s) {
    return sizeof(double) * ((size_t)kQrOwn * s + s + (size_t)(kQrOwn + 1) * kQrThreads + kQrOwn + 1);
}

__global__ void __launch_bounds__(kQrThreads) k_qr_persist(TailCtx c, unsigned *ready, int *flag) {
    extern __shared__ double qsm[];
    __shared__ int ok;
    __shared__ double qsc[2];                     // tau, scale of the current reflector
    __shared__ double qf[kQrOwn], qfs[kQrOwn];    // f and f scale of the columns being updated
    const int me = c.iscal[1];
    const int ncols = c.rel ? me + 1 : 2 * me;
    const int s = c.s;
    const int nref = min((c.method == SKF_METHOD_SGMRES) ? ncols : me, s);
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31;
    const bool warp0 = tid < 32;
    double *cols = qsm;                                   // [kQrOwn][s]: columns g, g + G, ...
    double *xs = cols + (size_t)kQrOwn * s;               // [s] pivot column
    double *sm = xs + s;                                  // reduction scratch
    double *tot = sm + (kQrOwn + 1) * kQrThreads;
    int nq = 0;
    for (int q = g; q < ncols; q += G) ++nq;
    for (int k = 0; k < nq; ++k)
        for (int i = tid; i < s; i += kQrThreads) cols[(size_t)k * s + i] = c.Aw[i + (int64_t)(g + k * G) * s];
    __syncthreads();
    for (int jj = 0; jj < nref; ++jj) {
        // own columns that trail the pivot: k >= kf (column g + k G > jj)
        const int kf = jj < g ? 0 : (jj - g) / G + 1;
        const bool writer = (jj % G) == g;                 // owns the pivot column
        if (kf >= nq && !writer) continue;
        // pivot column jj, rows jj .. s-1
        if (writer) {
            const double *xc = cols + (size_t)((jj - g) / G) * s;
            for (int i = jj + tid; i < s; i += kQrThreads) xs[i] = xc[i];
        } else {
            if (tid == 0) {
                const long long t0 = clock64();
                int good = 1;
                while (qr_ld_acquire(ready) < (unsigned)jj) {
                    if (*(volatile int *)flag != 0 || clock64() - t0 > kQrBudget) {
                        good = 0;
                        break;
                    }
                }
                if (!good) atomicExch(flag, 1);
                ok = good;
            }
            __syncthreads();
            if (!ok) {
                if (tid == 0) atomicExch(&c.iscal[2], (int)SKF_ERR_TIMEOUT);
                return;
            }
            const double *x = c.Aw + (int64_t)jj * s;
            for (int i = jj + tid; i < s; i += kQrThreads) xs[i] = __ldcg(x + i);
        }
        __syncthreads();
        const double x0 = xs[jj];
        // the next pivot column (jj + 1) is this CTA's first trailing one:
        // update and publish it before the others
        const bool pivot_owner = kf < nq && g + kf * G == jj + 1;
        const int n1 = pivot_owner ? 1 : nq - kf;
        double loc[kQrOwn + 1];
#pragma unroll
        for (int k = 0; k < kQrOwn + 1; ++k) loc[k] = 0.0;
        for (int i = jj + 1 + tid; i < s; i += kQrThreads) {
            const double xi = xs[i];
            loc[0] = fma(xi, xi, loc[0]);
#pragma unroll
            for (int k = 0; k < kQrOwn; ++k)
                if (k < n1) loc[1 + k] = fma(xi, cols[(size_t)(kf + k) * s + i], loc[1 + k]);
        }
        qr_block_sums(loc, 1 + (kf < nq ? n1 : 0), sm, tot);
        // The reflector (from one rsqrt and one reciprocal: with
        // r = (x0^2 + sig)^-1/2, ||x|| = (x0^2 + sig) r, beta = -sign(x0) ||x||,
        // tau = (beta - x0) / beta = 1 + |x0| r, 1 / (x0 - beta) =
        // sign(x0) / (|x0| + ||x||)) and the factors f = tau (y(jj) + scale x^T y)
        // of the columns, by warp 0 only: a warp instruction occupies the FP64
        // pipe for 16 cycles whatever its active lanes, so scalar FP64 work
        // repeated by every warp costs eight times the pipe time.
        if (warp0) {
            const double sig = tot[0];
            double tau = 0.0, beta = x0, scale = 0.0;
            if (sig > 0.0 || x0 == 0.0) {
                const double q2 = fma(x0, x0, sig);
                if (q2 > 0.0) {
                    const double r = rsqrt(q2);
                    const double nx = q2 * r;
                    const double sgn = x0 >= 0.0 ? 1.0 : -1.0;
                    beta = -sgn * nx;
                    tau = fma(fabs(x0), r, 1.0);
                    scale = sgn / (fabs(x0) + nx);
                }
            }
            if (lane == 0) {
                qsc[0] = tau;
                qsc[1] = scale;
                if (writer) c.Rdiag[jj] = beta;
            }
            if (lane < n1 && kf < nq) {
                const double f = tau * (cols[(size_t)(kf + lane) * s + jj] + scale * tot[1 + lane]);
                qf[lane] = f;
                qfs[lane] = f * scale;
            }
        }
        __syncthreads();
        if (kf >= nq) continue;
        const double tau = qsc[0];
        // y(jj) -= f, y(i) -= f scale x_i
        if (tau != 0.0) {
#pragma unroll
            for (int k = 0; k < kQrOwn; ++k) {
                if (k < n1) {
                    double *y = cols + (size_t)(kf + k) * s;
                    const double fs = qfs[k];
                    for (int i = jj + 1 + tid; i < s; i += kQrThreads) y[i] = fma(-fs, xs[i], y[i]);
                    if (tid == 0) y[jj] -= qf[k];
                }
            }
        }
        if (pivot_owner) {
            // publish column jj + 1 (rows jj + 1 .. s - 1: what the next reflector reads)
            __syncthreads();
            double *yg = c.Aw + (int64_t)(jj + 1) * s;
            const double *y = cols + (size_t)kf * s;
            for (int i = jj + 1 + tid; i < s; i += kQrThreads) yg[i] = y[i];
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(ready), "r"((unsigned)(jj + 1)) : "memory");
            }
            const int n2 = nq - kf - 1;
            if (n2 > 0) {   // the rest of this CTA's trailing columns
#pragma unroll
                for (int k = 0; k < kQrOwn + 1; ++k) loc[k] = 0.0;
                for (int i = jj + 1 + tid; i < s; i += kQrThreads) {
                    const double xi = xs[i];
#pragma unroll
                    for (int k = 0; k < kQrOwn; ++k)
                        if (k < n2) loc[k] = fma(xi, cols[(size_t)(kf + 1 + k) * s + i], loc[k]);
                }
                qr_block_sums(loc, n2, sm, tot);
                if (warp0 && lane < n2) {
                    const double f = tau * (cols[(size_t)(kf + 1 + lane) * s + jj] + qsc[1] * tot[lane]);
                    qf[lane] = f;
                    qfs[lane] = f * qsc[1];
                }
                __syncthreads();
                if (tau != 0.0) {
#pragma unroll
                    for (int k = 0; k < kQrOwn; ++k) {
                        if (k < n2) {
                            double *y = cols + (size_t)(kf + 1 + k) * s;
                            const double fs = qfs[k];
                            for (int i = jj + 1 + tid; i < s; i += kQrThreads) y[i] = fma(-fs, xs[i], y[i]);
                            if (tid == 0) y[jj] -= qf[k];
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    // the factored columns back to global memory (R above the diagonal, the
    // reflectors below it are not used later)
    for (int k = 0; k < nq; ++k)
        for (int i = tid; i < s; i += kQrThreads) c.Aw[i + (int64_t)(g + k * G) * s] = cols[(size_t)k * s + i];
}

// ---------------------------------------------------------------------------
// Sequential triangular solves with the whitening factor R = R_11 by one
// warp: lane l holds entries l, l + 32, ... of the vector in K register
// groups (K = ceil(m / 32) rounded up to 2, 4, 8 or 16).  An FP64 warp
// instruction keeps its SM sub-partition's FP64 unit busy for many cycles on
// this part, so a step issues as few as possible: the factors come with
// unit diagonals (k_r_pack: RTs = D^{-1} R row-major, Rcs = R D^{-1}
// column-major, D = diag(R)), a step is one broadcast and one FMA per
// register group still in play (the group of the next pivot first), the
// outer loop over register groups is unrolled so that the pivot's register
// is known at compile time, and the row or column a step needs is loaded
// four steps ahead.

template <int K>
__device__ __forceinline__ double hsel(const double (&x)[K], int k) {
    double v = x[0];
#pragma unroll
    for (int q = 1; q < K; ++q) v = (q == k) ? x[q] : v;
    return v;
}

// x' RTs = t with x' = x D, i.e. x R = t (row vector; t in x on entry, x'
// on exit: the caller scales by 1 / R_jj): x'_j = t_j, then
// t_l -= x'_j RTs_jl for l > j.  EST: the forward solve of the LINPACK
// condition estimator, z'^T = (b - v)^T with b_j = +-1 chosen step by step
// against the sign of the accumulated v (x starts at 0).
template <int K, bool EST>
__device__ void warp_row_solve(const double *RTs, int me, int m, double (&x)[K]) {
    const int lane = threadIdx.x & 31;
    const int ka = (me + 31) >> 5;
    auto load = [&](double (&bv)[K], int j) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int l = lane + 32 * kk;
            bv[kk] = (j < me && kk < ka && l > j && l < me) ? RTs[(int64_t)j * m + l] : 0.0;
        }
    };
    double b0[K], b1[K], b2[K], b3[K];
    load(b0, 0);
    load(b1, 1);
    load(b2, 2);
    load(b3, 3);
#pragma unroll
    for (int k0 = 0; k0 < K; ++k0) {
        if (k0 >= ka) break;
        auto step = [&](const double (&bv)[K], int L) {
            const int j = 32 * k0 + L;
            double tj = __shfl_sync(0xffffffffu, x[k0], L);
            if (EST) tj += (tj < 0.0) ? -1.0 : 1.0;
            const int l0 = lane + 32 * k0;
            if (l0 == j) x[k0] = tj;
            else if (l0 > j) x[k0] = fma(-tj, bv[k0], x[k0]);
#pragma unroll
            for (int kk = k0 + 1; kk < K; ++kk)
                if (kk < ka) x[kk] = fma(-tj, bv[kk], x[kk]);
        };
        for (int L = 0; L < 32; L += 4) {
            const int j = 32 * k0 + L;
            if (j >= me) break;
            step(b0, L);
            load(b0, j + 4);
            if (j + 1 >= me) break;
            step(b1, L + 1);
            load(b1, j + 5);
            if (j + 2 >= me) break;
            step(b2, L + 2);
            load(b2, j + 6);
            if (j + 3 >= me) break;
            step(b3, L + 3);
            load(b3, j + 7);
        }
    }
}

// Rcs y' = x with y' = D y, i.e. R y = x, in place (x' on exit: the caller
// scales by 1 / R_pp): y'_p = x_p, then x_i -= Rcs_ip y'_p for i < p.
template <int K>
__device__ void warp_back_solve(const double *Rcs, int me, int m, double (&x)[K]) {
    const int lane = threadIdx.x & 31;
    const int ka = (me + 31) >> 5;
    auto load = [&](double (&bv)[K], int p) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int i = lane + 32 * kk;
            bv[kk] = (p >= 0 && p < me && kk < ka && i < p) ? Rcs[i + (int64_t)p * m] : 0.0;
        }
    };
    double b0[K], b1[K], b2[K], b3[K];
    const int top = 32 * ka - 1;   // ring position of p is (top - p) mod 4
    load(b0, top);
    load(b1, top - 1);
    load(b2, top - 2);
    load(b3, top - 3);
#pragma unroll
    for (int k0 = K - 1; k0 >= 0; --k0) {
        if (k0 < ka) {
            auto step = [&](const double (&bv)[K], int L) {
                const int p = 32 * k0 + L;
                if (p >= me) return;
                const double yp = __shfl_sync(0xffffffffu, x[k0], L);
                const int i0 = lane + 32 * k0;
                if (i0 < p) x[k0] = fma(-bv[k0], yp, x[k0]);
#pragma unroll
                for (int kk = 0; kk < k0; ++kk) x[kk] = fma(-bv[kk], yp, x[kk]);
            };
            for (int L = 31; L >= 0; L -= 4) {
                const int p = 32 * k0 + L;
                step(b0, L);
                load(b0, p - 4);
                step(b1, L - 1);
                load(b1, p - 5);
                step(b2, L - 2);
                load(b2, p - 6);
                step(b3, L - 3);
                load(b3, p - 7);
            }
        }
    }
}

template <int K>
__device__ __forceinline__ double warp_sumsq(const double (&x)[K]) {
    double v = 0.0;
#pragma unroll
    for (int kk = 0; kk < K; ++kk) v = fma(x[kk], x[kk], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// R_11 in compact form: RT (row-major), RTs = D^{-1} R (row-major) and
// Rcs = R D^{-1} (column-major), ld m, upper triangles with the diagonal;
// rinv = 1 / R_jj (0 for a zero pivot, which sets qstate[7]); cn2[q] =
// ||R(:, q)||^2 (thread q, in row order).
__global__ void __launch_bounds__(kThreads) k_r_pack(TailCtx c) {
    const int me = c.iscal[1];
    const int m = c.m;
    const int64_t tot = (int64_t)me * me;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t idx = gid; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % me), q = (int)(idx / me);
        double v = 0.0, vr = 0.0, vc = 0.0;
        if (i <= q) {
            v = i < q ? c.Aw[i + (int64_t)q * c.s] : c.Rdiag[q];
            const double di = c.Rdiag[i], dq = c.Rdiag[q];
            vr = di != 0.0 ? v / di : 0.0;
            vc = dq != 0.0 ? v / dq : 0.0;
        }
        c.RT[q + (int64_t)i * m] = v;
        c.RTs[q + (int64_t)i * m] = vr;
        c.Rcs[i + (int64_t)q * m] = vc;
    }
    if (gid < me) {
        const int q = (int)gid;
        const double d = c.Rdiag[q];
        c.rinv[q] = d != 0.0 ? 1.0 / d : 0.0;
        if (!(d != 0.0)) c.qstate[7] = 1.0;
        double a2 = 0.0;
        for (int i = 0; i < q; ++i) a2 = fma(c.Aw[i + (int64_t)q * c.s], c.Aw[i + (int64_t)q * c.s], a2);
        c.cn2[q] = fma(d, d, a2);
    }
}

// Rows of X R = T for T = R12 (-> M) and T = R22 (-> R2), one warp per row
// (relation form: T = [R_11 H(1:m, 1:m-1), R(1:m, m+1)] -> M only).  Two
// warps per CTA, so that the rows spread over the SMs (each step is a few
// FP64 instructions per warp; more warps per SM would queue on the FP64
// pipe).  The last CTA computes meanwhile the estimate of cond(R) (qstate[5]):
// ||R^{-1}|| LINPACK-style (warp 0) times the largest column norm of R (warp
// 1), and, in the relation form, gamma = R(m+1, m+1) / R(m, m) (qstate[6]).
template <int K>
__global__ void __launch_bounds__(64) k_tri_right(TailCtx c, int nblk_rows) {
    const int me = c.iscal[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = c.m;
    const int ka = (me + 31) >> 5;
    const bool gm = c.method == SKF_METHOD_SGMRES;
    if ((int)blockIdx.x == nblk_rows) {   // the cond(R) estimate
        __shared__ double res[2];
        const bool zp = c.qstate[7] != 0.0;
        if (warp == 0) {
            double z[K];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) z[kk] = 0.0;
            double r = INFINITY;
            if (!zp && me > 0) {
                warp_row_solve<K, true>(c.RTs, me, m, z);   // z' = D z, R^T z = b
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const int i = lane + 32 * kk;
                    z[kk] = (kk < ka && i < me) ? z[kk] * c.rinv[i] : 0.0;
                }
                const double zn = warp_sumsq(z);
                warp_back_solve<K>(c.Rcs, me, m, z);         // y' = D y, R y = z
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const int i = lane + 32 * kk;
                    z[kk] = (kk < ka && i < me) ? z[kk] * c.rinv[i] : 0.0;
                }
                const double yn = warp_sumsq(z);
                r = zn > 0.0 ? sqrt(yn / zn) : 0.0;
            }
            if (lane == 0) res[0] = r;
        } else {
            double mx = 0.0;
            for (int q = lane; q < me; q += 32) mx = fmax(mx, c.cn2[q]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) res[1] = sqrt(mx);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double mn = INFINITY, mxd = 0.0;
            for (int a2 = 0; a2 < me; ++a2) {
                mn = fmin(mn, fabs(c.Rdiag[a2]));
                mxd = fmax(mxd, fabs(c.Rdiag[a2]));
            }
            c.qstate[3] = mxd > 0.0 ? mn / mxd : 0.0;
            // never less than the diagonal ratio, a lower bound of cond(R)
            c.qstate[5] = me == 0 ? 0.0 : fmax(res[0] * res[1], mn > 0.0 ? mxd / mn : INFINITY);
            c.qstate[6] = (c.rel && gm && me > 0 && c.Rdiag[me - 1] != 0.0) ? c.Rdiag[me] / c.Rdiag[me - 1] : 0.0;
        }
        return;
    }
    const int row = blockIdx.x * 2 + warp;
    const int nrows = (gm && !c.rel) ? 2 * me : me;
    if (row >= nrows) return;
    const bool second = row >= me;
    const int a = second ? row - me : row;
    double x[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int j = lane + 32 * kk;
        double tv = 0.0;
        if (kk < ka && j < me) {
            if (c.rel) {
                if (j == me - 1) {
                    tv = c.Aw[a + (int64_t)me * c.s];   // R(a, m+1)
                } else {   // (R_11 H)(a, j): rows max(a, j-k+1) .. j+1 of column j of H
                    const int i1 = min(j + 1, me - 1);
                    for (int i = max(a, j - c.kt + 1); i <= i1; ++i)
                        tv = fma(c.RT[(int64_t)a * m + i], c.H[i + (int64_t)j * c.ldh], tv);
                }
            } else if (!second) {
                tv = c.Aw[a + (int64_t)(me + j) * c.s];
            } else if (j == a) {
                tv = c.Rdiag[me + a];
            } else if (j > a) {
                tv = c.Aw[(me + a) + (int64_t)(me + j) * c.s];
            }
        }
        x[kk] = tv;
    }
    warp_row_solve<K, false>(c.RTs, me, m, x);
    double *dst = second ? c.R2 : c.M;
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int j = lane + 32 * kk;
        if (kk < ka && j < me) dst[a + (int64_t)j * m] = x[kk] * c.rinv[j];
    }
}

// B = M + M^T, C = M^T M (+ R2^T R2; relation form: + gamma^2 e_m e_m^T)
// for the Cholesky node solves (not needed by the Givens ones), the
// transposes, c = ||b|| R_11 e_1, M^T c.
__global__ void __launch_bounds__(kThreads) k_tail_prep(TailCtx c) {
    const int me = c.iscal[1];
    const int64_t tot = (int64_t)me * me;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; !c.hess && idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % me), j = (int)(idx / me);
        if (j > i) continue;
        double acc = 0.0;
        for (int a = 0; a < me; ++a) acc = fma(c.M[a + (int64_t)i * c.m], c.M[a + (int64_t)j * c.m], acc);
        if (c.method == SKF_METHOD_SGMRES) {
            if (c.rel) {
                if (i == me - 1 && j == me - 1) acc = fma(c.qstate[6], c.qstate[6], acc);
            } else {
                for (int a = 0; a <= j; ++a) acc = fma(c.R2[a + (int64_t)i * c.m], c.R2[a + (int64_t)j * c.m], acc);
            }
        }
        c.C[i + (int64_t)j * c.m] = acc;
        c.B[i + (int64_t)j * c.m] = c.M[i + (int64_t)j * c.m] + c.M[j + (int64_t)i * c.m];
    }
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % me), j = (int)(idx / me);
        c.MT[j + (int64_t)i * c.m] = c.M[i + (int64_t)j * c.m];
        if (c.method == SKF_METHOD_SGMRES && !c.rel) c.R2T[j + (int64_t)i * c.m] = c.R2[i + (int64_t)j * c.m];
    }
    if (blockIdx.x == 0) {
        const double c0 = (1.0 / c.vscale[0]) * c.Rdiag[0];
        for (int j = threadIdx.x; j < me; j += blockDim.x) {
            c.cvec[j] = (j == 0) ? c0 : 0.0;
            c.Mtc[j] = c0 * c.M[(int64_t)j * c.m];
        }
    }
}

constexpr int kMixedMaxM = 320;   // packed FP32 factor of order m must fit in shared memory

__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }   // packed lower, row-major

// Solve L L^T z = z with the packed FP32 factor; one warp, z in FP64 shared
// memory, the solve itself in FP32 (the factor only preconditions the FP64
// refinement).  Column-oriented: lane l keeps rows l, l + 32, ... of z in
// registers; at step p the lane owning row p scales it by rinv[p] = 1/L_pp
// and broadcasts it, and every lane updates its own unsolved rows.  One
// shuffle per row instead of a reduction tree, and no FP64 conversions
// inside the recurrence.
constexpr int kSolveRegs = (kMixedMaxM + 31) / 32;
__device__ __forceinline__ void packed_solve_warp(const float *L, const float *rinv, int me, double *z) {
    const int lane = threadIdx.x & 31;
    float zr[kSolveRegs];
    int rowb[kSolveRegs];   // packed offset of row min(i, me - 1)
#pragma unroll
    for (int k = 0; k < kSolveRegs; ++k) {
        const int i = lane + 32 * k;
        zr[k] = i < me ? (float)z[i] : 0.f;
        rowb[k] = pk(min(i, me - 1), 0);
    }
    // Branch-free per register: every lane loads an in-range entry (rows past
    // me - 1 read row me - 1; entries right of the diagonal belong to later
    // rows of the packed array) and keeps or replaces its value by selects.
    for (int p = 0; p < me; ++p) {          // L u = z
        const int kp = p >> 5, lp = p & 31;
        float zp = zr[0];
#pragma unroll
        for (int k = 1; k < kSolveRegs; ++k) zp = (k == kp) ? zr[k] : zp;
        const float up = __shfl_sync(0xffffffffu, zp * rinv[p], lp);
#pragma unroll
        for (int k = 0; k < kSolveRegs; ++k) {
            const int i = lane + 32 * k;
            const float nz = fmaf(-L[rowb[k] + p], up, zr[k]);
            zr[k] = (i == p) ? up : ((i > p) ? nz : zr[k]);
        }
    }
    for (int p = me - 1; p >= 0; --p) {     // L^T x = u
        const int kp = p >> 5, lp = p & 31;
        float zp = zr[0];
#pragma unroll
        for (int k = 1; k < kSolveRegs; ++k) zp = (k == kp) ? zr[k] : zp;
        const float xp = __shfl_sync(0xffffffffu, zp * rinv[p], lp);
        const float *Lp = L + pk(p, 0);
#pragma unroll
        for (int k = 0; k < kSolveRegs; ++k) {
            const int i = lane + 32 * k;
            const float nz = fmaf(-Lp[min(i, p)], xp, zr[k]);
            zr[k] = (i == p) ? xp : ((i < p) ? nz : zr[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < kSolveRegs; ++k) {
        const int i = lane + 32 * k;
        if (i < me) z[i] = (double)zr[k];
    }
    __syncwarp();
}

// One CTA per quadrature node.  The normal matrix N(t) = t^2 I + t (M + M^T)
// + C is factored in FP32 (packed, in shared memory); the least-squares
// solution is then refined in FP64 with the residual of the original problem
// (semi-normal equations with iterative refinement), so the result has the
// accuracy of an FP64 least-squares solve whenever cond(X)^2 u_fp32 < 1.
// Nodes that do not converge are flagged for the FP64 kernel.
// Row a of -R2 y, and row j of R2^T r (r of length m_eff), for the node
// residuals (the second added to v): R2 upper triangular (ld m, transpose
// R2T), or, in the relation form, the single row gamma e_m^T.
__device__ __forceinline__ double r2_row(const TailCtx &c, int a, int me, const double *y) {
    if (c.rel) return a == 0 ? -c.qstate[6] * y[me - 1] : 0.0;
    double u = 0.0;
    for (int j = a; j < me; ++j) u = fma(-c.R2[a + (int64_t)j * c.m], y[j], u);
    return u;
}

__device__ __forceinline__ double r2t_row(const TailCtx &c, int j, int me, const double *r, double v) {
    if (c.rel) return j == me - 1 ? fma(c.qstate[6], r[0], v) : v;
    for (int a = 0; a <= j; ++a) v = fma(c.R2T[j + (int64_t)a * c.m], r[a], v);
    return v;
}

// Stopping test of the FP64 refinement of a node solve, on the squared norms
// of the correction d and the iterate y (partials loc[0], loc[1] of each of
// the NT threads): converged when ||d|| <= 1e-14 ||y||; given up when, from
// the third step on, ||d|| no longer halves (then converged only if
// ||d|| <= 1e-12 ||y||).  The warps' partials are added by thread 0 in warp
// order, so the decision is the same on every run.  snorm holds
// 2 NT / 32 + 2 doubles of scratch.  Returns 0 to go on, 1 converged, -1 not
// converged; prev2 is the previous ||d||^2 (start at +inf).
template <int NT>
__device__ __forceinline__ int refine_stop(double loc[2], int it, double &prev2, double *snorm) {
    constexpr int kW = NT / 32;
    for (int o = 16; o > 0; o >>= 1) {
        loc[0] += __shfl_xor_sync(0xffffffffu, loc[0], o);
        loc[1] += __shfl_xor_sync(0xffffffffu, loc[1], o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        snorm[warp] = loc[0];
        snorm[kW + warp] = loc[1];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d2 = 0.0, y2 = 0.0;
        for (int w = 0; w < kW; ++w) {
            d2 += snorm[w];
            y2 += snorm[kW + w];
        }
        int st = 0;
        if (d2 <= 1e-28 * y2) st = 1;
        else if (it >= 2 && d2 > 0.25 * prev2) st = d2 <= 1e-24 * y2 ? 1 : -1;
        snorm[2 * kW] = (double)st;
        snorm[2 * kW + 1] = d2;
    }
    __syncthreads();
    prev2 = snorm[2 * kW + 1];   // rewritten only after the next call's first barrier
    return (int)snorm[2 * kW];
}

__global__ void __launch_bounds__(kThreads) k_nodes_mixed(TailCtx c, int n0, int off) {
    extern __shared__ double smd[];
    const int me = c.iscal[1];
    if (c.qstate[0] != 0.0 || me == 0) return;
    const int m = c.m;
    const int row = off + blockIdx.x;
    if (me > kMixedMaxM) {
        if (threadIdx.x == 0) c.nodebad[row] = 1;
        return;
    }
    double *y = smd, *rt = smd + m, *rb = smd + 2 * m, *g = smd + 3 * m;
    float *colp = (float *)(smd + 4 * m);
    float *L = colp + m;
    const int nd = n0 + row;
    const double t = c.t[nd], wt = c.w[nd];
    const bool gm = c.method == SKF_METHOD_SGMRES;
    __shared__ int bad;
    __shared__ double snorm[2 * kThreads / 32 + 2];
    if (threadIdx.x == 0) bad = 0;
    for (int i = threadIdx.x; i < me; i += blockDim.x)
        for (int j = 0; j <= i; ++j)
            L[pk(i, j)] = (float)((i == j ? t * t : 0.0) + t * c.B[i + (int64_t)j * m] + c.C[i + (int64_t)j * m]);
    // blocked right-looking FP32 Cholesky, 32-column panels: the diagonal
    // block by one warp (lane = row, the pivot column passed through shared
    // memory), the rows below it solved against that block (one row per
    // thread, in registers), then the rank-32 update of the trailing matrix
    // by all warps (one warp per row, lanes along the row).  Three block
    // barriers per panel instead of two per column.
    {
        constexpr int kPB = 32;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int k0 = 0; k0 < me; k0 += kPB) {
            __syncthreads();
            const int kb = min(kPB, me - k0), k1 = k0 + kb;
            if (warp == 0) {
                for (int p = 0; p < kb; ++p) {
                    const float d = L[pk(k0 + p, k0 + p)];
                    if (!(d > 0.f)) {
                        if (lane == 0) bad = 1;
                        break;
                    }
                    const float lpp = sqrtf(d), rl = 1.f / lpp;
                    const bool below = lane > p && lane < kb;
                    const float lip = below ? L[pk(k0 + lane, k0 + p)] * rl : 0.f;
                    if (below) L[pk(k0 + lane, k0 + p)] = lip;
                    if (lane == p) L[pk(k0 + p, k0 + p)] = lpp;
                    if (lane < kb) colp[k0 + lane] = lip;
                    __syncwarp();
                    if (below)
                        for (int q = p + 1; q <= lane; ++q) L[pk(k0 + lane, k0 + q)] -= lip * colp[k0 + q];
                    __syncwarp();
                }
            }
            __syncthreads();
            if (bad) break;
            // rows below the block: x D^T = row, D the factored diagonal block
            for (int i = k1 + threadIdx.x; i < me; i += blockDim.x) {
                float r[kPB];
                float *Li = L + pk(i, k0);
#pragma unroll
                for (int p = 0; p < kPB; ++p) r[p] = p < kb ? Li[p] : 0.f;
#pragma unroll
                for (int p = 0; p < kPB; ++p) {
                    if (p < kb) {
                        float v = r[p];
                        const float *Dp = L + pk(k0 + p, k0);
#pragma unroll
                        for (int q = 0; q < kPB; ++q)
                            if (q < p) v = fmaf(-r[q], Dp[q], v);
                        r[p] = v / Dp[p];
                    }
                }
#pragma unroll
                for (int p = 0; p < kPB; ++p)
                    if (p < kb) Li[p] = r[p];
            }
            __syncthreads();
            // trailing update: L[i][q] -= sum_p L[i][k0+p] L[q][k0+p], k1 <= q <= i
            constexpr int kW = kThreads / 32;
            for (int i = k1 + warp; i < me; i += kW) {
                const float *Li = L + pk(i, k0);
                float ri[kPB];
#pragma unroll
                for (int p = 0; p < kPB; ++p) ri[p] = p < kb ? Li[p] : 0.f;
                float *Lrow = L + pk(i, 0);
                for (int q = k1 + lane; q <= i; q += 32) {
                    const float *Lq = L + pk(q, k0);
                    float acc = 0.f;
#pragma unroll
                    for (int p = 0; p < kPB; ++p)
                        if (p < kb) acc = fmaf(ri[p], Lq[p], acc);
                    Lrow[q] -= acc;
                }
            }
        }
    }
    __syncthreads();
    if (!bad) {
        // y0 = N^{-1} (t c + M^T c); colp <- 1/L_pp for the solves
        for (int a = threadIdx.x; a < me; a += blockDim.x) {
            y[a] = t * c.cvec[a] + c.Mtc[a];
            colp[a] = 1.f / L[pk(a, a)];
        }
        __syncthreads();
        if (threadIdx.x < 32) packed_solve_warp(L, colp, me, y);
        __syncthreads();
        double prev = INFINITY;
        bool conv = false;
        for (int it = 0; it < 12; ++it) {
            // r = [c; 0] - [t I + M; R2] y   (FP64)
            for (int a = threadIdx.x; a < me; a += blockDim.x) {
                double v = c.cvec[a] - t * y[a];
                for (int j = 0; j < me; ++j) v = fma(-c.M[a + (int64_t)j * m], y[j], v);
                rt[a] = v;
                if (gm) rb[a] = r2_row(c, a, me, y);
            }
            __syncthreads();
            // g = [t I + M; R2]^T r
            for (int j = threadIdx.x; j < me; j += blockDim.x) {
                double v = t * rt[j];
                for (int a = 0; a < me; ++a) v = fma(c.MT[j + (int64_t)a * m], rt[a], v);
                if (gm) v = r2t_row(c, j, me, rb, v);
                g[j] = v;
            }
            __syncthreads();
            if (threadIdx.x < 32) packed_solve_warp(L, colp, me, g);
            __syncthreads();
            double loc[2] = {0.0, 0.0};
            for (int a = threadIdx.x; a < me; a += blockDim.x) {
                loc[0] = fma(g[a], g[a], loc[0]);
                y[a] += g[a];
                loc[1] = fma(y[a], y[a], loc[1]);
            }
            const int st = refine_stop<kThreads>(loc, it, prev, snorm);
            if (st != 0) { conv = st > 0; break; }
        }
        if (!conv && threadIdx.x == 0) bad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) c.nodebad[row] = bad;
    if (!bad)
        for (int a = threadIdx.x; a < me; a += blockDim.x) c.out[(size_t)row * m + a] = wt * y[a];
}

// ---------------------------------------------------------------------------
// Node solves with the Cholesky factor in global memory (one slot of m x m
// per CTA): FP32 factor + FP64 refinement for m above the shared-memory limit
// of k_nodes_mixed, and the FP64 factor for the nodes that the FP32 factor
// cannot resolve (any m).
constexpr int kNodeThreads = 512;   // one thread per row of a panel (m <= 512)
constexpr int kNB = 32;             // panel width of the blocked Cholesky
constexpr int kKC = 64;             // factored columns staged per pass of the panel update

template <typename T> struct NodeSmem {
    double *y, *rt, *rb, *g;   // [m] each
    T *P;                      // panel [mp x kNB], ld mp
    T *Lt;                     // [kKC x kNB]: rows c0.. of staged factored columns
    T *D;                      // [32 x 32] diagonal block for the triangular solves
    T *sd;                     // [kNB] pivots of the panel
    int mp;
};

template <typename T> __device__ NodeSmem<T> node_smem(unsigned char *base, int m) {
    NodeSmem<T> s;
    s.mp = (m + 31) & ~31;
    double *d = (double *)base;
    s.y = d; s.rt = d + m; s.rb = d + 2 * m; s.g = d + 3 * m;
    T *t = (T *)(d + 4 * m);
    s.P = t; s.Lt = t + (size_t)s.mp * kNB; s.D = s.Lt + kKC * kNB; s.sd = s.D + 32 * 32;
    return s;
}

template <typename T> size_t node_smem_bytes(int m) {
    const int mp = (m + 31) & ~31;
    return sizeof(double) * 4 * (size_t)m + sizeof(T) * ((size_t)mp * kNB + kKC * kNB + 32 * 32 + kNB);
}

// Blocked left-looking Cholesky of a symmetric positive definite matrix N
// of order me, N_ij (i >= j) given by the functor nval, into L lower in
// global memory (column-major, leading dimension ld), in precision T.  Each
// panel of kNB columns is formed as N minus the product of the already
// factored rows (register tiles, one row per thread), then factored in shared
// memory (right-looking, pivot division deferred to a final scaling).
// Returns false on a nonpositive pivot (uniform over the CTA).
template <typename T, class NF>
__device__ bool chol_blocked_f(NF nval, int me, int ld, T *L, const NodeSmem<T> &sm) {
    const int mp = sm.mp, tid = threadIdx.x;
    for (int c0 = 0; c0 < me; c0 += kNB) {
        const int nb = min(kNB, me - c0), rows = me - c0;
        T acc[kNB];
#pragma unroll
        for (int u = 0; u < kNB; ++u) acc[u] = (T)0;
        for (int pk = 0; pk < c0; pk += kKC) {
            const int kc = min(kKC, c0 - pk);
            __syncthreads();
            for (int idx = tid; idx < kc * kNB; idx += blockDim.x) {
                const int q = idx / kNB, jj = idx % kNB;
                sm.Lt[idx] = jj < nb ? L[(c0 + jj) + (int64_t)(pk + q) * ld] : (T)0;
            }
            __syncthreads();
            if (tid < rows) {
                const T *lrow = L + (c0 + tid) + (int64_t)pk * ld;
                for (int q = 0; q < kc; ++q) {
                    const T a = lrow[(int64_t)q * ld];
                    const T *lt = sm.Lt + q * kNB;
#pragma unroll
                    for (int u = 0; u < kNB; ++u) acc[u] = fma(a, lt[u], acc[u]);
                }
            }
        }
        __syncthreads();
        if (tid < rows) {
            const int i = c0 + tid;
#pragma unroll
            for (int u = 0; u < kNB; ++u) {
                const int j = c0 + u;
                T v = (T)0;
                if (u < nb && i >= j) v = (T)nval(i, j) - acc[u];
                sm.P[tid + u * mp] = v;
            }
        }
        for (int k = 0; k < nb; ++k) {
            __syncthreads();
            const T d = sm.P[k + k * mp];
            if (!(d > (T)0)) return false;
            const T inv = (T)1 / d;
            const int w = nb - k - 1;
            for (int idx = tid; idx < (rows - k - 1) * w; idx += blockDim.x) {
                const int r = k + 1 + idx / w, jj = k + 1 + idx % w;
                if (jj <= r) sm.P[r + jj * mp] -= sm.P[r + k * mp] * sm.P[jj + k * mp] * inv;
            }
        }
        __syncthreads();
        if (tid < nb) sm.sd[tid] = sqrt(sm.P[tid + tid * mp]);
        __syncthreads();
        for (int idx = tid; idx < rows * nb; idx += blockDim.x) {
            const int r = idx % rows, k = idx / rows;
            if (r >= k) L[(c0 + r) + (int64_t)(c0 + k) * ld] = (r == k) ? sm.sd[k] : sm.P[r + k * mp] / sm.sd[k];
        }
        __syncthreads();
    }
    return true;
}

// The normal matrix of a real node t, N(t) = t^2 I + t B + C (B, C: lower
// triangles, ld m), factored as above with ld = m.
template <typename T>
__device__ bool chol_blocked(const TailCtx &c, double t, int me, T *L, const NodeSmem<T> &sm) {
    const int m = c.m;
    const double *B = c.B, *C = c.C;
    return chol_blocked_f<T>(
        [=](int i, int j) { return (i == j ? t * t : 0.0) + t * B[i + (int64_t)j * m] + C[i + (int64_t)j * m]; },
        me, m, L, sm);
}

// z <- (L L^T)^{-1} z with the global factor of chol_blocked; z is FP64 in
// shared memory, the arithmetic is in T.  Blocks of 32 rows: the diagonal
// block is solved by one warp from shared memory, the rest of the rows are
// updated by all threads.
template <typename T>
__device__ void chol_solve_g(const T *L, int me, int m, double *z, const NodeSmem<T> &sm) {
    const int tid = threadIdx.x, lane = tid & 31;
    auto load_diag = [&](int b0, int nb) {
        __syncthreads();
        for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
            const int q = idx >> 5, r = idx & 31;
            sm.D[idx] = (r < nb && q < nb && r >= q) ? L[(b0 + r) + (int64_t)(b0 + q) * m] : (T)0;
        }
        __syncthreads();
    };
    for (int b0 = 0; b0 < me; b0 += 32) {               // L u = z
        const int nb = min(32, me - b0);
        load_diag(b0, nb);
        if (tid < 32) {
            T zr = lane < nb ? (T)z[b0 + lane] : (T)0;
            for (int q = 0; q < nb; ++q) {
                if (lane == q) zr = zr / sm.D[q * 33];
                const T uq = __shfl_sync(0xffffffffu, zr, q);
                if (lane > q) zr = fma(-sm.D[lane + q * 32], uq, zr);
            }
            if (lane < nb) z[b0 + lane] = (double)zr;
        }
        __syncthreads();
        for (int r = b0 + nb + tid; r < me; r += blockDim.x) {
            T acc = (T)0;
            for (int q = 0; q < nb; ++q) acc = fma(L[r + (int64_t)(b0 + q) * m], (T)z[b0 + q], acc);
            z[r] -= (double)acc;
        }
    }
    for (int b0 = ((me - 1) / 32) * 32; b0 >= 0; b0 -= 32) {   // L^T x = u
        const int nb = min(32, me - b0);
        load_diag(b0, nb);
        if (tid < 32) {
            T xr = lane < nb ? (T)z[b0 + lane] : (T)0;
            for (int q = nb - 1; q >= 0; --q) {
                if (lane == q) xr = xr / sm.D[q * 33];
                const T xq = __shfl_sync(0xffffffffu, xr, q);
                if (lane < q) xr = fma(-sm.D[q + lane * 32], xq, xr);
            }
            if (lane < nb) z[b0 + lane] = (double)xr;
        }
        __syncthreads();
        for (int r = tid; r < b0; r += blockDim.x) {
            const T *col = L + (b0) + (int64_t)r * m;
            T acc = (T)0;
            for (int q = 0; q < nb; ++q) acc = fma(col[q], (T)z[b0 + q], acc);
            z[r] -= (double)acc;
        }
    }
    __syncthreads();
}

// r = [c; 0] - [t I + M; R2] y  (FP64; rb only for sGMRES), then
// g = [t I + M; R2]^T r.  Threads over rows / columns.
__device__ void node_residual(const TailCtx &c, double t, int me, const double *y, double *rt, double *rb, double *g,
                              bool gm) {
    const int m = c.m;
    __syncthreads();
    for (int a = threadIdx.x; a < me; a += blockDim.x) {
        double v = c.cvec[a] - t * y[a];
        for (int j = 0; j < me; ++j) v = fma(-c.M[a + (int64_t)j * m], y[j], v);
        rt[a] = v;
        if (gm) rb[a] = r2_row(c, a, me, y);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < me; j += blockDim.x) {
        double v = t * rt[j];
        for (int a = 0; a < me; ++a) v = fma(c.MT[j + (int64_t)a * m], rt[a], v);
        if (gm) v = r2t_row(c, j, me, rb, v);
        g[j] = v;
    }
    __syncthreads();
}

// One CTA per node (node n0 + off + blockIdx.x, workspace slot blockIdx.x).
// MIXED: FP32 factor, then FP64 iterative refinement on the original
// least-squares residual (semi-normal equations); a node that does not
// converge is flagged for the FP64 variant.  !MIXED (T = double): runs only
// for flagged nodes: FP64 factor, solve, one refinement step.
template <typename T, bool MIXED>
__global__ void __launch_bounds__(kNodeThreads) k_nodes_g(TailCtx c, int n0, int off) {
    extern __shared__ __align__(16) unsigned char nsm_raw[];
    const int me = c.iscal[1];
    if (c.qstate[0] != 0.0 || me == 0) return;
    const int row = off + blockIdx.x;
    if (!MIXED && !c.nodebad[row]) return;
    if (!MIXED && threadIdx.x == 0) atomicAdd(&c.qstate[4], 1.0);
    const int m = c.m;
    const NodeSmem<T> sm = node_smem<T>(nsm_raw, m);
    T *L = (T *)(c.Nw + (size_t)blockIdx.x * m * m);
    const int nd = n0 + row;
    const double t = c.t[nd], wt = c.w[nd];
    const bool gm = c.method == SKF_METHOD_SGMRES;
    double *y = sm.y, *rt = sm.rt, *rb = sm.rb, *g = sm.g;
    __shared__ double snorm[2 * kNodeThreads / 32 + 2];
    bool ok = chol_blocked<T>(c, t, me, L, sm);
    if (!ok) {
        if (MIXED) {
            if (threadIdx.x == 0) c.nodebad[row] = 1;
        } else {
            for (int a = threadIdx.x; a < me; a += blockDim.x) c.out[(size_t)row * m + a] = 0.0;
            if (threadIdx.x == 0)
                atomicExch(&c.iscal[2], gm ? (int)SKF_ERR_ILL_CONDITIONED : (int)SKF_ERR_BRANCH_CUT);
        }
        return;
    }
    for (int a = threadIdx.x; a < me; a += blockDim.x) y[a] = t * c.cvec[a] + c.Mtc[a];
    chol_solve_g<T>(L, me, m, y, sm);
    bool conv = !MIXED;
    const int iters = MIXED ? 12 : 1;
    double prev = INFINITY;
    for (int it = 0; it < iters; ++it) {
        node_residual(c, t, me, y, rt, rb, g, gm);
        chol_solve_g<T>(L, me, m, g, sm);
        double loc[2] = {0.0, 0.0};
        for (int a = threadIdx.x; a < me; a += blockDim.x) {
            loc[0] = fma(g[a], g[a], loc[0]);
            y[a] += g[a];
            loc[1] = fma(y[a], y[a], loc[1]);
        }
        if constexpr (MIXED) {
            const int st = refine_stop<kNodeThreads>(loc, it, prev, snorm);
            if (st != 0) { conv = st > 0; break; }
        }
    }
    __syncthreads();
    if (MIXED && threadIdx.x == 0) c.nodebad[row] = conv ? 0 : 1;
    if (conv)
        for (int a = threadIdx.x; a < me; a += blockDim.x) c.out[(size_t)row * m + a] = wt * y[a];
}

// Real node solves of the relation form.  There M = T R_11^{-1} with T upper
// Hessenberg (T = [R_11 H(1:m, 1:m-1), R(1:m, m+1)]), so M is upper
// Hessenberg, and so are t I + M (sFOM) and [t I + M; gamma e_m^T] (sGMRES,
// (m+1) x m); the right-hand side is c = c_0 e_1.  One warp per node reduces
// the node matrix to triangular form by Givens rotations of rows (j, j+1),
// j = 0, 1, ... (row j+1 of t I + M is read when it enters; the rotated row j
// is final), rotating c along, then solves the triangle by column-oriented
// back substitution: a backward stable QR solve in FP64, without normal
// equations or refinement, O(m^2) work per node.  Row j of the triangle is
// stored divided by its diagonal (R_jj = r = (a^2 + b^2)^{1/2}, so the stored
// row is (a x + b y) / r^2 and the right-hand side entry c_j / r), which gives
// the back substitution a unit diagonal; the rows go to the node's scratch
// slot in packed column-major order (column q at q (q + 1) / 2, rows 0 .. q-1)
// so that the back substitution reads each column contiguously.  Lane l holds
// columns (and rows) l, l + 32, ... in K register groups; the loops over the
// groups are unrolled, so the pivot's register is known at compile time.
constexpr int kHessWarps = 4;   // nodes (warps) per CTA

template <int K>
__global__ void __launch_bounds__(32 * kHessWarps) k_nodes_hess(TailCtx c, int n0, int off, int nn, double *Rs,
                                                                 size_t rstride) {
    const int me = c.iscal[1];
    if (c.qstate[0] != 0.0 || me == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x * kHessWarps + warp;
    if (slot >= nn) return;
    const int row = off + slot;
    const int nd = n0 + row;
    const double t = c.t[nd], wt = c.w[nd];
    const bool gm = c.method == SKF_METHOD_SGMRES;
    const double gam = gm ? c.qstate[6] : 0.0;
    const int m = c.m;
    const int ka = (me + 31) >> 5;   // register groups in use (warp-uniform)
    double *R = Rs + (size_t)slot * rstride;
    const double *MT = c.MT;         // row a of M at MT + a m
    double cr[K], nw[K], u[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int col = lane + 32 * kk;
        const bool in = kk < ka && col < me;
        cr[kk] = in ? __ldg(MT + col) + (col == 0 ? t : 0.0) : 0.0;   // row 0 of t I + M
        nw[kk] = (in && me > 1) ? __ldg(MT + m + col) : 0.0;            // row 1 of M
        u[kk] = 0.0;
    }
    double gc = c.cvec[0];   // the rotated right-hand side below the rows done
    bool bad = false;
#pragma unroll
    for (int k0 = 0; k0 < K; ++k0) {
        if (k0 >= ka) break;
        for (int L = 0; L < 32; ++L) {
            const int j = 32 * k0 + L;
            if (j >= me) break;
            const bool enter = j + 1 < me || gm;
            if (j + 1 < me) {   // shift of row j + 1
                if (L < 31) nw[k0] += (lane == L + 1) ? t : 0.0;
                else if (k0 + 1 < K) nw[k0 + 1] += (lane == 0) ? t : 0.0;
            } else if (gm) {    // the row gamma e_m^T of the sGMRES problem
#pragma unroll
                for (int kk = 0; kk < K; ++kk) nw[kk] = (lane + 32 * kk == me - 1) ? gam : 0.0;
            }
            // row j + 2 of M (columns > j), for the next step
            double pf[K];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const int col = lane + 32 * kk;
                pf[kk] = (kk >= k0 && kk < ka && j + 2 < me && col > j && col < me)
                             ? __ldg(MT + (size_t)(j + 2) * m + col) : 0.0;
            }
            const double a = __shfl_sync(0xffffffffu, cr[k0], L);
            const double b = __shfl_sync(0xffffffffu, nw[k0], L);
            double cs = 1.0, sn = 0.0, cs2 = 0.0, sn2 = 0.0, ri = 0.0;
            if (enter) {
                const double q = fma(a, a, b * b);
                if (q > 0.0 && q < INFINITY) {
                    ri = rsqrt(q);   // 1 / R_jj
                    cs = a * ri;
                    sn = b * ri;
                    cs2 = cs * ri;
                    sn2 = sn * ri;
                } else {
                    bad = true;
                }
            } else if (a != 0.0 && fabs(a) < INFINITY) {   // sFOM, last row: R_jj = a
                ri = 1.0 / a;
                cs2 = ri;
            } else {
                bad = true;
            }
            // row j of R / R_jj and the rotated carried row (columns > j);
            // the group of column j + 1 first
#pragma unroll
            for (int kk = k0; kk < K; ++kk) {
                if (kk < ka) {
                    const int col = lane + 32 * kk;
                    if (col > j && col < me) {
                        const double rj = fma(cs2, cr[kk], sn2 * nw[kk]);
                        cr[kk] = fma(cs, nw[kk], -(sn * cr[kk]));
                        R[(size_t)col * (col + 1) / 2 + j] = rj;
                    }
                }
            }
            u[k0] = (lane == L) ? cs * gc * ri : u[k0];
            gc = -sn * gc;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) nw[kk] = pf[kk];
        }
    }
    __syncwarp();
    // R y = u with the unit-diagonal rows: y_p = u_p, then u_i -= R_ip y_p for
    // i < p; column p - 4 is loaded while column p is applied
    auto load = [&](double (&bv)[K], int p) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const int i = lane + 32 * kk;
            bv[kk] = (p >= 0 && p < me && kk < ka && i < p) ? R[(size_t)p * (p + 1) / 2 + i] : 0.0;
        }
    };
    double b0[K], b1[K], b2[K], b3[K];
    const int top = 32 * ka - 1;
    load(b0, top);
    load(b1, top - 1);
    load(b2, top - 2);
    load(b3, top - 3);
#pragma unroll
    for (int k0 = K - 1; k0 >= 0; --k0) {
        if (k0 < ka) {
            auto step = [&](const double (&bv)[K], int L) {
                const int p = 32 * k0 + L;
                if (p >= me) return;
                const double yp = __shfl_sync(0xffffffffu, u[k0], L);
                const int i0 = lane + 32 * k0;
                if (i0 < p) u[k0] = fma(-bv[k0], yp, u[k0]);
#pragma unroll
                for (int kk = 0; kk < k0; ++kk) u[kk] = fma(-bv[kk], yp, u[kk]);
            };
            for (int L = 31; L >= 0; L -= 4) {
                const int p = 32 * k0 + L;
                step(b0, L);
                load(b0, p - 4);
                step(b1, L - 1);
                load(b1, p - 5);
                step(b2, L - 2);
                load(b2, p - 6);
                step(b3, L - 3);
                load(b3, p - 7);
            }
        }
    }
    bad = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int i = lane + 32 * kk;
        if (kk < ka && i < me) c.out[(size_t)row * m + i] = bad ? 0.0 : wt * u[kk];
    }
    if (bad && lane == 0) atomicExch(&c.iscal[2], gm ? (int)SKF_ERR_ILL_CONDITIONED : (int)SKF_ERR_BRANCH_CUT);
}

// Complex nodes (contour rules for a non-Stieltjes f, Algorithm 2): for
// t = alpha + i beta the node problem min || [t I + M; R2] y - [c; 0] || (or
// (t I + M) y = c for sFOM) is solved in real arithmetic for y = u + i v:
// the normal matrix of the real 4m x 2m least-squares problem
//   [[A1, -beta I], [beta I, A1], [R2, 0], [0, R2]] [u; v] ~ [c; 0; 0; 0],
// A1 = alpha I + M, is the 2m x 2m symmetric positive definite
//   [[N(alpha) + beta^2 I, beta (M - M^T)], [beta (M^T - M), N(alpha) + beta^2 I]]
// with N(alpha) = alpha^2 I + alpha B + C, and the right-hand side
// [alpha c + M^T c; -beta c].  FP64 factor (blocked, global slot of order
// 2 m_eff), solve, one refinement step on the residual of the original
// problem; the node contributes Re(w y) = Re(w) u - Im(w) v.
__device__ void node_residual_cplx(const TailCtx &c, double al, double be, int me, const double *y, double *rt,
                                   double *rb, double *g, bool gm) {
    const int m = c.m;
    const double *u = y, *v = y + me;
    __syncthreads();
    for (int a = threadIdx.x; a < me; a += blockDim.x) {
        double mu = 0.0, mv = 0.0;
        for (int j = 0; j < me; ++j) {
            const double mij = c.M[a + (int64_t)j * m];
            mu = fma(mij, u[j], mu);
            mv = fma(mij, v[j], mv);
        }
        rt[a] = c.cvec[a] - al * u[a] - mu + be * v[a];      // r1
        rt[me + a] = -be * u[a] - al * v[a] - mv;            // r2
        if (gm) {
            rb[a] = r2_row(c, a, me, u);        // r3
            rb[me + a] = r2_row(c, a, me, v);   // r4
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < me; j += blockDim.x) {
        double g1 = al * rt[j] + be * rt[me + j], g2 = -be * rt[j] + al * rt[me + j];
        for (int a = 0; a < me; ++a) {
            const double mt = c.MT[j + (int64_t)a * m];
            g1 = fma(mt, rt[a], g1);
            g2 = fma(mt, rt[me + a], g2);
        }
        if (gm) {
            g1 = r2t_row(c, j, me, rb, g1);
            g2 = r2t_row(c, j, me, rb + me, g2);
        }
        g[j] = g1;
        g[me + j] = g2;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kNodeThreads) k_nodes_cplx(TailCtx c, int n0, int off) {
    extern __shared__ __align__(16) unsigned char nsm_raw[];
    const int me = c.iscal[1];
    if (c.qstate[0] != 0.0 || me == 0) return;
    const int m = c.m, m2 = 2 * me, ld = 2 * m;
    const NodeSmem<double> sm = node_smem<double>(nsm_raw, 2 * m);
    const int row = off + blockIdx.x;
    double *L = c.Nw + (size_t)blockIdx.x * 4 * (size_t)m * m;
    const int nd = n0 + row;
    const double al = c.t[nd], be = c.ti[nd], wr = c.w[nd], wim = c.wi[nd];
    const bool gm = c.method == SKF_METHOD_SGMRES;
    const double *B = c.B, *C = c.C, *Mm = c.M;
    const bool ok = chol_blocked_f<double>(
        [=](int i, int j) {
            const int bi = i >= me, bj = j >= me;
            const int ii = i - bi * me, jj = j - bj * me;
            if (bi == bj)
                return (ii == jj ? al * al + be * be : 0.0) + al * B[ii + (int64_t)jj * m] + C[ii + (int64_t)jj * m];
            return be * (Mm[jj + (int64_t)ii * m] - Mm[ii + (int64_t)jj * m]);   // block (2,1) = beta (M^T - M)
        },
        m2, ld, L, sm);
    if (!ok) {
        for (int a = threadIdx.x; a < me; a += blockDim.x) c.out[(size_t)row * m + a] = 0.0;
        if (threadIdx.x == 0) atomicExch(&c.iscal[2], gm ? (int)SKF_ERR_ILL_CONDITIONED : (int)SKF_ERR_BRANCH_CUT);
        return;
    }
    double *y = sm.y, *rt = sm.rt, *rb = sm.rb, *g = sm.g;
    for (int a = threadIdx.x; a < me; a += blockDim.x) {
        y[a] = al * c.cvec[a] + c.Mtc[a];
        y[me + a] = -be * c.cvec[a];
    }
    chol_solve_g<double>(L, m2, ld, y, sm);
    node_residual_cplx(c, al, be, me, y, rt, rb, g, gm);
    chol_solve_g<double>(L, m2, ld, g, sm);
    for (int a = threadIdx.x; a < me; a += blockDim.x)
        c.out[(size_t)row * m + a] = wr * (y[a] + g[a]) - wim * (y[me + a] + g[me + a]);
}

// Sum the node solutions of each level of the batch (CTA i: level lev0 + i,
// four interleaved partial sums over its nodes, added in a fixed order), then
// the last CTA to finish runs the acceptance test of Sec. 4.1 level by level.
__global__ void __launch_bounds__(kThreads) k_levels(TailCtx c, int lev0, int nlev, const int *lev_start,
                                                     const int *lev_ell, int n0, double tol, int last_batch) {
    __shared__ double red[64];
    __shared__ int is_last;
    const int me = c.iscal[1];
    if (c.qstate[0] != 0.0 || me == 0) return;
    const int m = c.m;
    {
        const int l = lev0 + (int)blockIdx.x;
        const int a0 = lev_start[l] - n0, a1 = lev_start[l + 1] - n0;
        double *ql = c.qbuf + (size_t)l * m;
        for (int a = threadIdx.x; a < me; a += blockDim.x) {
            double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
            int nd = a0;
            for (; nd + 3 < a1; nd += 4) {
                p0 += c.out[(size_t)nd * m + a];
                p1 += c.out[(size_t)(nd + 1) * m + a];
                p2 += c.out[(size_t)(nd + 2) * m + a];
                p3 += c.out[(size_t)(nd + 3) * m + a];
            }
            for (; nd < a1; ++nd) p0 += c.out[(size_t)nd * m + a];
            ql[a] = (p0 + p1) + (p2 + p3);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(c.lev_cnt, 1u) == (unsigned)(nlev - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) *c.lev_cnt = 0u;   // ready for the next batch
    for (int l = lev0; l < lev0 + nlev; ++l) {
        const double *ql = c.qbuf + (size_t)l * m;
        bool accept = false;
        double rel = 0.0;
        if (c.nlevels == 1) {
            accept = true;
        } else if (l > 0) {
            const double *qp = c.qbuf + (size_t)(l - 1) * m;
            double v[2] = {0.0, 0.0};
            for (int a = threadIdx.x; a < me; a += blockDim.x) {
                const double qa = __ldcg(ql + a);
                const double d = qa - __ldcg(qp + a);
                v[0] = fma(d, d, v[0]);
                v[1] = fma(qa, qa, v[1]);
            }
            block_sum<2>(v, red);
            __shared__ double sv2[2];
            if (threadIdx.x == 0) { sv2[0] = v[0]; sv2[1] = v[1]; }
            __syncthreads();
            rel = sv2[1] > 0.0 ? sqrt(sv2[0] / sv2[1]) : 0.0;
            accept = sqrt(sv2[0]) <= tol * sqrt(sv2[1]);
        }
        const bool final_level = last_batch && (l == lev0 + nlev - 1);
        if (accept || final_level) {
            for (int a = threadIdx.x; a < me; a += blockDim.x) c.qacc[a] = __ldcg(ql + a);
            if (threadIdx.x == 0) {
                c.qstate[0] = 1.0;
                c.qstate[1] = (double)lev_ell[l];
                c.qstate[2] = rel;
                if (!accept && c.iscal[2] == SKF_OK) c.iscal[2] = SKF_ERR_QUAD_NOT_CONVERGED;
            }
            __syncthreads();
            return;
        }
        __syncthreads();
    }
}

// y = R^{-1} q_acc, z = vscale .* y: one warp (warp_back_solve);
// ILL_CONDITIONED when R has a zero pivot or the estimate of cond(R)
// (k_tri_right) exceeds cond_max.
template <int K>
__global__ void __launch_bounds__(32) k_coeffs(TailCtx c) {
    const int me = c.iscal[1];
    const int lane = threadIdx.x & 31;
    const bool zero_pivot = c.qstate[7] != 0.0;
    double x[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) x[kk] = (lane + 32 * kk < me) ? c.qacc[lane + 32 * kk] : 0.0;
    if (!zero_pivot) warp_back_solve<K>(c.Rcs, me, c.m, x);
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int i = lane + 32 * kk;
        if (i < me) c.z[i] = zero_pivot ? 0.0 : c.vscale[i] * (x[kk] * c.rinv[i]);
    }
    if (lane == 0 && me > 0 && c.iscal[2] == SKF_OK &&
        (zero_pivot || (c.cond_max > 0.0 && c.qstate[5] > c.cond_max)))
        c.iscal[2] = SKF_ERR_ILL_CONDITIONED;
}

// x = V z (tall-skinny GEMV over the stored basis).
__global__ void __launch_bounds__(kThreads) k_recombine(const double *__restrict__ V, int64_t ldv, int64_t n,
                                                        const double *__restrict__ z, const int *iscal,
                                                        double *__restrict__ x) {
    const int me = iscal[1];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < me; ++j) acc = fma(V[r + (int64_t)j * ldv], z[j], acc);
        x[r] = acc;
    }
}

// Two recombinations in one pass over V: x0 = V z0, x1 = V z1 (the sFOM and
// sGMRES approximants of one Arnoldi process); each sum in the order of
// k_recombine, so each output equals the one-method result bit for bit.
__global__ void __launch_bounds__(kThreads) k_recombine2(const double *__restrict__ V, int64_t ldv, int64_t n,
                                                         const double *__restrict__ z0,
                                                         const double *__restrict__ z1, const int *iscal,
                                                         double *__restrict__ x0, double *__restrict__ x1) {
    extern __shared__ double zz[];   // [2 me]
    const int me = iscal[1];
    for (int j = threadIdx.x; j < me; j += blockDim.x) {
        zz[2 * j] = z0[j];
        zz[2 * j + 1] = z1[j];
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double a0 = 0.0, a1 = 0.0;
        for (int j = 0; j < me; ++j) {
            const double v = V[r + (int64_t)j * ldv];
            a0 = fma(v, zz[2 * j], a0);
            a1 = fma(v, zz[2 * j + 1], a1);
        }
        x0[r] = a0;
        x1[r] = a1;
    }
}

// A second method's tail on the shared whitening: its state starts from the
// first method's (rdiag ratio, cond(R) estimate, gamma, zero-pivot flag;
// convergence fields cleared), and a failure of the shared part (a QR
// timeout) is carried over to its status.
__global__ void k_fork_state(const double *__restrict__ q0, double *__restrict__ q1, const int *__restrict__ isc0,
                             int *__restrict__ isc1) {
    if (threadIdx.x < 8) {
        const int i = threadIdx.x;
        q1[i] = (i == 3 || i >= 5) ? q0[i] : 0.0;
    }
    if (threadIdx.x == 0 && isc1[2] == SKF_OK && isc0[2] == SKF_ERR_TIMEOUT) isc1[2] = SKF_ERR_TIMEOUT;
}

// f = V_m z for an FP32 or BF16 basis.  Each product v z_j is formed exactly
// as a float pair (z_j = zh + zl, Dekker product through fmaf) and summed in
// double-float arithmetic (Knuth's TwoSum), so the sum keeps about 44 bits
// while running on the FP32 pipes; the pair is added in FP64 once per row.
__device__ __forceinline__ float load_basis(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_basis(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ double load_basis_any(const double *p) { return __ldg(p); }
__device__ __forceinline__ float load_basis_any(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_basis_any(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

template <typename TB>
__global__ void __launch_bounds__(kThreads) k_recombine_lp(const TB *__restrict__ V, int64_t ldv, int64_t n,
                                                           const double *__restrict__ z, const int *iscal,
                                                           double *__restrict__ x) {
    extern __shared__ float zs[];   // [2 me]: hi and lo parts of z
    const int me = iscal[1];
    for (int j = threadIdx.x; j < me; j += blockDim.x) {
        const float hi = (float)z[j];
        zs[2 * j] = hi;
        zs[2 * j + 1] = (float)(z[j] - (double)hi);
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        float sh = 0.f, sl = 0.f;
        for (int j = 0; j < me; ++j) {
            const float v = load_basis(V + r + (int64_t)j * ldv);
            const float zh = zs[2 * j], zl = zs[2 * j + 1];
            const float ph = v * zh;
            const float pe = fmaf(v, zl, fmaf(v, zh, -ph));
            const float t = sh + ph;
            const float bp = t - sh;
            const float err = (sh - (t - bp)) + (ph - bp);
            sh = t;
            sl += err + pe;
        }
        x[r] = (double)sh + (double)sl;
    }
}

// S f = S V y = sum_j S v_j y_j with y_j = z_j / vscale_j (sketched form of
// the approximant, for the stopping criterion); one thread per row of S.
__global__ void __launch_bounds__(kThreads) k_sketch_f(TailCtx c, const double *__restrict__ SV, double *__restrict__ sf) {
    const int me = c.iscal[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.s; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < me; ++j) acc = fma(SV[i + (size_t)j * c.s], c.z[j] / c.vscale[j], acc);
        sf[i] = acc;
    }
}

// z_out[j] = z_j for j < m_eff, 0 beyond.
__global__ void k_copy_z(TailCtx c, double *__restrict__ z_out) {
    const int me = c.iscal[1];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < c.m) z_out[j] = j < me ? c.z[j] : 0.0;
}

// Two-pass recombination, one column at a time: x (+)= z_j w_j.
template <typename TB>
__global__ void __launch_bounds__(kThreads) k_accum(const TB *__restrict__ w, const double *__restrict__ z,
                                                    const int *__restrict__ iscal, int j, int64_t n,
                                                    double *__restrict__ x) {
    const int me = iscal[1];
    if (j > 0 && j >= me) return;
    const double zj = j < me ? z[j] : 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double wr = (double)load_basis_any(w + r);
        x[r] = j == 0 ? fma(wr, zj, 0.0) : fma(wr, zj, x[r]);
    }
}

// Checkpoint p of the stopping criterion: skipped (m_eff 0 for the tail)
// once the recurrence has stopped.
__global__ void k_check_begin(const int *__restrict__ iscal, int *__restrict__ iscal_chk, int p) {
    if (threadIdx.x != 0) return;
    iscal_chk[0] = 0;
    iscal_chk[1] = iscal[0] != 0 ? 0 : p;
    iscal_chk[2] = SKF_OK;
    iscal_chk[3] = p;
}

// est_p = ||S f_p - S f_{p-d}|| / sqrt(1 - eps) / (||S f_p|| / sqrt(1 + eps)),
// eps = max_{j<p} | ||S v_j||^2 - 1 | (Sec. 4.3); on est_p <= stop_tol the
// recurrence stops at m_eff = p.  One CTA.
__global__ void __launch_bounds__(kThreads) k_check_end(const double *__restrict__ SV, int s, int p, int *iscal,
                                                        const int *__restrict__ iscal_chk, double *sf_prev,
                                                        const double *__restrict__ sf_cur, double *state,
                                                        double stop_tol) {
    __shared__ double red[64];
    if (iscal_chk[1] == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double eps = 0.0;
    for (int j = warp; j < p; j += kThreads / 32) {
        double a = 0.0;
        for (int i = lane; i < s; i += 32) a = fma(SV[i + (size_t)j * s], SV[i + (size_t)j * s], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        eps = fmax(eps, fabs(a - 1.0));
    }
    eps = block_max(eps, red);
    __syncthreads();
    double v[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
        const double d = sf_cur[i] - sf_prev[i];
        v[0] = fma(d, d, v[0]);
        v[1] = fma(sf_cur[i], sf_cur[i], v[1]);
    }
    block_sum<2>(v, red);
    __shared__ double sv2[2];
    if (threadIdx.x == 0) { sv2[0] = v[0]; sv2[1] = v[1]; }
    __syncthreads();
    const bool ok = iscal_chk[2] == SKF_OK;
    if (threadIdx.x == 0) {
        if (ok && state[0] != 0.0 && eps < 1.0 && sv2[1] > 0.0) {
            const double rel = sqrt(sv2[0] / (1.0 - eps)) / sqrt(sv2[1] / (1.0 + eps));
            state[1] = rel;
            if (rel <= stop_tol && iscal[0] == 0) {
                iscal[0] = 2;
                iscal[1] = p;
                iscal[3] = p;
                state[2] = (double)p;
            }
        }
        state[0] = ok ? 1.0 : 0.0;
    }
    if (ok)
        for (int i = threadIdx.x; i < s; i += blockDim.x) sf_prev[i] = sf_cur[i];
}

__global__ void k_write_info(TailCtx c, skf_info *info, const double *stop_state) {
    if (threadIdx.x != 0 || info == nullptr) return;
    info->stop_m = stop_state ? (int)stop_state[2] : 0;
    info->err_est = stop_state ? stop_state[1] : 0.0;
    info->status = c.iscal[2];
    info->m_eff = c.iscal[1];
    info->ell = (int)c.qstate[1];
    info->quad_err = c.qstate[2];
    info->rdiag_ratio = c.qstate[3];
    info->nodes_fp64 = (int)c.qstate[4];
    info->cond_est = c.qstate[5];
}

}  // namespace

// Host driver of the tail.  `rule` holds all levels of the adaptive
// schedule; levels are evaluated in batches (speculatively, several levels per
// launch) and accepted in schedule order, which gives the same accepted order
// as evaluating one level at a time.
static int g_qr_mode = 0;   // 0 automatic (cooperative QR where it fits), 1 per-reflector launches
void set_qr_mode(int mode) { g_qr_mode = mode; }
int qr_mode() { return g_qr_mode; }
static int g_tail_form = 0;   // 0 automatic (relation form with an FP64 basis), 1 full QR of [S V_m, S A V_m]
void set_tail_form(int form) { g_tail_form = form; }
int tail_form() { return g_tail_form; }

skf_status tail_run_multi(int nout, const TailOut *outs, int s, int m, int64_t n, const void *V, skf_dtype vdt,
                          int64_t ldv, const double *vscale, const double *SV, const double *SAV, const RuleDev &rule,
                          double tol, cudaStream_t st, double *sketch_out, const double *stop_state, double cond_max,
                          const double *H, int ldh, int kt) {
    if (nout < 1 || nout > 2) return fail(SKF_ERR_INVALID_ARG, "tail: one or two methods");
    // the shared part (QR, M, cond(R), gamma) is that of the most demanding method
    skf_method method = outs[0].method;
    for (int i = 1; i < nout; ++i)
        if (outs[i].method == SKF_METHOD_SGMRES) method = SKF_METHOD_SGMRES;
    int *iscal = outs[0].iscal;
    TailCtx c{};
    c.cond_max = cond_max;
    // relation form where H is given and the sketched relation holds for the
    // stored basis: FP64, and FP32 (whose S A v_j, j < m - 1, are formed from
    // that relation with the coefficients the update applied).  A BF16 basis
    // keeps the full form: its relation is off by the storage rounding of
    // w_{j+1}, which S A v_j takes off.
    c.rel = (tail_form() != 1 && H != nullptr && (vdt == SKF_F64 || vdt == SKF_F32) && m >= 1) ? 1 : 0;
    c.H = H;
    c.ldh = ldh;
    c.kt = kt;
    c.hess = (c.rel && !rule.cplx) ? 1 : 0;
    c.s = s;
    c.m = m;
    c.method = method;
    c.iscal = iscal;
    c.vscale = vscale;
    c.t = rule.t;
    c.ti = rule.t_im;
    c.wi = rule.w_im;
    c.w = rule.w;
    c.nlevels = rule.nlevels;
    int max_level = 0;
    for (int l = 0; l < rule.nlevels; ++l) max_level = std::max(max_level, rule.h_start[l + 1] - rule.h_start[l]);
    // batches of consecutive levels filling at most one wave of node CTAs
    // (2 per SM; Givens node solves: 4 warps per SM); a larger level forms a
    // batch of its own (never split)
    const int wave = (c.hess ? 4 : 2) * num_sms();
    const int cap = std::max(wave, max_level);
    std::vector<std::pair<int, int>> batches;   // (first level, count)
    for (int l = 0; l < rule.nlevels;) {
        int cnt = 0, nodes = 0;
        while (l + cnt < rule.nlevels) {
            const int sz = rule.h_start[l + cnt + 1] - rule.h_start[l + cnt];
            if (cnt > 0 && nodes + sz > wave) break;
            nodes += sz;
            ++cnt;
        }
        batches.push_back({l, cnt});
        l += cnt;
    }
    const int chunk = wave;   // node solves per launch (scratch slots)
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t mm = (size_t)m * m;
    const size_t rstride = (size_t)m * (m + 1) / 2;   // Givens node solves: packed triangle per slot
    const size_t nw_bytes = c.hess ? sizeof(double) * chunk * rstride
                                   : sizeof(double) * chunk * mm * (rule.cplx ? 4 : 1);
    const size_t sizes[] = {sizeof(double) * (size_t)s * 2 * m, sizeof(double) * 2 * m, sizeof(double) * mm,
                            sizeof(double) * mm, sizeof(double) * mm, sizeof(double) * mm, sizeof(double) * m,
                            sizeof(double) * m, nw_bytes, sizeof(double) * (size_t)cap * m,
                            sizeof(double) * (size_t)rule.nlevels * m * nout, sizeof(double) * m * nout,
                            sizeof(double) * m * nout, sizeof(double) * 8 * nout, sizeof(double) * mm,
                            sizeof(double) * mm, sizeof(int) * (size_t)cap, sizeof(double) * 2 * (size_t)m,
                            sizeof(unsigned) * 4, sizeof(double) * mm, sizeof(double) * mm, sizeof(double) * m,
                            sizeof(double) * mm, sizeof(double) * m};
    constexpr int kNbuf = sizeof(sizes) / sizeof(sizes[0]);
    size_t total = 0;
    for (size_t v : sizes) total += al(v);
    char *ws = nullptr;
    skf_status stt = dalloc((void **)&ws, total, st);
    if (stt != SKF_OK) return stt;
    double *ptrs[kNbuf];
    size_t off = 0;
    for (int i = 0; i < kNbuf; ++i) {
        ptrs[i] = (double *)(ws + off);
        off += al(sizes[i]);
    }
    c.Aw = ptrs[0]; c.Rdiag = ptrs[1]; c.M = ptrs[2]; c.R2 = ptrs[3]; c.B = ptrs[4]; c.C = ptrs[5];
    c.cvec = ptrs[6]; c.Mtc = ptrs[7]; c.Nw = ptrs[8]; c.out = ptrs[9]; c.qbuf = ptrs[10]; c.qacc = ptrs[11];
    c.z = ptrs[12]; c.qstate = ptrs[13]; c.MT = ptrs[14]; c.R2T = ptrs[15]; c.nodebad = (int *)ptrs[16];
    c.hsig = ptrs[17];
    unsigned *qr_ready = (unsigned *)ptrs[18];   // [0] published pivot columns, [1] timeout flag
    c.RT = ptrs[19];
    c.RTs = ptrs[20];
    c.rinv = ptrs[21];
    c.Rcs = ptrs[22];
    c.cn2 = ptrs[23];
    c.lev_cnt = qr_ready + 2;
    const int G = std::min(2 * num_sms(), 1024);
    long long nlaunch = 0;
    k_tail_copy<<<G, kThreads, 0, st>>>(SV, SAV, c);
    ++nlaunch;
    const int ncols_max = c.rel ? m + 1 : 2 * m;   // columns of the factored matrix at m_eff = m
    const int nref = (method == SKF_METHOD_SGMRES) ? ncols_max : m;
    // the QR in one cooperative launch (k_qr_persist): every column's owner
    // CTA must be resident, with at most kQrOwn columns per CTA
    bool qr_done = false;
    if (qr_mode() != 1) {
        const int cols = std::max(1, ncols_max);   // every column has an owner CTA holding it
        int Gq = std::min(cols, num_sms());
        if ((cols + kQrOwn - 1) / kQrOwn > Gq) Gq = (cols + kQrOwn - 1) / kQrOwn;
        int dev = 0, per_sm = 0, coop = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
            cudaFuncSetAttribute(k_qr_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)qr_smem_bytes(s)) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_persist, kQrThreads, qr_smem_bytes(s)) ==
                cudaSuccess &&
            Gq <= per_sm * num_sms()) {
            cudaMemsetAsync(qr_ready, 0, sizeof(unsigned) * 4, st);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeCooperative;
            at[0].val.cooperative = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)Gq);
            cfg.blockDim = dim3(kQrThreads);
            cfg.dynamicSmemBytes = qr_smem_bytes(s);
            cfg.stream = st;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            qr_done = cudaLaunchKernelEx(&cfg, k_qr_persist, c, qr_ready, (int *)(qr_ready + 1)) == cudaSuccess;
            if (!qr_done) cudaGetLastError();
            else ++nlaunch;
        } else {
            cudaGetLastError();
        }
    }
    // otherwise the 2m (sGMRES) or m (sFOM) reflector launches, each a
    // programmatic dependent of the one before, so that launch latency
    // overlaps the previous reflector
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    for (int jj = 0; !qr_done && jj < nref; ++jj) {
        const int ntrail = std::max(1, ncols_max - jj - 1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)ntrail);
        cfg.blockDim = dim3(kHhThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cfg.attrs = pdl;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_householder, c, jj);
    }
    if (!qr_done) nlaunch += nref;
    k_r_pack<<<(unsigned)std::max<size_t>(1, std::min<size_t>((mm + kThreads - 1) / kThreads, 4 * num_sms())),
               kThreads, 0, st>>>(c);
    ++nlaunch;
    {
        const int rows = (method == SKF_METHOD_SGMRES && !c.rel) ? 2 * m : m;
        const unsigned blocks = (unsigned)((rows + 1) / 2);
        // + 1 CTA: the cond(R) estimate
        if (m <= 64) k_tri_right<2><<<blocks + 1, 64, 0, st>>>(c, (int)blocks);
        else if (m <= 128) k_tri_right<4><<<blocks + 1, 64, 0, st>>>(c, (int)blocks);
        else if (m <= 256) k_tri_right<8><<<blocks + 1, 64, 0, st>>>(c, (int)blocks);
        else k_tri_right<16><<<blocks + 1, 64, 0, st>>>(c, (int)blocks);
        ++nlaunch;
    }
    // FP32 factor: packed in shared memory up to kMixedMaxM, else a global slot
    const bool packed = m <= kMixedMaxM;
    const size_t msmem = sizeof(double) * 4 * m + sizeof(float) * ((size_t)m + (size_t)m * (m + 1) / 2);
    const size_t gsm32 = node_smem_bytes<float>(m), gsm64 = node_smem_bytes<double>(m);
    const size_t gsmC = node_smem_bytes<double>(2 * m);
    if (rule.cplx && gsmC > 48 * 1024)
        cudaFuncSetAttribute(k_nodes_cplx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmC);
    if (packed && msmem > 48 * 1024)
        cudaFuncSetAttribute(k_nodes_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
    if (!packed && gsm32 > 48 * 1024)
        cudaFuncSetAttribute(k_nodes_g<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm32);
    if (gsm64 > 48 * 1024)
        cudaFuncSetAttribute(k_nodes_g<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm64);
    // per method: its context (own qstate, quadrature buffers, coefficients,
    // status), node solves, level sums and coefficients
    TailCtx cm[2];
    for (int i = 0; i < nout; ++i) {
        cm[i] = c;
        cm[i].method = outs[i].method;
        cm[i].iscal = outs[i].iscal;
        cm[i].qbuf = c.qbuf + (size_t)i * rule.nlevels * m;
        cm[i].qacc = c.qacc + (size_t)i * m;
        cm[i].z = c.z + (size_t)i * m;
        cm[i].qstate = c.qstate + (size_t)i * 8;
    }
    for (int mi = 0; mi < nout; ++mi) {
        const TailCtx &cc = cm[mi];
        if (mi > 0) {
            k_fork_state<<<1, 32, 0, st>>>(c.qstate, cc.qstate, iscal, cc.iscal);
            ++nlaunch;
        }
        // the normal matrices of the Cholesky node solves depend on the method
        if (mi == 0 || !c.hess) {
            k_tail_prep<<<G, kThreads, 0, st>>>(cc);
            ++nlaunch;
        }
        for (size_t bi = 0; bi < batches.size(); ++bi) {
            const int l0 = batches[bi].first, nl = batches[bi].second;
            const int n0 = rule.h_start[l0];
            const int nn = rule.h_start[l0 + nl] - n0;
            for (int o = 0; o < nn; o += chunk) {
                const int nb = std::min(chunk, nn - o);
                if (cc.hess) {
                    const unsigned g = (unsigned)((nb + kHessWarps - 1) / kHessWarps);
                    if (m <= 64) k_nodes_hess<2><<<g, 32 * kHessWarps, 0, st>>>(cc, n0, o, nb, cc.Nw, rstride);
                    else if (m <= 128) k_nodes_hess<4><<<g, 32 * kHessWarps, 0, st>>>(cc, n0, o, nb, cc.Nw, rstride);
                    else if (m <= 256) k_nodes_hess<8><<<g, 32 * kHessWarps, 0, st>>>(cc, n0, o, nb, cc.Nw, rstride);
                    else k_nodes_hess<16><<<g, 32 * kHessWarps, 0, st>>>(cc, n0, o, nb, cc.Nw, rstride);
                    nlaunch += 1;
                    continue;
                }
                if (rule.cplx) {
                    k_nodes_cplx<<<nb, kNodeThreads, gsmC, st>>>(cc, n0, o);
                } else {
                    if (packed) k_nodes_mixed<<<nb, kThreads, msmem, st>>>(cc, n0, o);
                    else k_nodes_g<float, true><<<nb, kNodeThreads, gsm32, st>>>(cc, n0, o);
                    k_nodes_g<double, false><<<nb, kNodeThreads, gsm64, st>>>(cc, n0, o);
                }
                nlaunch += 2;
            }
            k_levels<<<(unsigned)nl, kThreads, 0, st>>>(cc, l0, nl, rule.lev_start, rule.lev_ell, n0, tol,
                                             bi + 1 == batches.size() ? 1 : 0);
            ++nlaunch;
        }
        if (m <= 64) k_coeffs<2><<<1, 32, 0, st>>>(cc);
        else if (m <= 128) k_coeffs<4><<<1, 32, 0, st>>>(cc);
        else if (m <= 256) k_coeffs<8><<<1, 32, 0, st>>>(cc);
        else k_coeffs<16><<<1, 32, 0, st>>>(cc);
        ++nlaunch;
        if (outs[mi].z_out) {
            k_copy_z<<<(m + kThreads - 1) / kThreads, kThreads, 0, st>>>(cc, outs[mi].z_out);
            ++nlaunch;
        }
    }
    const int64_t rb = std::min<int64_t>((n + kThreads - 1) / kThreads, 16 * num_sms());
    const unsigned rgrid = (unsigned)std::max<int64_t>(rb, 1);
    const size_t zsm = sizeof(float) * 2 * (size_t)m;
    if (sketch_out) {
        k_sketch_f<<<(s + kThreads - 1) / kThreads, kThreads, 0, st>>>(cm[0], SV, sketch_out);
        ++nlaunch;
    } else if (nout == 2 && vdt == SKF_F64 && outs[0].x && outs[1].x) {
        k_recombine2<<<rgrid, kThreads, sizeof(double) * 2 * m, st>>>((const double *)V, ldv, n, cm[0].z, cm[1].z,
                                                                        iscal, outs[0].x, outs[1].x);
        ++nlaunch;
    } else {
        for (int mi = 0; mi < nout; ++mi) {
            double *x = outs[mi].x;
            if (x == nullptr) continue;   // coefficients only (two-pass mode)
            if (vdt == SKF_F64)
                k_recombine<<<rgrid, kThreads, 0, st>>>((const double *)V, ldv, n, cm[mi].z, iscal, x);
            else if (vdt == SKF_F32)
                k_recombine_lp<float><<<rgrid, kThreads, zsm, st>>>((const float *)V, ldv, n, cm[mi].z, iscal, x);
            else
                k_recombine_lp<__nv_bfloat16><<<rgrid, kThreads, zsm, st>>>((const __nv_bfloat16 *)V, ldv, n,
                                                                            cm[mi].z, iscal, x);
            ++nlaunch;
        }
    }
    for (int mi = 0; mi < nout; ++mi) {
        k_write_info<<<1, 32, 0, st>>>(cm[mi], outs[mi].info, stop_state);
        ++nlaunch;
    }
    count_launches(nlaunch);
    cudaError_t e = cudaGetLastError();
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "tail kernels");
    return SKF_OK;
}

skf_status tail_run(skf_method method, int s, int m, int64_t n, const void *V, skf_dtype vdt, int64_t ldv,
                    const double *vscale, const double *SV, const double *SAV, int *iscal, const RuleDev &rule,
                    double tol, double *x, skf_info *info, cudaStream_t st, double *sketch_out,
                    const double *stop_state, double *z_out, double cond_max, const double *H, int ldh, int kt) {
    TailOut o{method, x, info, z_out, iscal};
    return tail_run_multi(1, &o, s, m, n, V, vdt, ldv, vscale, SV, SAV, rule, tol, st, sketch_out, stop_state,
                          cond_max, H, ldh, kt);
}

skf_status stop_check(skf_method method, int s, int p, const double *vscale, const double *SV, const double *SAV,
                      int *iscal, int *iscal_chk, double *sf_prev, double *sf_cur, double *state, const RuleDev &rule,
                      double tol_quad, double stop_tol, cudaStream_t st) {
    k_check_begin<<<1, 32, 0, st>>>(iscal, iscal_chk, p);
    count_launches(1);
    skf_status e = tail_run(method, s, p, 0, nullptr, SKF_F64, 0, vscale, SV, SAV, iscal_chk, rule, tol_quad, nullptr,
                            nullptr, st, sf_cur, nullptr);
    if (e != SKF_OK) return e;
    k_check_end<<<1, kThreads, 0, st>>>(SV, s, p, iscal, iscal_chk, sf_prev, sf_cur, state, stop_tol);
    count_launches(1);
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "stopping-criterion kernels");
    return SKF_OK;
}

skf_status accumulate_column(const void *w, skf_dtype vdt, const double *z, const int *iscal, int j, int64_t n,
                             double *x, cudaStream_t st) {
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads,
                                                                          16ll * num_sms()));
    if (vdt == SKF_F64) k_accum<double><<<grid, kThreads, 0, st>>>((const double *)w, z, iscal, j, n, x);
    else if (vdt == SKF_F32) k_accum<float><<<grid, kThreads, 0, st>>>((const float *)w, z, iscal, j, n, x);
    else k_accum<__nv_bfloat16><<<grid, kThreads, 0, st>>>((const __nv_bfloat16 *)w, z, iscal, j, n, x);
    count_launches(1);
    return SKF_OK;
}

}  // namespace skf
