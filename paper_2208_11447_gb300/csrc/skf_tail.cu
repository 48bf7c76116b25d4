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
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

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
    double *B, *C;     // m x m, ld m (lower triangles used)
    double *cvec, *Mtc;  // [m]
    double *Nw;        // node workspace [batch][m*m]
    double *out;       // [batch][m] weighted node solutions
    double *qbuf;      // [levels][m]
    double *qacc;      // [m]
    double *z;         // [m] coefficients for V (scaled by vscale)
    double *qstate;    // [0] converged, [1] ell, [2] quad_err, [3] rdiag_ratio
    const double *t, *w;      // node table
    int nlevels;
};

namespace {

__global__ void k_tail_copy(const double *__restrict__ SV, const double *__restrict__ SAV, TailCtx c) {
    const int me = c.iscal[1];
    const int64_t tot = (int64_t)c.s * 2 * c.m;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(idx / c.s);
        const int64_t r = idx % c.s;
        double v = 0.0;
        if (col < me) v = SV[r + (int64_t)col * c.s];
        else if (col < 2 * me) v = SAV[r + (int64_t)(col - me) * c.s];
        c.Aw[idx] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) c.qstate[threadIdx.x] = 0.0;
}

// Householder reflector for column jj, applied to the trailing columns.
// Every CTA forms the reflector; trailing column cc belongs to CTA
// (cc - jj - 1) mod G.  Column jj itself is not modified (its diagonal goes
// to Rdiag), so no CTA reads data another CTA writes in this launch.
__global__ void __launch_bounds__(kThreads) k_householder(TailCtx c, int jj) {
    __shared__ double red[64];
    const int me = c.iscal[1];
    const int ncols = 2 * me;
    const int nref = (c.method == SKF_METHOD_SGMRES) ? 2 * me : me;
    if (jj >= nref || jj >= c.s) return;
    const double *x = c.Aw + (int64_t)jj * c.s;
    double acc[1] = {0.0};
    for (int i = jj + 1 + threadIdx.x; i < c.s; i += kThreads) acc[0] = fma(x[i], x[i], acc[0]);
    block_sum<1>(acc, red);
    __shared__ double sp[3];
    if (threadIdx.x == 0) {
        const double x0 = x[jj];
        const double sig = acc[0];
        double tau = 0.0, beta = x0, scale = 0.0;
        if (sig > 0.0 || x0 == 0.0) {
            const double nx = sqrt(x0 * x0 + sig);
            beta = (x0 >= 0.0) ? -nx : nx;
            if (nx > 0.0) {
                tau = (beta - x0) / beta;
                scale = 1.0 / (x0 - beta);
            }
        }
        sp[0] = tau;
        sp[1] = beta;
        sp[2] = scale;
        if (blockIdx.x == 0) c.Rdiag[jj] = beta;
    }
    __syncthreads();
    const double tau = sp[0], scale = sp[2];
    if (tau == 0.0) return;
    for (int cc = jj + 1 + blockIdx.x; cc < ncols; cc += gridDim.x) {
        double *y = c.Aw + (int64_t)cc * c.s;
        double d[1] = {0.0};
        for (int i = jj + threadIdx.x; i < c.s; i += kThreads) {
            const double vi = (i == jj) ? 1.0 : x[i] * scale;
            d[0] = fma(vi, y[i], d[0]);
        }
        block_sum<1>(d, red);
        const double f = tau * d[0];
        for (int i = jj + threadIdx.x; i < c.s; i += kThreads) {
            const double vi = (i == jj) ? 1.0 : x[i] * scale;
            y[i] = fma(-f, vi, y[i]);
        }
        __syncthreads();
    }
}

// Rows of X R = T for T = R12 (-> M) and T = R22 (-> R2); one warp per row.
__global__ void __launch_bounds__(kThreads) k_tri_right(TailCtx c) {
    extern __shared__ double xs[];   // [warps][m]
    const int me = c.iscal[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (kThreads / 32) + warp;
    const int nrows = (c.method == SKF_METHOD_SGMRES) ? 2 * me : me;
    if (row >= nrows) return;
    double *x = xs + (size_t)warp * c.m;
    const bool second = row >= me;
    const int a = second ? row - me : row;
    for (int jcol = 0; jcol < me; ++jcol) {
        double part = 0.0;
        for (int i = lane; i < jcol; i += 32) part = fma(x[i], c.Aw[i + (int64_t)jcol * c.s], part);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) {
            double tv;
            if (!second) tv = c.Aw[a + (int64_t)(me + jcol) * c.s];
            else if (jcol < a) tv = 0.0;
            else if (jcol == a) tv = c.Rdiag[me + a];
            else tv = c.Aw[(me + a) + (int64_t)(me + jcol) * c.s];
            x[jcol] = (tv - part) / c.Rdiag[jcol];
        }
        __syncwarp();
    }
    double *dst = second ? c.R2 : c.M;
    for (int jcol = lane; jcol < me; jcol += 32) dst[a + (int64_t)jcol * c.m] = x[jcol];
}

// B = M + M^T, C = M^T M (+ R2^T R2), c = ||b|| R_11 e_1, M^T c.
__global__ void __launch_bounds__(kThreads) k_tail_prep(TailCtx c) {
    const int me = c.iscal[1];
    const int64_t tot = (int64_t)me * me;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % me), j = (int)(idx / me);
        if (j > i) continue;
        double acc = 0.0;
        for (int a = 0; a < me; ++a) acc = fma(c.M[a + (int64_t)i * c.m], c.M[a + (int64_t)j * c.m], acc);
        if (c.method == SKF_METHOD_SGMRES)
            for (int a = 0; a <= j; ++a) acc = fma(c.R2[a + (int64_t)i * c.m], c.R2[a + (int64_t)j * c.m], acc);
        c.C[i + (int64_t)j * c.m] = acc;
        c.B[i + (int64_t)j * c.m] = c.M[i + (int64_t)j * c.m] + c.M[j + (int64_t)i * c.m];
    }
    if (blockIdx.x == 0) {
        const double c0 = (1.0 / c.vscale[0]) * c.Rdiag[0];
        for (int j = threadIdx.x; j < me; j += blockDim.x) {
            c.cvec[j] = (j == 0) ? c0 : 0.0;
            c.Mtc[j] = c0 * c.M[(int64_t)j * c.m];
        }
    }
}

// Cholesky solve L L^T y = y in place (L in the lower triangle of N, ld m).
__device__ void chol_solve(const double *N, int me, int ld, double *y) {
    for (int p = 0; p < me; ++p) {
        __syncthreads();
        const double yp = y[p] / N[p + (int64_t)p * ld];
        __syncthreads();
        if (threadIdx.x == 0) y[p] = yp;
        for (int i = p + 1 + threadIdx.x; i < me; i += blockDim.x) y[i] = fma(-N[i + (int64_t)p * ld], yp, y[i]);
    }
    for (int p = me - 1; p >= 0; --p) {
        __syncthreads();
        const double yp = y[p] / N[p + (int64_t)p * ld];
        __syncthreads();
        if (threadIdx.x == 0) y[p] = yp;
        for (int i = threadIdx.x; i < p; i += blockDim.x) y[i] = fma(-N[p + (int64_t)i * ld], yp, y[i]);
    }
    __syncthreads();
}

// One CTA per quadrature node: node n0 + off + blockIdx.x of the table,
// result row off + blockIdx.x of `out`, workspace slot blockIdx.x.
__global__ void __launch_bounds__(kThreads) k_nodes(TailCtx c, int n0, int off) {
    extern __shared__ double sm[];   // y[m], r[m], g[m], colp[m]
    const int me = c.iscal[1];
    if (c.qstate[0] != 0.0 || me == 0) return;
    const int m = c.m;
    double *y = sm, *r = sm + m, *g = sm + 2 * m, *colp = sm + 3 * m;
    const int nd = n0 + off + blockIdx.x;
    const double t = c.t[nd], wt = c.w[nd];
    double *outrow = c.out + (size_t)(off + blockIdx.x) * c.m;
    double *N = c.Nw + (size_t)blockIdx.x * m * m;
    const bool gm = c.method == SKF_METHOD_SGMRES;
    // N(t) = t^2 I + t (M + M^T) + C, lower triangle
    for (int64_t idx = threadIdx.x; idx < (int64_t)me * me; idx += blockDim.x) {
        const int i = (int)(idx % me), j = (int)(idx / me);
        if (j > i) continue;
        N[i + (int64_t)j * m] = (i == j ? t * t : 0.0) + t * c.B[i + (int64_t)j * m] + c.C[i + (int64_t)j * m];
    }
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    // right-looking Cholesky
    for (int p = 0; p < me; ++p) {
        __syncthreads();
        const double d = N[p + (int64_t)p * m];
        if (!(d > 0.0)) {
            if (threadIdx.x == 0) bad = 1;
            break;
        }
        const double lpp = sqrt(d);
        for (int i = p + threadIdx.x; i < me; i += blockDim.x) {
            const double v = (i == p) ? lpp : N[i + (int64_t)p * m] / lpp;
            colp[i] = v;
        }
        __syncthreads();
        for (int i = p + threadIdx.x; i < me; i += blockDim.x) N[i + (int64_t)p * m] = colp[i];
        for (int i = p + 1 + threadIdx.x; i < me; i += blockDim.x) {
            const double lip = colp[i];
            for (int q = p + 1; q <= i; ++q) N[i + (int64_t)q * m] = fma(-lip, colp[q], N[i + (int64_t)q * m]);
        }
    }
    __syncthreads();
    if (bad) {
        for (int a = threadIdx.x; a < me; a += blockDim.x) outrow[a] = 0.0;
        if (threadIdx.x == 0) atomicExch(&c.iscal[2], gm ? (int)SKF_ERR_ILL_CONDITIONED : (int)SKF_ERR_BRANCH_CUT);
        return;
    }
    // y = N^{-1} (t c + M^T c)
    for (int a = threadIdx.x; a < me; a += blockDim.x) y[a] = t * c.cvec[a] + c.Mtc[a];
    chol_solve(N, me, m, y);
    // one refinement step on the original residual
    for (int a = threadIdx.x; a < me; a += blockDim.x) {
        double v = c.cvec[a] - t * y[a];
        for (int j = 0; j < me; ++j) v = fma(-c.M[a + (int64_t)j * m], y[j], v);
        r[a] = v;
    }
    if (gm) {
        for (int a = threadIdx.x; a < me; a += blockDim.x) {
            double v = 0.0;
            for (int j = a; j < me; ++j) v = fma(-c.R2[a + (int64_t)j * m], y[j], v);
            colp[a] = v;   // bottom residual
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < me; j += blockDim.x) {
        double v = t * r[j];
        for (int a = 0; a < me; ++a) v = fma(c.M[a + (int64_t)j * m], r[a], v);
        if (gm)
            for (int a = 0; a <= j; ++a) v = fma(c.R2[a + (int64_t)j * m], colp[a], v);
        g[j] = v;
    }
    chol_solve(N, me, m, g);
    for (int a = threadIdx.x; a < me; a += blockDim.x) outrow[a] = wt * (y[a] + g[a]);
}

// Sum the node solutions of each level of the batch, then run the
// acceptance test of Sec. 4.1 level by level.  One CTA.
__global__ void __launch_bounds__(kThreads) k_levels(TailCtx c, int lev0, int nlev, const int *lev_start,
                                                     const int *lev_ell, int n0, double tol, int last_batch) {
    __shared__ double red[64];
    const int me = c.iscal[1];
    if (c.qstate[0] != 0.0 || me == 0) return;
    const int m = c.m;
    for (int l = lev0; l < lev0 + nlev; ++l) {
        const int a0 = lev_start[l] - n0, a1 = lev_start[l + 1] - n0;
        double *ql = c.qbuf + (size_t)l * m;
        for (int a = threadIdx.x; a < me; a += blockDim.x) {
            double acc = 0.0;
            for (int nd = a0; nd < a1; ++nd) acc += c.out[(size_t)nd * m + a];
            ql[a] = acc;
        }
        __syncthreads();
        bool accept = false;
        double rel = 0.0;
        if (c.nlevels == 1) {
            accept = true;
        } else if (l > 0) {
            const double *qp = c.qbuf + (size_t)(l - 1) * m;
            double v[2] = {0.0, 0.0};
            for (int a = threadIdx.x; a < me; a += blockDim.x) {
                const double d = ql[a] - qp[a];
                v[0] = fma(d, d, v[0]);
                v[1] = fma(ql[a], ql[a], v[1]);
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
            for (int a = threadIdx.x; a < me; a += blockDim.x) c.qacc[a] = ql[a];
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

// y = R^{-1} q_acc, z = vscale .* y (single CTA, column-oriented back substitution).
__global__ void __launch_bounds__(kThreads) k_coeffs(TailCtx c) {
    extern __shared__ double q[];
    __shared__ double red[64];
    const int me = c.iscal[1];
    for (int a = threadIdx.x; a < me; a += blockDim.x) q[a] = c.qacc[a];
    for (int p = me - 1; p >= 0; --p) {
        __syncthreads();
        const double yp = q[p] / c.Rdiag[p];
        __syncthreads();
        if (threadIdx.x == 0) q[p] = yp;
        for (int i = threadIdx.x; i < p; i += blockDim.x) q[i] = fma(-c.Aw[i + (int64_t)p * c.s], yp, q[i]);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < me; a += blockDim.x) c.z[a] = c.vscale[a] * q[a];
    // min |R_jj| / max |R_jj| over the whitening factor
    double mn = INFINITY, mx = 0.0;
    for (int a = threadIdx.x; a < me; a += blockDim.x) {
        mn = fmin(mn, fabs(c.Rdiag[a]));
        mx = fmax(mx, fabs(c.Rdiag[a]));
    }
    mx = block_max(mx, red);
    mn = -block_max(-mn, red);
    if (threadIdx.x == 0) {
        c.qstate[3] = mx > 0.0 ? mn / mx : 0.0;
        if (!(mn > 0.0) && me > 0 && c.iscal[2] == SKF_OK) c.iscal[2] = SKF_ERR_ILL_CONDITIONED;
    }
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

__global__ void k_write_info(TailCtx c, skf_info *info) {
    if (threadIdx.x != 0 || info == nullptr) return;
    info->status = c.iscal[2];
    info->m_eff = c.iscal[1];
    info->ell = (int)c.qstate[1];
    info->quad_err = c.qstate[2];
    info->rdiag_ratio = c.qstate[3];
}

}  // namespace

// Host driver of the tail.  `rule` holds all levels of the adaptive
// schedule; levels are evaluated in batches (speculatively, several levels per
// launch) and accepted in schedule order, which gives the same accepted order
// as evaluating one level at a time.
skf_status tail_run(skf_method method, int s, int m, int64_t n, const double *V, int64_t ldv, const double *vscale,
                    const double *SV, const double *SAV, int *iscal, const RuleDev &rule, double tol, double *x,
                    skf_info *info, cudaStream_t st) {
    TailCtx c{};
    c.s = s;
    c.m = m;
    c.method = method;
    c.iscal = iscal;
    c.vscale = vscale;
    c.t = rule.t;
    c.w = rule.w;
    c.nlevels = rule.nlevels;
    int max_level = 0;
    for (int l = 0; l < rule.nlevels; ++l) max_level = std::max(max_level, rule.h_start[l + 1] - rule.h_start[l]);
    const int cap = std::max(2 * num_sms(), max_level);
    // batches of consecutive levels with at most `cap` nodes (a level never splits)
    std::vector<std::pair<int, int>> batches;   // (first level, count)
    for (int l = 0; l < rule.nlevels;) {
        int cnt = 0, nodes = 0;
        while (l + cnt < rule.nlevels) {
            const int sz = rule.h_start[l + cnt + 1] - rule.h_start[l + cnt];
            if (cnt > 0 && nodes + sz > cap) break;
            nodes += sz;
            ++cnt;
        }
        batches.push_back({l, cnt});
        l += cnt;
    }
    const int chunk = 2 * num_sms();
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t mm = (size_t)m * m;
    const size_t sizes[] = {sizeof(double) * (size_t)s * 2 * m, sizeof(double) * 2 * m, sizeof(double) * mm,
                            sizeof(double) * mm, sizeof(double) * mm, sizeof(double) * mm, sizeof(double) * m,
                            sizeof(double) * m, sizeof(double) * chunk * mm, sizeof(double) * (size_t)cap * m,
                            sizeof(double) * (size_t)rule.nlevels * m, sizeof(double) * m, sizeof(double) * m,
                            sizeof(double) * 4};
    size_t total = 0;
    for (size_t v : sizes) total += al(v);
    char *ws = nullptr;
    skf_status stt = dalloc((void **)&ws, total, st);
    if (stt != SKF_OK) return stt;
    double *ptrs[14];
    size_t off = 0;
    for (int i = 0; i < 14; ++i) {
        ptrs[i] = (double *)(ws + off);
        off += al(sizes[i]);
    }
    c.Aw = ptrs[0]; c.Rdiag = ptrs[1]; c.M = ptrs[2]; c.R2 = ptrs[3]; c.B = ptrs[4]; c.C = ptrs[5];
    c.cvec = ptrs[6]; c.Mtc = ptrs[7]; c.Nw = ptrs[8]; c.out = ptrs[9]; c.qbuf = ptrs[10]; c.qacc = ptrs[11];
    c.z = ptrs[12]; c.qstate = ptrs[13];

    const int G = std::min(2 * num_sms(), 1024);
    k_tail_copy<<<G, kThreads, 0, st>>>(SV, SAV, c);
    const int hhG = std::max(1, std::min(num_sms(), 2 * m));
    const int nref = (method == SKF_METHOD_SGMRES) ? 2 * m : m;
    for (int jj = 0; jj < nref; ++jj) k_householder<<<hhG, kThreads, 0, st>>>(c, jj);
    {
        const int rows = (method == SKF_METHOD_SGMRES) ? 2 * m : m;
        const int blocks = (rows + (kThreads / 32) - 1) / (kThreads / 32);
        const size_t smem = sizeof(double) * (kThreads / 32) * m;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_tri_right, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tri_right<<<blocks, kThreads, smem, st>>>(c);
    }
    k_tail_prep<<<G, kThreads, 0, st>>>(c);
    const size_t nsmem = sizeof(double) * 4 * m;
    if (nsmem > 48 * 1024) cudaFuncSetAttribute(k_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsmem);
    for (size_t bi = 0; bi < batches.size(); ++bi) {
        const int l0 = batches[bi].first, nl = batches[bi].second;
        const int n0 = rule.h_start[l0];
        const int nn = rule.h_start[l0 + nl] - n0;
        for (int o = 0; o < nn; o += chunk) k_nodes<<<std::min(chunk, nn - o), kThreads, nsmem, st>>>(c, n0, o);
        k_levels<<<1, kThreads, 0, st>>>(c, l0, nl, rule.lev_start, rule.lev_ell, n0, tol,
                                         bi + 1 == batches.size() ? 1 : 0);
    }
    const size_t qsm = sizeof(double) * m;
    if (qsm > 48 * 1024) cudaFuncSetAttribute(k_coeffs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm);
    k_coeffs<<<1, kThreads, qsm, st>>>(c);
    const int64_t rb = std::min<int64_t>((n + kThreads - 1) / kThreads, 16 * num_sms());
    k_recombine<<<(unsigned)std::max<int64_t>(rb, 1), kThreads, 0, st>>>(V, ldv, n, c.z, iscal, x);
    k_write_info<<<1, 32, 0, st>>>(c, info);
    cudaError_t e = cudaGetLastError();
    dfree(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "tail kernels");
    return SKF_OK;
}

}  // namespace skf
