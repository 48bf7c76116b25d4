// C ABI entry points (include/skf.h): argument validation, handles, the
// quadrature-rule cache and the orchestration of the device pipelines.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "skf_internal.cuh"

namespace skf {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
skf_status fail(skf_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}
skf_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return SKF_ERR_OOM;
    return SKF_ERR_CUDA;
}

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int num_sms() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            cached = v;
        else
            return 1;
    }
    return cached;
}

// Stream-ordered workspace comes from a memory pool owned by the library, one
// per device, whose release threshold keeps freed blocks mapped across
// synchronisations: the workspace of one solve (mostly the m basis columns,
// 8 m N bytes in FP64) is then taken over by the next solve instead of being
// mapped again.  skf_workspace_trim returns the cached blocks.  Allocations
// made while the stream is being captured into a graph use the graph's own
// memory nodes (cudaMallocAsync) instead.
static std::mutex &pool_mutex() {
    static std::mutex *mu = new std::mutex();
    return *mu;
}

static std::map<int, cudaMemPool_t> &pools() {
    static std::map<int, cudaMemPool_t> *p = new std::map<int, cudaMemPool_t>();
    return *p;
}

static cudaMemPool_t workspace_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(pool_mutex());
    auto it = pools().find(dev);
    if (it != pools().end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
    } else {
        uint64_t keep = ~(uint64_t)0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pools()[dev] = pool;
    return pool;
}

skf_status dalloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    cudaMemPool_t pool = cap == cudaStreamCaptureStatusNone ? workspace_pool() : nullptr;
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_fail(e, "stream-ordered allocation");
    }
    return SKF_OK;
}
void dfree(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// ------------------------------------------------------- quadrature rules
// Gauss-Legendre nodes by Newton's method on theta with x = cos(theta), so
// that 1 + x = 2 cos^2(theta/2) and 1 - x = 2 sin^2(theta/2) are accurate near
// the end points; the weights are 2 / (sin^2 theta P_n'(x)^2).
static void gauss_legendre_theta(int n, std::vector<double> &theta, std::vector<double> &omega) {
    theta.resize(n);
    omega.resize(n);
    for (int i = 0; i < n; ++i) {
        double th = M_PI * (i + 0.75) / (n + 0.5);
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            const double x = cos(th), st = sin(th);
            double p0 = 1.0, p1 = x;
            for (int kk = 2; kk <= n; ++kk) {
                const double p2 = ((2.0 * kk - 1.0) * x * p1 - (kk - 1.0) * p0) / kk;
                p0 = p1;
                p1 = p2;
            }
            const double pn = (n == 0) ? 1.0 : (n == 1 ? x : p1);
            const double pm = (n == 1) ? 1.0 : p0;
            // d/dtheta P_n(cos theta) = n (x P_n - P_{n-1}) / sin(theta)
            dp = n * (x * pn - pm) / st;
            const double step = pn / dp;
            th -= step;
            if (fabs(step) < 1e-16 * (1.0 + fabs(th))) break;
        }
        theta[i] = th;
        omega[i] = 2.0 / (dp * dp);   // = 2 / (sin^2 P_n'^2)
    }
}

// Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b (a, b > -1): the nodes
// are the eigenvalues of the symmetric tridiagonal Jacobi matrix of the
// orthonormal recurrence (Golub-Welsch), each found by bisection on Sturm
// counts (negative pivots of T - lambda I = L D L^T); the weights are
// mu_0 times the squared first component of the normalised eigenvector,
// obtained by inverse iteration at the computed eigenvalue.  The diagonal
// entry k = 0 and the off-diagonal entry k = 1 are used in their cancelled
// forms, so a + b = -1 (the z^-alpha weight) is well defined.  Returns false
// unless the nodes are distinct and ordered and the weights add up to mu_0.
static bool gauss_jacobi(int n, double a, double b, std::vector<double> &x, std::vector<double> &omega) {
    if (n < 1 || !(a > -1.0) || !(b > -1.0)) return false;
    const double ab = a + b;
    std::vector<double> dg(n), of2(n, 0.0);
    dg[0] = (b - a) / (ab + 2.0);
    for (int k = 1; k < n; ++k) dg[k] = (b * b - a * a) / ((2.0 * k + ab) * (2.0 * k + ab + 2.0));
    if (n > 1) of2[1] = 4.0 * (1.0 + a) * (1.0 + b) / ((2.0 + ab) * (2.0 + ab) * (3.0 + ab));
    for (int k = 2; k < n; ++k) {
        const double k2 = 2.0 * k + ab;
        of2[k] = 4.0 * k * (k + a) * (k + b) * (k + ab) / (k2 * k2 * (k2 + 1.0) * (k2 - 1.0));
    }
    auto below = [&](double lam) {
        int cnt = 0;
        double d = 1.0;
        for (int k = 0; k < n; ++k) {
            d = (dg[k] - lam) - (k > 0 ? of2[k] / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++cnt;
        }
        return cnt;
    };
    const double mu0 = pow(2.0, ab + 1.0) * tgamma(a + 1.0) * tgamma(b + 1.0) / tgamma(ab + 2.0);
    std::vector<double> of(n, 0.0), v(n), dd(n), ll(n);
    for (int k = 1; k < n; ++k) of[k] = sqrt(of2[k]);
    x.assign(n, 0.0);
    omega.assign(n, 0.0);
    double sum = 0.0;
    for (int k = 0; k < n; ++k) {
        double lo = -1.0, hi = 1.0;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            if (below(mid) > k) hi = mid;
            else lo = mid;
        }
        const double xk = 0.5 * (lo + hi);
        // normalised eigenvector by two steps of inverse iteration on the
        // tridiagonal T - x I (elimination without pivoting; a zero pivot is
        // replaced by a tiny one, which only sharpens the iteration)
        for (int j = 0; j < n; ++j) v[j] = 1.0;
        for (int it = 0; it < 2; ++it) {
            double piv = dg[0] - xk;
            if (piv == 0.0) piv = 1e-300;
            dd[0] = piv;
            for (int j = 1; j < n; ++j) {
                const double l = of[j] / dd[j - 1];
                ll[j] = l;
                piv = (dg[j] - xk) - l * of[j];
                if (piv == 0.0) piv = 1e-300;
                dd[j] = piv;
                v[j] -= l * v[j - 1];
            }
            v[n - 1] /= dd[n - 1];
            for (int j = n - 2; j >= 0; --j) v[j] = (v[j] - of[j + 1] * v[j + 1]) / dd[j];
            double mx = 0.0;
            for (int j = 0; j < n; ++j) mx = std::max(mx, fabs(v[j]));
            for (int j = 0; j < n; ++j) v[j] /= mx;
        }
        double ss = 0.0;
        for (int j = 0; j < n; ++j) ss += v[j] * v[j];
        x[k] = xk;
        omega[k] = mu0 * v[0] * v[0] / ss;
        sum += omega[k];
        if (!(xk > -1.0 && xk < 1.0) || (k > 0 && !(xk > x[k - 1]))) return false;
    }
    return fabs(sum - mu0) <= 1e-11 * mu0;
}

// Contour rule for f(z) = exp(-z) on the parabola t(zeta) = a - c zeta^2 +
// i zeta (a = f.alpha, c = f.scale): trapezoidal rule in zeta on [0, L],
// c L^2 = 37, step h = L / (ell - 1), weights of zeta > 0 doubled (the
// conjugate half of the contour): w = h e^t (i - 2 c zeta) / (2 pi i).
static bool contour_rule(const skf_func &f, int ell, double *tr, double *ti, double *wr, double *wi) {
    if (f.kind != SKF_FUNC_EXP_NEG || ell < 2 || !(f.scale > 0.0)) return false;
    const double c = f.scale, a = f.alpha;
    const double L = sqrt(37.0 / c), h = L / (ell - 1);
    for (int k = 0; k < ell; ++k) {
        const double z = k * h;
        const double mag = (k == 0 ? 1.0 : 2.0) * h * exp(a - c * z * z) / (2.0 * M_PI);
        const double cs = cos(z), sn = sin(z);
        tr[k] = a - c * z * z;
        ti[k] = z;
        wr[k] = mag * (cs - 2.0 * c * z * sn);
        wi[k] = mag * (sn + 2.0 * c * z * cs);
    }
    return true;
}

bool quadrature_rule(const skf_func &f, int ell, double *t, double *w) {
    if (f.kind == SKF_FUNC_INV) {
        t[0] = 0.0;
        w[0] = 1.0;
        return true;
    }
    if (f.kind == SKF_FUNC_CUSTOM) return f.rule != nullptr && f.rule(ell, t, w, f.ctx) == 0;
    const double c = f.scale;
    if (f.kind == SKF_FUNC_INVPOW && f.alpha != 0.5) {
        // z^-alpha = (sin(alpha pi)/pi) int t^-alpha (t+z)^-1 dt with t = c (1-x)/(1+x):
        // Gauss-Jacobi(-alpha, alpha-1) in x, w = (sin(alpha pi)/pi) 2 c^(1-alpha) omega / (1+x)
        if (!(f.alpha > 0.0 && f.alpha < 1.0)) return false;
        std::vector<double> xs, om;
        if (!gauss_jacobi(ell, -f.alpha, f.alpha - 1.0, xs, om)) return false;
        const double k = sin(f.alpha * M_PI) / M_PI * 2.0 * pow(c, 1.0 - f.alpha);
        for (int i = 0; i < ell; ++i) {
            t[i] = c * (1.0 - xs[i]) / (1.0 + xs[i]);
            w[i] = k * om[i] / (1.0 + xs[i]);
        }
        return true;
    }
    if (f.kind == SKF_FUNC_INVSQRT || (f.kind == SKF_FUNC_INVPOW && f.alpha == 0.5)) {
        // Gauss-Chebyshev: theta_i = (2i-1) pi / (2 ell), omega_i = pi / ell;
        // t = c tan^2(theta/2), w = 2 sqrt(c) / (ell (1 + x)).
        for (int i = 0; i < ell; ++i) {
            const double th = (2.0 * i + 1.0) * M_PI / (2.0 * ell);
            const double ch = cos(0.5 * th), sh = sin(0.5 * th);
            t[i] = c * (sh * sh) / (ch * ch);
            w[i] = sqrt(c) / (ell * ch * ch);
        }
        return true;
    }
    if (f.kind == SKF_FUNC_LOG1P_OVER_Z) {
        std::vector<double> th, om;
        gauss_legendre_theta(ell, th, om);
        for (int i = 0; i < ell; ++i) {
            const double ch = cos(0.5 * th[i]), sh = sin(0.5 * th[i]);
            t[i] = 1.0 + c * (sh * sh) / (ch * ch);
            // w = 2 c omega / ((1 + x)^2 t), 1 + x = 2 cos^2(theta/2)
            w[i] = c * om[i] / (2.0 * ch * ch * ch * ch * t[i]);
        }
        return true;
    }
    return false;
}

// Device copies of the adaptive schedule, cached per (f, schedule).
struct RuleCache {
    std::mutex mu;
    std::map<std::string, RuleDev *> tables;
};
static RuleCache &rule_cache() {
    static RuleCache *rc = new RuleCache();
    return *rc;
}

static skf_status get_rule(const skf_func &f, const skf_params &p, const RuleDev **out) {
    char key[256];
    snprintf(key, sizeof key, "%d|%.17g|%.17g|%d|%d|%d|%d|%p|%p", (int)f.kind, f.alpha, f.scale, p.ell1, p.ell2,
             p.ell_max, f.n_nodes, f.kind == SKF_FUNC_CUSTOM ? (void *)f.rule : nullptr,
             f.kind == SKF_FUNC_CUSTOM ? f.ctx : nullptr);
    std::string k(key);
    if (f.n_nodes > 0) {
        for (int i = 0; i < f.n_nodes; ++i) {
            char b[64];
            snprintf(b, sizeof b, "|%a|%a", f.nodes[i], f.weights[i]);
            k += b;
        }
    }
    RuleCache &rc = rule_cache();
    std::lock_guard<std::mutex> lk(rc.mu);
    auto it = rc.tables.find(k);
    if (it != rc.tables.end()) {
        *out = it->second;
        return SKF_OK;
    }
    std::vector<int> ells;
    if (f.n_nodes > 0) {
        ells.push_back(f.n_nodes);
    } else if (f.kind == SKF_FUNC_INV) {
        ells.push_back(1);
    } else {
        ells.push_back(p.ell1);
        ells.push_back(p.ell2);
        while (true) {
            const int nx = (int)floor(sqrt(2.0) * ells.back());
            if (nx > p.ell_max) break;
            ells.push_back(nx);
        }
    }
    std::vector<double> ht, hw, hti, hwi;
    std::vector<int> hs{0};
    const bool cplx = f.n_nodes == 0 && f.kind == SKF_FUNC_EXP_NEG;
    for (int ell : ells) {
        const size_t o = ht.size();
        ht.resize(o + ell);
        hw.resize(o + ell);
        hti.resize(o + ell);
        hwi.resize(o + ell);
        if (f.n_nodes > 0) {
            std::copy(f.nodes, f.nodes + ell, ht.begin() + o);
            std::copy(f.weights, f.weights + ell, hw.begin() + o);
        } else if (cplx) {
            if (!contour_rule(f, ell, ht.data() + o, hti.data() + o, hw.data() + o, hwi.data() + o))
                return fail(SKF_ERR_INVALID_ARG, "contour rule needs ell >= 2 and scale > 0");
        } else if (!quadrature_rule(f, ell, ht.data() + o, hw.data() + o)) {
            return fail(SKF_ERR_NOT_SUPPORTED, f.kind == SKF_FUNC_CUSTOM
                                                   ? "the custom rule callback failed for order " + std::to_string(ell)
                                                   : "quadrature rule of order " + std::to_string(ell) +
                                                         " not available for this function");
        }
        hs.push_back((int)ht.size());
    }
    RuleDev *r = new RuleDev();
    r->cplx = cplx;
    if (cplx) {
        if (cudaMalloc(&r->t_im, sizeof(double) * hti.size()) != cudaSuccess ||
            cudaMalloc(&r->w_im, sizeof(double) * hwi.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(SKF_ERR_OOM, "rule table allocation failed");
        }
        if (cudaMemcpy(r->t_im, hti.data(), sizeof(double) * hti.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(r->w_im, hwi.data(), sizeof(double) * hwi.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "rule table upload");
    }
    r->nlevels = (int)ells.size();
    r->h_start = hs;
    r->h_ell = ells;
    if (cudaMalloc(&r->t, sizeof(double) * ht.size()) != cudaSuccess ||
        cudaMalloc(&r->w, sizeof(double) * hw.size()) != cudaSuccess ||
        cudaMalloc(&r->lev_start, sizeof(int) * hs.size()) != cudaSuccess ||
        cudaMalloc(&r->lev_ell, sizeof(int) * ells.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(SKF_ERR_OOM, "rule table allocation failed");
    }
    if (cudaMemcpy(r->t, ht.data(), sizeof(double) * ht.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(r->w, hw.data(), sizeof(double) * hw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(r->lev_start, hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(r->lev_ell, ells.data(), sizeof(int) * ells.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "rule table upload");
    rc.tables[k] = r;
    *out = r;
    return SKF_OK;
}

namespace {

__global__ void k_rowptr32(const int64_t *__restrict__ in, int64_t n, int32_t *__restrict__ out, int *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = in[i];
        out[i] = (int32_t)v;
        if (v < 0 || (i > 0 && in[i - 1] > v)) atomicExch(bad, 1);
    }
}

template <typename TV>
__global__ void k_row_abs_sum(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const TV *__restrict__ v,
                              int64_t n, int *bad, unsigned long long *maxbits) {
    double mx = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int p = rp[r]; p < rp[r + 1]; ++p) {
            acc += fabs((double)v[p]);
            if (ci[p] < 0 || ci[p] >= n) atomicExch(bad, 1);
        }
        mx = fmax(mx, acc);
    }
    // non-negative doubles order like their bit patterns
    atomicMax(maxbits, (unsigned long long)__double_as_longlong(mx));
}

// SELL-32 entries (see skf_csr); rows longer than `cut` entries are left
// empty (they take the row-split path).
template <typename TV>
__global__ void k_sell_fill(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const TV *__restrict__ v,
                            int64_t n, int64_t nslices, int cut, const int32_t *__restrict__ perm,
                            const int64_t *__restrict__ off, const int32_t *__restrict__ w, TV *__restrict__ sv,
                            int32_t *__restrict__ sc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 32 * nslices;
         i += (int64_t)gridDim.x * blockDim.x) {   // slot i: row perm[i]
        const int64_t t = i >> 5;
        const int l = (int)(i & 31);
        const int wt = w[t];
        const int64_t r = i < n ? (perm ? (int64_t)perm[i] : i) : n;
        const int b = r < n ? rp[r] : 0;
        int len = r < n ? rp[r + 1] - b : 0;
        if (len > cut) len = 0;   // a long row: row-split path
        const int self = r < n ? (int)r : 0;
        for (int p = 0; p < wt; ++p) {
            const int64_t o = off[t] + 32ll * p + l;
            sv[o] = p < len ? v[b + p] : (TV)0;
            sc[o] = p < len ? ci[b + p] : self;
        }
    }
}


static skf_status check_common(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype, int m, int k,
                               skf_dtype basis) {
    if (!A || !S || !b) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    if (S->n != A->n) return fail(SKF_ERR_INVALID_ARG, "sketch and matrix sizes differ");
    if (m < 1 || m >= S->s) return fail(SKF_ERR_INVALID_ARG, "need 1 <= m < s");
    if (m > A->n) return fail(SKF_ERR_INVALID_ARG, "need m <= n");
    if (k < 1 || k > kMaxK) return fail(SKF_ERR_INVALID_ARG, "need 1 <= k <= 16");
    if (bdtype != SKF_F64) return fail(SKF_ERR_NOT_SUPPORTED, "b must be F64 in this build");
    if (basis == SKF_F64) {
        if (A->vdtype != SKF_F64) return fail(SKF_ERR_NOT_SUPPORTED, "an F64 basis needs F64 matrix values");
    } else if (basis == SKF_F32 || basis == SKF_BF16) {
        if (A->vdtype != SKF_F32) return fail(SKF_ERR_NOT_SUPPORTED, "an F32 or BF16 basis needs F32 matrix values");
        const bool dense = S->kind == SKF_SKETCH_SRHT || S->kind == SKF_SKETCH_SRDCT;
        if (S->kind != SKF_SKETCH_SPARSE_SIGN && S->kind != SKF_SKETCH_IDENTITY && !(dense && basis == SKF_F32))
            return fail(SKF_ERR_NOT_SUPPORTED, "sketch kind not implemented for this basis type");
    } else {
        return fail(SKF_ERR_INVALID_ARG, "unknown basis dtype");
    }
    return SKF_OK;
}

static size_t dtype_size(skf_dtype d) { return d == SKF_F64 ? 8 : d == SKF_F32 ? 4 : 2; }

static skf_status run_arnoldi(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, skf_dtype basis,
                              void *V, int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                              skf_info *info, cudaStream_t cs, const StepHook *hook = nullptr, int vring = 0) {
    if (basis == SKF_F64)
        return arnoldi_run(A, S, b, m, k, (double *)V, ldv, vscale, SV, SAV, H, iscal, info, cs, hook, vring);
    if (basis == SKF_F32) {
        // the persistent form where it applies (as for FP64: no per-step hooks,
        // one-pass storage), else the two-kernel form
        if (step_mode() != 1 && hook == nullptr && vring == 0) {
            const skf_status ps =
                arnoldi_run_persistent_f32(A, S, b, m, k, (float *)V, ldv, vscale, SV, SAV, H, iscal, info, cs);
            if (ps != SKF_ERR_NOT_SUPPORTED) return ps;
            if (step_mode() == 2) return fail(SKF_ERR_NOT_SUPPORTED, "persistent Arnoldi form does not apply here");
        }
        return arnoldi_run_f32(A, S, b, m, k, (float *)V, ldv, vscale, SV, SAV, H, iscal, info, cs, hook, vring);
    }
    return arnoldi_run_bf16(A, S, b, m, k, V, ldv, vscale, SV, SAV, H, iscal, info, cs, hook, vring);
}

// Checkpoints of the stopping criterion, enqueued from the Arnoldi drivers'
// hook at p = d, 2d, ... < m as soon as the leading p columns are final.
struct StopCtx {
    skf_method method;
    int s, m, d, next_p;
    const double *vscale, *SV, *SAV;
    int *iscal, *iscal_chk;
    double *sf_prev, *sf_cur, *state;
    const RuleDev *rule;
    double tol_quad, stop_tol;
    skf_status err;
};

// Second pass of the two-pass mode: x (+)= z_j w_j as each column appears;
// a stop of the first pass by the criterion is copied to the second pass's
// state right after its start kernel (same columns, same m_eff).
struct AccCtx {
    const void *V;
    skf_dtype vdt;
    int64_t ldv, n;
    int vring;
    const double *z;
    const int *iscal1;
    int *iscal2;
    double *x;
    skf_status err;
};

__global__ void k_copy_stop(const int *__restrict__ iscal1, int *__restrict__ iscal2) {
    if (threadIdx.x == 0 && iscal1[0] == 2) {
        iscal2[0] = 2;
        iscal2[1] = iscal1[1];
        iscal2[3] = iscal1[3];
    }
}

static void acc_hook(void *ctx, int j, cudaStream_t st) {
    AccCtx *a = (AccCtx *)ctx;
    if (a->err != SKF_OK) return;
    if (j == 0) {
        k_copy_stop<<<1, 32, 0, st>>>(a->iscal1, a->iscal2);
        count_launches(1);
    }
    const char *w = (const char *)a->V + (size_t)(j % a->vring) * a->ldv * dtype_size(a->vdt);
    a->err = accumulate_column(w, a->vdt, a->z, a->iscal1, j, a->n, a->x, st);
}

static void stop_hook(void *ctx, int done, cudaStream_t st) {
    StopCtx *k = (StopCtx *)ctx;
    while (k->err == SKF_OK && k->next_p <= done && k->next_p < k->m) {
        const int p = k->next_p;
        k->next_p += k->d;
        k->err = stop_check(k->method, k->s, p, k->vscale, k->SV, k->SAV, k->iscal, k->iscal_chk, k->sf_prev,
                            k->sf_cur, k->state, *k->rule, k->tol_quad, k->stop_tol, st);
    }
}

// ------------------------------------------------------------ solve parts
// Argument validation of one skf_solve call and its quadrature rule (host
// work only; may upload a new rule synchronously).
static skf_status solve_check(skf_method method, const skf_csr *A, const skf_sketch *S, const void *b,
                              skf_dtype bdtype, const skf_func *f, const skf_params *p, const void *x,
                              skf_dtype xdtype, const RuleDev **rule) {
    if (!f || !p || !x) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    skf_status st = check_common(A, S, b, bdtype, p->m, p->k, p->basis_dtype);
    if (st != SKF_OK) return st;
    if (method != SKF_METHOD_SFOM && method != SKF_METHOD_SGMRES) return fail(SKF_ERR_INVALID_ARG, "bad method");
    if (xdtype != SKF_F64) return fail(SKF_ERR_NOT_SUPPORTED, "x must be F64 in this build");
    if (p->m > 512) return fail(SKF_ERR_NOT_SUPPORTED, "m > 512 is not supported by the dense tail");
    if (method == SKF_METHOD_SGMRES && S->s < 2 * p->m)
        return fail(SKF_ERR_SKETCH_TOO_SMALL, "sGMRES needs s >= 2m");
    if (f->n_nodes < 0 || (f->n_nodes > 0 && (!f->nodes || !f->weights)))
        return fail(SKF_ERR_INVALID_ARG, "bad explicit rule");
    if (f->n_nodes == 0 && f->kind != SKF_FUNC_INV) {
        if (!(f->scale > 0.0)) return fail(SKF_ERR_INVALID_ARG, "rule scale must be > 0");
        if (p->ell1 < 1 || p->ell2 <= p->ell1 || p->ell2 < 3 || p->ell_max < p->ell2)
            return fail(SKF_ERR_INVALID_ARG, "need 1 <= ell1 < ell2, ell2 >= 3, ell_max >= ell2");
        if (!(p->tol > 0.0)) return fail(SKF_ERR_INVALID_ARG, "tol must be > 0");
    }
    if (f->kind == SKF_FUNC_INVPOW && f->n_nodes == 0 && !(f->alpha > 0.0 && f->alpha < 1.0))
        return fail(SKF_ERR_INVALID_ARG, "z^-alpha needs 0 < alpha < 1");
    if (f->kind == SKF_FUNC_CUSTOM && f->n_nodes == 0 && f->rule == nullptr)
        return fail(SKF_ERR_INVALID_ARG, "a custom function needs a rule callback or explicit nodes");
    if (f->kind < SKF_FUNC_INVSQRT || f->kind > SKF_FUNC_CUSTOM) return fail(SKF_ERR_INVALID_ARG, "unknown function kind");
    if (f->kind == SKF_FUNC_EXP_NEG) {
        if (f->n_nodes > 0) return fail(SKF_ERR_NOT_SUPPORTED, "explicit rules are real; exp(-z) uses the contour");
        if (p->ell1 < 2) return fail(SKF_ERR_INVALID_ARG, "the contour rule needs ell1 >= 2");
        if (p->m > 256) return fail(SKF_ERR_NOT_SUPPORTED, "complex quadrature nodes need m <= 256");
    }
    if (p->check_every < 0 || !(p->stop_tol >= 0.0))
        return fail(SKF_ERR_INVALID_ARG, "need check_every >= 0 and stop_tol >= 0");
    return get_rule(*f, *p, rule);
}

// Enqueue one validated solve on `cs`: stream-ordered workspace, the
// Arnoldi process, the tail, release of the workspace.
static skf_status solve_enqueue(skf_method method, const skf_csr *A, const skf_sketch *S, const void *b,
                                const skf_params &p, void *x, skf_info *info, const RuleDev &rule, cudaStream_t cs) {
    const int m = p.m;
    const int64_t n = A->n;
    const int s = S->s;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const skf_dtype bt = p.basis_dtype;
    const int64_t ldv = (n + 63) / 64 * 64;   // 256-byte aligned columns
    const bool two = p.two_pass != 0;
    const int vring = two ? std::min(m, p.k + 2) : 0;   // ring slots of the two-pass mode
    const size_t szV = dtype_size(bt) * (size_t)ldv * (two ? vring : m);
    const size_t szS = sizeof(double) * (size_t)s * m;
    const size_t szH = sizeof(double) * (size_t)(m + 1) * m;
    const bool stopping = p.check_every > 0 && p.check_every < m;
    // stopping criterion: iscal_chk[4] | state[4] | sf_prev[s] | sf_cur[s]
    const size_t szStop = stopping ? al(sizeof(int) * 4) + al(sizeof(double) * (4 + 2 * (size_t)s)) : 0;
    // two-pass: coefficients z[m] and the second pass's iscal[4]
    const size_t szTwo = two ? al(sizeof(double) * m) + al(sizeof(int) * 4) : 0;
    const size_t total =
        al(szV) + 2 * al(szS) + al(szH) + al(sizeof(double) * m) + al(sizeof(int) * 4) + szStop + szTwo;
    char *ws = nullptr;
    skf_status st = dalloc((void **)&ws, total, cs);
    if (st != SKF_OK) return st;
    size_t off = 0;
    void *V = (void *)(ws + off); off += al(szV);
    double *SV = (double *)(ws + off); off += al(szS);
    double *SAV = (double *)(ws + off); off += al(szS);
    double *H = (double *)(ws + off); off += al(szH);
    double *vscale = (double *)(ws + off); off += al(sizeof(double) * m);
    int *iscal = (int *)(ws + off); off += al(sizeof(int) * 4);
    StopCtx sc{};
    StepHook hook{};
    if (stopping) {
        sc.iscal_chk = (int *)(ws + off); off += al(sizeof(int) * 4);
        sc.state = (double *)(ws + off); off += al(sizeof(double) * (4 + 2 * (size_t)s));
        sc.sf_prev = sc.state + 4;
        sc.sf_cur = sc.sf_prev + s;
        cudaMemsetAsync(sc.state, 0, sizeof(double) * (4 + 2 * (size_t)s), cs);
        sc.method = method;
        sc.s = s;
        sc.m = m;
        sc.d = p.check_every;
        sc.next_p = p.check_every;
        sc.vscale = vscale;
        sc.SV = SV;
        sc.SAV = SAV;
        sc.iscal = iscal;
        sc.rule = &rule;
        sc.tol_quad = p.tol;
        sc.stop_tol = p.stop_tol;
        sc.err = SKF_OK;
        hook.fn = stop_hook;
        hook.ctx = &sc;
    }
    double *z = nullptr;
    int *iscal2 = nullptr;
    if (two) {
        z = (double *)(ws + off); off += al(sizeof(double) * m);
        iscal2 = (int *)(ws + off); off += al(sizeof(int) * 4);
    }
    st = run_arnoldi(A, S, (const double *)b, m, p.k, bt, V, ldv, vscale, SV, SAV, H, iscal, info, cs,
                     stopping ? &hook : nullptr, vring);
    if (st == SKF_OK && sc.err != SKF_OK) st = sc.err;
    if (st == SKF_OK)
        st = tail_run(method, s, m, n, V, bt, ldv, vscale, SV, SAV, iscal, rule, p.tol, two ? nullptr : (double *)x,
                      info, cs, nullptr, stopping ? sc.state : nullptr, z,
                      p.cond_max == 0.0 ? 1e12 : (p.cond_max < 0.0 ? 0.0 : p.cond_max), H, m + 1, p.k);
    if (st == SKF_OK && two) {
        // second pass: the same recurrence (same sketches, H, vscale rewritten
        // with identical values), accumulating x column by column
        AccCtx ac{V, bt, ldv, n, vring, z, iscal, iscal2, (double *)x, SKF_OK};
        StepHook h2{};
        h2.col_fn = acc_hook;
        h2.col_ctx = &ac;
        st = run_arnoldi(A, S, (const double *)b, m, p.k, bt, V, ldv, vscale, SV, SAV, H, iscal2, nullptr, cs, &h2,
                         vring);
        if (st == SKF_OK) st = ac.err;
    }
    dfree(ws, cs);
    return st;
}

// ---------------------------------------------------------------- lanes
constexpr int kMaxLanes = 16;

// Non-blocking streams and fork/join events of skf_solve_batched, created
// once per device and kept until the process exits.
struct LanePool {
    cudaStream_t s[kMaxLanes];
    cudaEvent_t join[kMaxLanes];
    cudaEvent_t fork;
};

static std::mutex &lane_mutex() {
    static std::mutex *mu = new std::mutex();
    return *mu;
}

// Caller holds lane_mutex().
static skf_status lane_pool(LanePool **out) {
    static std::map<int, LanePool *> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    auto it = pools.find(dev);
    if (it != pools.end()) {
        *out = it->second;
        return SKF_OK;
    }
    LanePool *p = new LanePool();
    e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    for (int l = 0; l < kMaxLanes && e == cudaSuccess; ++l) {
        e = cudaStreamCreateWithFlags(&p->s[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join[l], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "lane stream creation");   // partial pool leaks; rare
    pools[dev] = p;
    *out = p;
    return SKF_OK;
}

// Estimated device seconds of one problem: m steps, each the larger of its
// streamed bytes at HBM speed and a launch-latency floor, plus a tail that
// grows with m (Householder columns and quadrature nodes).
static double solve_cost(const skf_problem &q) {
    const double vb = (double)dtype_size(q.p->basis_dtype);
    const double ab = (double)dtype_size(q.A->vdtype) + 4.0;
    const double bytes = (double)q.A->nnz * ab + 3.0 * (double)q.A->n * vb;
    const double step = std::max(bytes / 6.0e12, 12.0e-6);
    return q.p->m * (step + 40.0e-6);
}

// Longest-processing-time-first: problems by decreasing cost, each onto the
// lane with the least work so far (ties: lowest lane, then lowest index).
static void assign_lanes(int n, const skf_problem *probs, int L, int *lane_of, int *order) {
    std::vector<double> cost((size_t)n);
    for (int i = 0; i < n; ++i) {
        cost[i] = solve_cost(probs[i]);
        order[i] = i;
    }
    std::stable_sort(order, order + n, [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load((size_t)L, 0.0);
    for (int t = 0; t < n; ++t) {
        const int i = order[t];
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane_of[i] = l;
        load[l] += cost[i];
    }
}

}  // namespace
}  // namespace skf

using namespace skf;

extern "C" {

const char *skf_last_error(void) { return g_last_error.c_str(); }

const char *skf_status_string(skf_status s) {
    switch (s) {
        case SKF_OK: return "ok";
        case SKF_ERR_INVALID_ARG: return "invalid argument";
        case SKF_ERR_CUDA: return "CUDA error";
        case SKF_ERR_OOM: return "out of device memory";
        case SKF_ERR_ILL_CONDITIONED: return "ill-conditioned";
        case SKF_ERR_BRANCH_CUT: return "singular shifted system (branch cut)";
        case SKF_ERR_QUAD_NOT_CONVERGED: return "quadrature not converged";
        case SKF_ERR_SKETCH_TOO_SMALL: return "sketch too small";
        case SKF_ERR_NOT_SUPPORTED: return "not supported";
        case SKF_ERR_ZERO_RHS: return "zero right-hand side";
        case SKF_ERR_TIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

int32_t skf_version(void) { return 100; }

int64_t skf_kernel_launch_count(void) { return (int64_t)g_launches.load(); }

skf_status skf_set_arnoldi_mode(int32_t mode) {
    if (mode < 0 || mode > 2) return fail(SKF_ERR_INVALID_ARG, "Arnoldi mode must be 0, 1 or 2");
    set_step_mode(mode);
    return SKF_OK;
}

static int g_block_mode = 0;   // 0 columns one after another, 1 lockstep with one SpMM per step

skf_status skf_set_block_mode(int32_t mode) {
    if (mode < 0 || mode > 1) return fail(SKF_ERR_INVALID_ARG, "block mode must be 0 or 1");
    g_block_mode = mode;
    return SKF_OK;
}

skf_status skf_set_qr_mode(int32_t mode) {
    if (mode < 0 || mode > 1) return fail(SKF_ERR_INVALID_ARG, "QR mode must be 0 or 1");
    set_qr_mode(mode);
    return SKF_OK;
}

// FP64 FMA throughput of this device: every SM runs 32 warps, each thread
// four independent accumulations x_c += y_c b (the operand pattern of a dot
// product; on this part it retires faster than chains that reuse one
// multiplier register, 1.20 against 1.01 TFLOP/s measured), timed with events.
constexpr int kRateChains = 4;
__global__ void __launch_bounds__(512) k_fp64_rate(double *sink, double a, double b, int iters) {
    double x[kRateChains], y[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) {
        x[c] = a + c * 1e-3 * threadIdx.x;
        y[c] = b - c * 1e-4;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kRateChains; ++c) x[c] = fma(y[c], b, x[c]);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) t += x[c] + y[c];
    if (t == 12345.678) sink[0] = t;   // keeps the chains live; never true for these inputs
}

skf_status skf_fp64_peak(double *gflops, skf_stream_t stream) {
    if (!gflops) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    double *sink = nullptr;
    skf_status s = dalloc((void **)&sink, sizeof(double), st);
    if (s != SKF_OK) return s;
    const int grid = 2 * num_sms(), iters = 8192;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        dfree(sink, st);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    k_fp64_rate<<<grid, 512, 0, st>>>(sink, 0.5, 0.999, iters);   // warm-up
    cudaEventRecord(e0, st);
    k_fp64_rate<<<grid, 512, 0, st>>>(sink, 0.5, 0.999, iters);
    cudaEventRecord(e1, st);
    count_launches(2);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(sink, st);
    if (e != cudaSuccess) return cuda_fail(e, "FP64 rate probe");
    *gflops = 2.0 * kRateChains * iters * (double)grid * 512.0 / (ms * 1e-3) / 1e9;
    return SKF_OK;
}

skf_status skf_workspace_trim(void) {
    std::lock_guard<std::mutex> lk(pool_mutex());
    for (auto &kv : pools()) {
        if (!kv.second) continue;
        const cudaError_t e = cudaMemPoolTrimTo(kv.second, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolTrimTo");
    }
    return SKF_OK;
}

skf_status skf_set_tail_form(int32_t form) {
    if (form < 0 || form > 1) return fail(SKF_ERR_INVALID_ARG, "tail form must be 0 or 1");
    set_tail_form(form);
    return SKF_OK;
}

skf_status skf_barrier_selftest(int32_t ctas, int64_t budget_cycles, int32_t *status_device, skf_stream_t stream) {
    if (!status_device) return fail(SKF_ERR_INVALID_ARG, "status_device is NULL");
    if (ctas < 1 || ctas > num_sms()) return fail(SKF_ERR_INVALID_ARG, "need 1 <= ctas <= number of SMs");
    if (budget_cycles < 1000 || budget_cycles > 10000000000ll)
        return fail(SKF_ERR_INVALID_ARG, "budget_cycles must be in [1e3, 1e10]");
    return barrier_selftest(ctas, budget_cycles, (int *)status_device, (cudaStream_t)stream);
}

// The slice layout of A (see skf_csr): rows longer than `cut` entries take
// the row-split path; sort: 1 rows sorted by length in windows of kSortWin,
// 0 not sorted, -1 sorted when that saves over a fifth of the padded entries.
// Replaces any earlier layout (sell_w and sell_off stay allocated).
static void free_layout(skf_csr *A) {
    if (A->sell_val) cudaFree(A->sell_val);
    if (A->sell_col) cudaFree(A->sell_col);
    if (A->perm) cudaFree(A->perm);
    if (A->sell_long) cudaFree(A->sell_long);
    if (A->long_seg0) cudaFree(A->long_seg0);
    if (A->seg_beg) cudaFree(A->seg_beg);
    if (A->seg_end) cudaFree(A->seg_end);
    A->sell_val = nullptr;
    A->sell_col = nullptr;
    A->perm = nullptr;
    A->sell_long = nullptr;
    A->long_seg0 = A->seg_beg = A->seg_end = nullptr;
    A->nlong = A->nseg = 0;
    A->max_width = 0;
    A->max_chunk_entries = 0;
}

static skf_status build_layout(skf_csr *A, int cut, int sort, cudaStream_t st) {
    const int64_t n = A->n;
    const size_t esz = A->vdtype == SKF_F64 ? 8 : 4;
    cudaError_t e = cudaStreamSynchronize(st);   // an earlier layout may still be in use on st
    if (e != cudaSuccess) return cuda_fail(e, "layout");
    free_layout(A);
    A->long_cut = cut;
    std::vector<int32_t> hw(A->nslices);
    std::vector<int64_t> hoff(A->nslices + 1);
    std::vector<int32_t> hrp((size_t)n + 1);
    cudaMemcpyAsync(hrp.data(), A->rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "row lengths");
    auto eff = [&](int64_t r) {
        const int32_t len = hrp[r + 1] - hrp[r];
        return len > cut ? 0 : len;
    };
    std::vector<int32_t> hperm((size_t)n);
    for (int64_t i = 0; i < n; ++i) hperm[i] = (int32_t)i;
    auto padded_of = [&]() {
        int64_t pad = 0;
        for (int64_t t = 0; t < A->nslices; ++t) {
            int mx = 0;
            for (int64_t i = 32 * t; i < std::min<int64_t>(n, 32 * t + 32); ++i) mx = std::max(mx, eff(hperm[i]));
            pad += 32ll * mx;
        }
        return pad;
    };
    bool sorted = false;
    if (sort != 0) {
        const int64_t pad_plain = padded_of();
        for (int64_t w0 = 0; w0 < n; w0 += kSortWin) {
            const int64_t w1 = std::min<int64_t>(n, w0 + kSortWin);
            std::stable_sort(hperm.begin() + w0, hperm.begin() + w1,
                             [&](int32_t x, int32_t y) { return eff(x) > eff(y); });
        }
        sorted = sort == 1 || padded_of() * 5 < pad_plain * 4;
        if (!sorted)
            for (int64_t i = 0; i < n; ++i) hperm[i] = (int32_t)i;
    }
    for (int64_t t = 0; t < A->nslices; ++t) {
        int mx = 0;
        for (int64_t i = 32 * t; i < std::min<int64_t>(n, 32 * t + 32); ++i) mx = std::max(mx, eff(hperm[i]));
        hw[t] = mx;
    }
    if (sorted) {
        if (cudaMalloc(&A->perm, sizeof(int32_t) * n) != cudaSuccess) {
            cudaGetLastError();
            return fail(SKF_ERR_OOM, "slice permutation allocation");
        }
        cudaMemcpyAsync(A->perm, hperm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    }
    cudaMemcpyAsync(A->sell_w, hw.data(), sizeof(int32_t) * A->nslices, cudaMemcpyHostToDevice, st);
    // row split: long rows, their segments and the per-slice masks
    std::vector<uint2> hl((size_t)A->nslices, make_uint2(0u, 0u));
    std::vector<int32_t> seg0{0}, sb, se;
    int64_t nl = 0;
    for (int64_t t = 0; t < A->nslices; ++t) {
        hl[t].y = (unsigned)nl;
        for (int l = 0; l < 32 && 32 * t + l < n; ++l) {
            const int64_t r = hperm[32 * t + l];
            const int32_t b0 = hrp[r], b1 = hrp[r + 1];
            if (b1 - b0 <= cut) continue;
            hl[t].x |= 1u << l;
            for (int32_t p0 = b0; p0 < b1; p0 += kSegLen) {
                sb.push_back(p0);
                se.push_back(std::min(b1, p0 + kSegLen));
            }
            seg0.push_back((int32_t)sb.size());
            ++nl;
        }
    }
    A->nlong = nl;
    A->nseg = (int64_t)sb.size();
    if (nl > 0) {
        if (cudaMalloc(&A->sell_long, sizeof(uint2) * A->nslices) != cudaSuccess ||
            cudaMalloc(&A->long_seg0, sizeof(int32_t) * seg0.size()) != cudaSuccess ||
            cudaMalloc(&A->seg_beg, sizeof(int32_t) * sb.size()) != cudaSuccess ||
            cudaMalloc(&A->seg_end, sizeof(int32_t) * se.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(SKF_ERR_OOM, "row-split allocation");
        }
        cudaMemcpyAsync(A->sell_long, hl.data(), sizeof(uint2) * A->nslices, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(A->long_seg0, seg0.data(), sizeof(int32_t) * seg0.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(A->seg_beg, sb.data(), sizeof(int32_t) * sb.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(A->seg_end, se.data(), sizeof(int32_t) * se.size(), cudaMemcpyHostToDevice, st);
    }
    hoff[0] = 0;
    for (int64_t t = 0; t < A->nslices; ++t) {
        hoff[t + 1] = hoff[t] + 32ll * hw[t];
        A->max_width = std::max(A->max_width, hw[t]);
    }
    for (int64_t t0 = 0; t0 < A->nslices; t0 += kChunkRows / 32) {
        const int64_t t1 = std::min<int64_t>(A->nslices, t0 + kChunkRows / 32);
        A->max_chunk_entries = std::max<int64_t>(A->max_chunk_entries, hoff[t1] - hoff[t0]);
    }
    const int64_t padded = hoff[A->nslices];
    if (cudaMalloc(&A->sell_val, esz * std::max<int64_t>(padded, 1)) != cudaSuccess ||
        cudaMalloc(&A->sell_col, sizeof(int32_t) * std::max<int64_t>(padded, 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SKF_ERR_OOM, "SELL allocation");
    }
    cudaMemcpyAsync(A->sell_off, hoff.data(), sizeof(int64_t) * (A->nslices + 1), cudaMemcpyHostToDevice, st);
    const int blocks = (int)std::min<int64_t>((n + 256) / 256, 8 * num_sms());
    if (A->vdtype == SKF_F64)
        k_sell_fill<<<blocks, 256, 0, st>>>(A->rowptr, A->colind, (const double *)A->values, n, A->nslices, cut,
                                            A->perm, A->sell_off, A->sell_w, (double *)A->sell_val, A->sell_col);
    else
        k_sell_fill<<<blocks, 256, 0, st>>>(A->rowptr, A->colind, (const float *)A->values, n, A->nslices, cut,
                                            A->perm, A->sell_off, A->sell_w, (float *)A->sell_val, A->sell_col);
    count_launches(1);
    e = cudaStreamSynchronize(st);   // the host vectors above are released on return
    if (e != cudaSuccess) return cuda_fail(e, "SELL fill");
    return SKF_OK;
}

skf_status skf_create_csr(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind, const void *values,
                          skf_dtype vdtype, skf_copy_mode mode, skf_stream_t stream, skf_csr **A_out) {
    if (!A_out) return fail(SKF_ERR_INVALID_ARG, "A_out is NULL");
    *A_out = nullptr;
    if (n < 1 || n >= (1ll << 31)) return fail(SKF_ERR_INVALID_ARG, "n must be in [1, 2^31)");
    if (nnz < 0 || nnz >= (1ll << 31)) return fail(SKF_ERR_INVALID_ARG, "nnz must be in [0, 2^31)");
    if (!rowptr || (nnz > 0 && (!colind || !values))) return fail(SKF_ERR_INVALID_ARG, "NULL CSR array");
    if (vdtype != SKF_F64 && vdtype != SKF_F32) return fail(SKF_ERR_NOT_SUPPORTED, "matrix values must be F64 or F32");
    const size_t esz = vdtype == SKF_F64 ? sizeof(double) : sizeof(float);
    if (mode != SKF_BORROW && mode != SKF_COPY) return fail(SKF_ERR_INVALID_ARG, "bad copy mode");
    cudaStream_t st = (cudaStream_t)stream;
    skf_csr *A = new skf_csr();
    A->n = n;
    A->nnz = nnz;
    A->vdtype = vdtype;
    int *dbad = nullptr;
    unsigned long long *dmax = nullptr;
    auto cleanup = [&](skf_status s) {
        if (dbad) cudaFree(dbad);
        if (dmax) cudaFree(dmax);
        skf_destroy_csr(A);
        return s;
    };
    if (cudaMalloc(&A->rowptr, sizeof(int32_t) * (n + 1)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(SKF_ERR_OOM, "rowptr allocation"));
    }
    if (mode == SKF_COPY && nnz > 0) {
        if (cudaMalloc(&A->colind_own, sizeof(int32_t) * nnz) != cudaSuccess ||
            cudaMalloc(&A->values_own, esz * nnz) != cudaSuccess) {
            cudaGetLastError();
            return cleanup(fail(SKF_ERR_OOM, "CSR copy allocation"));
        }
        if (cudaMemcpyAsync(A->colind_own, colind, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(A->values_own, values, esz * nnz, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return cleanup(cuda_fail(cudaGetLastError(), "CSR copy"));
        A->colind = A->colind_own;
        A->values = A->values_own;
    } else {
        A->colind = colind;
        A->values = values;
    }
    if (cudaMalloc(&dbad, sizeof(int)) != cudaSuccess || cudaMalloc(&dmax, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(SKF_ERR_OOM, "scratch allocation"));
    }
    cudaMemsetAsync(dbad, 0, sizeof(int), st);
    cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st);
    const int blocks = (int)std::min<int64_t>((n + 256) / 256, 8 * num_sms());
    k_rowptr32<<<blocks, 256, 0, st>>>(rowptr, n, A->rowptr, dbad);
    count_launches(1);
    int64_t last = 0, first = 0;
    cudaMemcpyAsync(&last, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&first, rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "skf_create_csr"));
    if (hbad || first != 0 || last != nnz) return cleanup(fail(SKF_ERR_INVALID_ARG, "invalid row pointer"));
    if (vdtype == SKF_F64)
        k_row_abs_sum<<<blocks, 256, 0, st>>>(A->rowptr, A->colind, (const double *)A->values, n, dbad, dmax);
    else
        k_row_abs_sum<<<blocks, 256, 0, st>>>(A->rowptr, A->colind, (const float *)A->values, n, dbad, dmax);
    count_launches(1);
    unsigned long long hmax = 0;
    cudaMemcpyAsync(&hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "skf_create_csr"));
    if (hbad) return cleanup(fail(SKF_ERR_INVALID_ARG, "column index out of range"));
    memcpy(&A->norm_inf, &hmax, sizeof(double));
    // SELL-32 copy for the kernels: rows over kLongRow entries split off,
    // slices unsorted (sorting paid on neither graph workload when timed:
    // skf_csr_autotune chooses it where it does)
    A->nslices = (n + 31) / 32;
    if (cudaMalloc(&A->sell_w, sizeof(int32_t) * A->nslices) != cudaSuccess ||
        cudaMalloc(&A->sell_off, sizeof(int64_t) * (A->nslices + 1)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(SKF_ERR_OOM, "SELL allocation"));
    }
    {
        const skf_status ls = build_layout(A, kLongRow, 0, st);
        if (ls != SKF_OK) return cleanup(ls);
    }
    cudaFree(dbad);
    cudaFree(dmax);
    *A_out = A;
    return SKF_OK;
}

skf_status skf_destroy_csr(skf_csr *A) {
    if (!A) return SKF_OK;
    if (A->rowptr) cudaFree(A->rowptr);
    if (A->colind_own) cudaFree(A->colind_own);
    if (A->values_own) cudaFree(A->values_own);
    if (A->sell_off) cudaFree(A->sell_off);
    if (A->sell_w) cudaFree(A->sell_w);
    if (A->sell_val) cudaFree(A->sell_val);
    if (A->sell_col) cudaFree(A->sell_col);
    if (A->sell_long) cudaFree(A->sell_long);
    if (A->perm) cudaFree(A->perm);
    if (A->long_seg0) cudaFree(A->long_seg0);
    if (A->seg_beg) cudaFree(A->seg_beg);
    if (A->seg_end) cudaFree(A->seg_end);
    delete A;
    return SKF_OK;
}

// Deterministic probe vector for the layout autotuner: entries in [-1, 1)
// from SplitMix64 of the row index (no meaning beyond "dense and signed").
__global__ void k_probe_rhs(double *b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        b[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

skf_status skf_csr_set_layout(skf_csr *A, int32_t cut, int32_t sorted, skf_stream_t stream) {
    if (!A) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    if (cut < 1 || sorted < -1 || sorted > 1) return fail(SKF_ERR_INVALID_ARG, "need cut >= 1 and sorted in -1..1");
    return build_layout(A, cut, sorted, (cudaStream_t)stream);
}

// Layout candidates of skf_csr_autotune: (row-split cut, sorted slices).
static const int kTuneCut[] = {16, 32, 64, 16, 32, 64};
static const int kTuneSort[] = {0, 0, 0, 1, 1, 1};
constexpr int kTuneCandidates = 6;

skf_status skf_csr_autotune(skf_csr *A, const skf_sketch *S, int32_t k, skf_dtype basis, int32_t m_probe,
                            double *times_us, int32_t *choice, skf_stream_t stream) {
    if (!A || !S) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    if (m_probe <= 0) m_probe = 8;
    const double dummy = 0.0;
    skf_status stt = check_common(A, S, &dummy, SKF_F64, m_probe, k, basis);
    if (stt != SKF_OK) return stt;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = A->n;
    const int m = m_probe;
    const int s = S->s;
    const int64_t ldv = (n + 63) / 64 * 64;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t szV = dtype_size(basis) * (size_t)ldv * m;
    const size_t total = al(sizeof(double) * n) + al(szV) + 2 * al(sizeof(double) * (size_t)s * m) +
                         al(sizeof(double) * (size_t)(m + 1) * m) + al(sizeof(double) * m) + al(sizeof(int) * 4);
    char *ws = nullptr;
    stt = dalloc((void **)&ws, total, st);
    if (stt != SKF_OK) return stt;
    size_t off = 0;
    auto take = [&](size_t sz) {
        char *p = ws + off;
        off += al(sz);
        return p;
    };
    double *b = (double *)take(sizeof(double) * n);
    void *V = take(szV);
    double *SV = (double *)take(sizeof(double) * (size_t)s * m);
    double *SAV = (double *)take(sizeof(double) * (size_t)s * m);
    double *H = (double *)take(sizeof(double) * (size_t)(m + 1) * m);
    double *vscale = (double *)take(sizeof(double) * m);
    int *iscal = (int *)take(sizeof(int) * 4);
    k_probe_rhs<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8ll * num_sms()), 256, 0, st>>>(b, n);
    count_launches(1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        dfree(ws, st);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    double t[kTuneCandidates];
    int best = -1;
    for (int c = 0; c < kTuneCandidates && stt == SKF_OK; ++c) {
        stt = build_layout(A, kTuneCut[c], kTuneSort[c], st);
        double tmin = INFINITY;
        for (int rep = 0; rep < 3 && stt == SKF_OK; ++rep) {   // the first run warms up
            cudaEventRecord(e0, st);
            stt = run_arnoldi(A, S, b, m, k, basis, V, ldv, vscale, SV, SAV, H, iscal, nullptr, st);
            cudaEventRecord(e1, st);
            if (stt != SKF_OK) break;
            float ms = 0.f;
            const cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                stt = cuda_fail(ce != cudaSuccess ? ce : cudaGetLastError(), "autotune timing");
                break;
            }
            if (rep > 0) tmin = std::min(tmin, (double)ms * 1e3 / m);
        }
        t[c] = tmin;
        if (stt == SKF_OK && (best < 0 || t[c] < t[best])) best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(ws, st);
    // keep the fastest layout (or restore the default one after a failure)
    const skf_status ls = best >= 0 && stt == SKF_OK ? build_layout(A, kTuneCut[best], kTuneSort[best], st)
                                                     : build_layout(A, kLongRow, 0, st);
    if (stt != SKF_OK) return stt;
    if (ls != SKF_OK) return ls;
    if (times_us)
        for (int c = 0; c < kTuneCandidates; ++c) times_us[c] = t[c];
    if (choice) *choice = best;
    return SKF_OK;
}

skf_status skf_csr_norm_inf(const skf_csr *A, double *out_host) {
    if (!A || !out_host) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    *out_host = A->norm_inf;
    return SKF_OK;
}

skf_status skf_sketch_create(skf_sketch_kind kind, int64_t n, int32_t s, int32_t zeta, uint64_t seed,
                             skf_stream_t stream, skf_sketch **S_out) {
    if (!S_out) return fail(SKF_ERR_INVALID_ARG, "S_out is NULL");
    *S_out = nullptr;
    if (n < 1 || s < 1) return fail(SKF_ERR_INVALID_ARG, "n and s must be positive");
    if (kind == SKF_SKETCH_SPARSE_SIGN) {
        if (zeta < 1 || zeta > s || zeta > kMaxZeta) return fail(SKF_ERR_INVALID_ARG, "need 1 <= zeta <= min(s, 16)");
        if (s / zeta > 32768) return fail(SKF_ERR_INVALID_ARG, "s / zeta must be <= 32768");
    } else if (kind == SKF_SKETCH_IDENTITY) {
        if (s != n) return fail(SKF_ERR_INVALID_ARG, "identity sketch needs s == n");
        zeta = 1;
    } else if (kind == SKF_SKETCH_SRHT || kind == SKF_SKETCH_SRDCT) {
        zeta = 0;
    } else {
        return fail(SKF_ERR_INVALID_ARG, "unknown sketch kind");
    }
    skf_sketch *S = new skf_sketch();
    S->kind = kind;
    S->n = n;
    S->s = s;
    S->zeta = zeta;
    S->seed = seed;
    if (kind != SKF_SKETCH_IDENTITY) {
        const skf_status st = kind == SKF_SKETCH_SRHT    ? build_srht_tables(S)
                              : kind == SKF_SKETCH_SRDCT ? build_srdct_tables(S)
                                                         : build_sparse_sign_tables(S, (cudaStream_t)stream);
        if (st != SKF_OK) {
            skf_sketch_destroy(S);
            return st;
        }
    }
    *S_out = S;
    return SKF_OK;
}

skf_status skf_sketch_destroy(skf_sketch *S) {
    if (!S) return SKF_OK;
    if (S->P) cudaFree(S->P);
    if (S->pattern) cudaFree(S->pattern);
    if (S->binmax) cudaFree(S->binmax);
    if (S->pattern8) cudaFree(S->pattern8);
    if (S->E) cudaFree(S->E);
    if (S->costab) cudaFree(S->costab);
    if (S->tw) cudaFree(S->tw);
    if (S->twist) cudaFree(S->twist);
    delete S;
    return SKF_OK;
}

skf_status skf_sketch_apply(const skf_sketch *S, const void *X, skf_dtype xdtype, int64_t ldx, int32_t ncols,
                            double *SX, skf_stream_t stream) {
    if (!S || (!X && ncols > 0) || (!SX && ncols > 0)) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    if (ncols < 0 || ldx < S->n) return fail(SKF_ERR_INVALID_ARG, "ncols < 0 or ldx < n");
    if (xdtype != SKF_F64) return fail(SKF_ERR_NOT_SUPPORTED, "X must be F64 in this build");
    return sketch_apply_f64(S, (const double *)X, ldx, ncols, SX, (cudaStream_t)stream);
}

skf_status skf_sketch_apply_noalloc(const skf_sketch *S, const void *X, skf_dtype xdtype, int64_t ldx, int32_t ncols,
                                    double *SX, skf_stream_t stream) {
    if (!S || (!X && ncols > 0) || (!SX && ncols > 0)) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    if (ncols < 0 || ldx < S->n) return fail(SKF_ERR_INVALID_ARG, "ncols < 0 or ldx < n");
    if (xdtype != SKF_F64) return fail(SKF_ERR_NOT_SUPPORTED, "X must be F64 in this build");
    return sketch_apply_f64_noalloc(S, (const double *)X, ldx, ncols, SX, (cudaStream_t)stream);
}

skf_status skf_arnoldi_trunc(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype, int32_t m,
                             int32_t k, skf_dtype basis_dtype, void *V, int64_t ldv, double *vscale, double *SV,
                             double *SAV, double *H, skf_info *info, skf_stream_t stream) {
    skf_status st = check_common(A, S, b, bdtype, m, k, basis_dtype);
    if (st != SKF_OK) return st;
    if (!V || !vscale || !SV || !SAV || !H) return fail(SKF_ERR_INVALID_ARG, "NULL output");
    if (ldv < A->n) return fail(SKF_ERR_INVALID_ARG, "ldv < n");
    cudaStream_t cs = (cudaStream_t)stream;
    int *iscal = nullptr;
    st = dalloc((void **)&iscal, sizeof(int) * 4, cs);
    if (st != SKF_OK) return st;
    st = run_arnoldi(A, S, (const double *)b, m, k, basis_dtype, V, ldv, vscale, SV, SAV, H, iscal, info, cs);
    dfree(iscal, cs);
    return st;
}

skf_status skf_solve(skf_method method, const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype,
                     const skf_func *f, const skf_params *p, void *x, skf_dtype xdtype, skf_info *info,
                     skf_stream_t stream) {
    const RuleDev *rule = nullptr;
    skf_status st = solve_check(method, A, S, b, bdtype, f, p, x, xdtype, &rule);
    if (st != SKF_OK) return st;
    return solve_enqueue(method, A, S, b, *p, x, info, *rule, (cudaStream_t)stream);
}

// Both methods on one Arnoldi process (skf_sfom_sgmres).
skf_status skf_solve_block(skf_method method, const skf_csr *A, const skf_sketch *S, const double *B, int64_t ldb,
                           int32_t nrhs, const skf_func *f, const skf_params *p, double *X, int64_t ldx,
                           skf_info *info, skf_stream_t stream) {
    if (nrhs < 0 || (nrhs > 0 && (!B || !X))) return fail(SKF_ERR_INVALID_ARG, "bad block arguments");
    if (nrhs == 0) return SKF_OK;
    if (!A || ldb < A->n || ldx < A->n) return fail(SKF_ERR_INVALID_ARG, "need ldb, ldx >= N");
    const RuleDev *rule = nullptr;
    skf_status st = solve_check(method, A, S, B, SKF_F64, f, p, X, SKF_F64, &rule);
    if (st != SKF_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const int m = p->m, s = S->s;
    const int64_t n = A->n;
    auto col = [](const double *base, int64_t ld, int q) { return base + (size_t)q * ld; };
    // the lockstep form (skf_set_block_mode(1)): F32 basis, one pass, no
    // stopping criterion
    const bool lockstep = g_block_mode == 1 && p->basis_dtype == SKF_F32 && p->two_pass == 0 &&
                          !(p->check_every > 0 && p->check_every < m) && nrhs > 1;
    if (!lockstep) {
        for (int q = 0; q < nrhs; ++q) {
            st = solve_enqueue(method, A, S, col(B, ldb, q), *p, X + (size_t)q * ldx, info ? info + q : nullptr,
                               *rule, cs);
            if (st != SKF_OK) return st;
        }
        return SKF_OK;
    }
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const int64_t ldv = (n + 63) / 64 * 64;
    const size_t szV = sizeof(float) * (size_t)ldv * m;
    const size_t szS = sizeof(double) * (size_t)s * m;
    const size_t szH = sizeof(double) * (size_t)(m + 1) * m;
    const size_t per = al(szV) + 2 * al(szS) + al(szH) + al(sizeof(double) * m) + al(sizeof(int) * 4);
    char *ws = nullptr;
    st = dalloc((void **)&ws, per * (size_t)nrhs, cs);
    if (st != SKF_OK) return st;
    std::vector<const double *> bq(nrhs);
    std::vector<float *> Vq(nrhs);
    std::vector<double *> vs(nrhs), SVq(nrhs), SAVq(nrhs), Hq(nrhs);
    std::vector<int *> isc(nrhs);
    std::vector<skf_info *> inf(nrhs);
    for (int q = 0; q < nrhs; ++q) {
        char *w = ws + per * (size_t)q;
        size_t off = 0;
        Vq[q] = (float *)(w + off); off += al(szV);
        SVq[q] = (double *)(w + off); off += al(szS);
        SAVq[q] = (double *)(w + off); off += al(szS);
        Hq[q] = (double *)(w + off); off += al(szH);
        vs[q] = (double *)(w + off); off += al(sizeof(double) * m);
        isc[q] = (int *)(w + off);
        bq[q] = col(B, ldb, q);
        inf[q] = info ? info + q : nullptr;
    }
    st = arnoldi_run_f32_block(A, S, nrhs, bq.data(), m, p->k, Vq.data(), ldv, vs.data(), SVq.data(), SAVq.data(),
                               Hq.data(), isc.data(), inf.data(), cs);
    const double cond_max = p->cond_max == 0.0 ? 1e12 : (p->cond_max < 0.0 ? 0.0 : p->cond_max);
    for (int q = 0; q < nrhs && st == SKF_OK; ++q)
        st = tail_run(method, s, m, n, Vq[q], SKF_F32, ldv, vs[q], SVq[q], SAVq[q], isc[q], *rule, p->tol,
                      X + (size_t)q * ldx, inf[q], cs, nullptr, nullptr, nullptr, cond_max, Hq[q], m + 1, p->k);
    dfree(ws, cs);
    return st;
}

static skf_status solve_enqueue_pair(const skf_csr *A, const skf_sketch *S, const void *b, const skf_params &p,
                                     void *x_fom, void *x_gmres, skf_info *info_fom, skf_info *info_gmres,
                                     const RuleDev &rule, cudaStream_t cs) {
    const int m = p.m;
    const int64_t n = A->n;
    const int s = S->s;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const skf_dtype bt = p.basis_dtype;
    const int64_t ldv = (n + 63) / 64 * 64;   // 256-byte aligned columns
    const size_t szV = dtype_size(bt) * (size_t)ldv * m;
    const size_t szS = sizeof(double) * (size_t)s * m;
    const size_t szH = sizeof(double) * (size_t)(m + 1) * m;
    const size_t total = al(szV) + 2 * al(szS) + al(szH) + al(sizeof(double) * m) + 2 * al(sizeof(int) * 4);
    char *ws = nullptr;
    skf_status st = dalloc((void **)&ws, total, cs);
    if (st != SKF_OK) return st;
    size_t off = 0;
    void *V = (void *)(ws + off); off += al(szV);
    double *SV = (double *)(ws + off); off += al(szS);
    double *SAV = (double *)(ws + off); off += al(szS);
    double *H = (double *)(ws + off); off += al(szH);
    double *vscale = (double *)(ws + off); off += al(sizeof(double) * m);
    int *iscal = (int *)(ws + off); off += al(sizeof(int) * 4);
    int *iscal2 = (int *)(ws + off); off += al(sizeof(int) * 4);
    st = run_arnoldi(A, S, (const double *)b, m, p.k, bt, V, ldv, vscale, SV, SAV, H, iscal, info_fom, cs, nullptr, 0);
    if (st == SKF_OK) {
        // the second method starts from the same Arnoldi record
        cudaMemcpyAsync(iscal2, iscal, sizeof(int) * 4, cudaMemcpyDeviceToDevice, cs);
        if (info_fom && info_gmres)
            cudaMemcpyAsync(info_gmres, info_fom, sizeof(skf_info), cudaMemcpyDefault, cs);
        TailOut outs[2] = {{SKF_METHOD_SFOM, (double *)x_fom, info_fom, nullptr, iscal},
                           {SKF_METHOD_SGMRES, (double *)x_gmres, info_gmres, nullptr, iscal2}};
        st = tail_run_multi(2, outs, s, m, n, V, bt, ldv, vscale, SV, SAV, rule, p.tol, cs, nullptr, nullptr,
                            p.cond_max == 0.0 ? 1e12 : (p.cond_max < 0.0 ? 0.0 : p.cond_max), H, m + 1, p.k);
    }
    dfree(ws, cs);
    return st;
}

skf_status skf_sfom_sgmres(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype, const skf_func *f,
                           const skf_params *p, void *x_fom, void *x_gmres, skf_dtype xdtype, skf_info *info_fom,
                           skf_info *info_gmres, skf_stream_t stream) {
    if (!x_gmres) return fail(SKF_ERR_INVALID_ARG, "NULL argument");
    const RuleDev *rule = nullptr;
    skf_status st = solve_check(SKF_METHOD_SGMRES, A, S, b, bdtype, f, p, x_fom, xdtype, &rule);
    if (st != SKF_OK) return st;
    if (p->check_every > 0 || p->two_pass)
        return fail(SKF_ERR_NOT_SUPPORTED, "the pair solve offers neither the stopping criterion nor two passes");
    return solve_enqueue_pair(A, S, b, *p, x_fom, x_gmres, info_fom, info_gmres, *rule, (cudaStream_t)stream);
}

skf_status skf_solve_batched(int32_t nprob, const skf_problem *probs, int32_t lanes, skf_stream_t stream) {
    if (nprob < 0 || (nprob > 0 && !probs)) return fail(SKF_ERR_INVALID_ARG, "bad problem array");
    if (lanes < 1 || lanes > kMaxLanes) return fail(SKF_ERR_INVALID_ARG, "lanes must be in 1..16");
    std::vector<const RuleDev *> rules((size_t)nprob, nullptr);
    for (int i = 0; i < nprob; ++i) {
        const skf_problem &q = probs[i];
        const skf_status st = solve_check(q.method, q.A, q.S, q.b, q.bdtype, q.f, q.p, q.x, q.xdtype, &rules[i]);
        if (st != SKF_OK) return fail(st, "problem " + std::to_string(i) + ": " + skf_last_error());
    }
    if (nprob == 0) return SKF_OK;
    cudaStream_t cs = (cudaStream_t)stream;
    const int L = std::min<int>(lanes, nprob);
    std::vector<int> lane_of((size_t)nprob, 0), order((size_t)nprob);
    assign_lanes(nprob, probs, L, lane_of.data(), order.data());
    if (L == 1) {
        for (int i : order) {
            const skf_problem &q = probs[i];
            const skf_status st = solve_enqueue(q.method, q.A, q.S, q.b, *q.p, q.x, q.info, *rules[i], cs);
            if (st != SKF_OK) return fail(st, "problem " + std::to_string(i) + ": " + skf_last_error());
        }
        return SKF_OK;
    }
    std::lock_guard<std::mutex> lk(lane_mutex());
    LanePool *pool = nullptr;
    skf_status st = lane_pool(&pool);
    if (st != SKF_OK) return st;
    cudaError_t e = cudaEventRecord(pool->fork, cs);
    for (int l = 0; l < L && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(pool->s[l], pool->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "lane fork");
    // enqueue in order; on a failure stop enqueuing but still join every lane
    std::string err;
    for (int i : order) {
        if (st != SKF_OK) break;
        const skf_problem &q = probs[i];
        st = solve_enqueue(q.method, q.A, q.S, q.b, *q.p, q.x, q.info, *rules[i], pool->s[lane_of[i]]);
        if (st != SKF_OK) err = "problem " + std::to_string(i) + ": " + skf_last_error();
    }
    for (int l = 0; l < L; ++l) {
        cudaError_t ej = cudaEventRecord(pool->join[l], pool->s[l]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(cs, pool->join[l], 0);
        if (ej != cudaSuccess && e == cudaSuccess) e = ej;
    }
    if (st != SKF_OK) return fail(st, err);
    if (e != cudaSuccess) return cuda_fail(e, "lane join");
    return SKF_OK;
}

// ---------------------------------------------------------------- precision plan
// iscal of one query of skf_plan_basis_precision: the leading min(m_q, m_eff)
// columns of the pilot basis, status OK, not stopped.
__global__ void k_plan_query(const int *__restrict__ pilot_iscal, int mq, int *__restrict__ iscal) {
    if (threadIdx.x == 0) {
        const int me = pilot_iscal[1] < mq ? pilot_iscal[1] : mq;
        iscal[0] = 0;
        iscal[1] = me;
        iscal[2] = SKF_OK;
        iscal[3] = me;
    }
}

skf_status skf_plan_basis_precision(int32_t nprob, const skf_problem *probs, double tol, double *cond_host,
                                    int32_t *f32_host, skf_stream_t stream) {
    if (nprob < 0 || (nprob > 0 && (!probs || !cond_host || !f32_host)))
        return fail(SKF_ERR_INVALID_ARG, "bad problem or output array");
    if (!(tol > 0.0)) return fail(SKF_ERR_INVALID_ARG, "tol must be > 0");
    std::vector<const RuleDev *> rules((size_t)nprob, nullptr);
    for (int i = 0; i < nprob; ++i) {
        const skf_problem &q = probs[i];
        const skf_status st = solve_check(q.method, q.A, q.S, q.b, q.bdtype, q.f, q.p, q.x, q.xdtype, &rules[i]);
        if (st != SKF_OK) return fail(st, "problem " + std::to_string(i) + ": " + skf_last_error());
        if (q.p->basis_dtype == SKF_BF16)
            return fail(SKF_ERR_NOT_SUPPORTED, "problem " + std::to_string(i) + ": plan from an FP64 or FP32 basis");
    }
    cudaStream_t cs = (cudaStream_t)stream;
    const double u32 = 5.9604644775390625e-08;   // 2^-24
    std::vector<bool> done((size_t)nprob, false);
    for (int i = 0; i < nprob; ++i) {
        if (done[i]) continue;
        // the problems on this operator; the pilot is the one with the largest m
        std::vector<int> grp;
        int pl = i;
        for (int r = i; r < nprob; ++r)
            if (!done[r] && probs[r].A == probs[i].A) {
                grp.push_back(r);
                if (probs[r].p->m > probs[pl].p->m) pl = r;
            }
        const skf_problem &q = probs[pl];
        const skf_params &pp = *q.p;
        const int m = pp.m, s = q.S->s;
        const int64_t n = q.A->n;
        const int64_t ldv = (n + 63) / 64 * 64;
        auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
        const size_t szV = dtype_size(pp.basis_dtype) * (size_t)ldv * m;
        const size_t szS = sizeof(double) * (size_t)s * m;
        const size_t szH = sizeof(double) * (size_t)(m + 1) * m;
        const size_t nq = grp.size();
        const size_t total = al(szV) + 2 * al(szS) + al(szH) + al(sizeof(double) * m) + al(sizeof(int) * 4) +
                             nq * (al(sizeof(int) * 4) + al(sizeof(skf_info)));
        char *ws = nullptr;
        skf_status st = dalloc((void **)&ws, total, cs);
        if (st != SKF_OK) return st;
        size_t off = 0;
        void *V = (void *)(ws + off); off += al(szV);
        double *SV = (double *)(ws + off); off += al(szS);
        double *SAV = (double *)(ws + off); off += al(szS);
        double *H = (double *)(ws + off); off += al(szH);
        double *vscale = (double *)(ws + off); off += al(sizeof(double) * m);
        int *iscal = (int *)(ws + off); off += al(sizeof(int) * 4);
        std::vector<int *> qis(nq);
        std::vector<skf_info *> qinf(nq);
        for (size_t t = 0; t < nq; ++t) {
            qis[t] = (int *)(ws + off); off += al(sizeof(int) * 4);
            qinf[t] = (skf_info *)(ws + off); off += al(sizeof(skf_info));
        }
        st = run_arnoldi(q.A, q.S, (const double *)q.b, m, pp.k, pp.basis_dtype, V, ldv, vscale, SV, SAV, H, iscal,
                         nullptr, cs);
        // the whitening of the leading m_r columns: its cond(R) estimate
        for (size_t t = 0; t < nq && st == SKF_OK; ++t) {
            k_plan_query<<<1, 32, 0, cs>>>(iscal, probs[grp[t]].p->m, qis[t]);
            count_launches(1);
            st = tail_run(SKF_METHOD_SGMRES, s, probs[grp[t]].p->m, 0, nullptr, SKF_F64, 0, vscale, SV, SAV, qis[t],
                          *rules[pl], pp.tol, nullptr, qinf[t], cs, nullptr, nullptr, nullptr, 0.0, H, m + 1, pp.k);
        }
        std::vector<skf_info> hinf(nq);
        cudaError_t e = cudaSuccess;
        for (size_t t = 0; t < nq && st == SKF_OK && e == cudaSuccess; ++t)
            e = cudaMemcpyAsync(&hinf[t], qinf[t], sizeof(skf_info), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        dfree(ws, cs);
        if (st != SKF_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "precision plan");
        for (size_t t = 0; t < nq; ++t) {
            const int r = grp[t];
            done[r] = true;
            const double cnd = hinf[t].cond_est;
            cond_host[r] = cnd;
            f32_host[r] = (cnd > 0.0 && cnd * u32 <= tol) ? 1 : 0;
        }
    }
    return SKF_OK;
}

skf_status skf_sfom(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype, const skf_func *f,
                    const skf_params *p, void *x, skf_dtype xdtype, skf_info *info, skf_stream_t stream) {
    return skf_solve(SKF_METHOD_SFOM, A, S, b, bdtype, f, p, x, xdtype, info, stream);
}

skf_status skf_sgmres(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype, const skf_func *f,
                      const skf_params *p, void *x, skf_dtype xdtype, skf_info *info, skf_stream_t stream) {
    return skf_solve(SKF_METHOD_SGMRES, A, S, b, bdtype, f, p, x, xdtype, info, stream);
}

skf_status skf_quadrature_rule_c(const skf_func *f, int32_t ell, double *t_re, double *t_im, double *w_re,
                                 double *w_im) {
    if (!f || !t_re || !t_im || !w_re || !w_im || ell < 1) return fail(SKF_ERR_INVALID_ARG, "bad argument");
    if (f->kind != SKF_FUNC_EXP_NEG) {
        if (!quadrature_rule(*f, ell, t_re, w_re))
            return fail(SKF_ERR_NOT_SUPPORTED, "no quadrature rule of this order for this function");
        for (int i = 0; i < ell; ++i) t_im[i] = w_im[i] = 0.0;
        return SKF_OK;
    }
    if (!contour_rule(*f, ell, t_re, t_im, w_re, w_im))
        return fail(SKF_ERR_INVALID_ARG, "the contour rule needs ell >= 2 and scale > 0");
    return SKF_OK;
}

skf_status skf_quadrature_rule(const skf_func *f, int32_t ell, double *t_host, double *w_host) {
    if (!f || !t_host || !w_host || ell < 1) return fail(SKF_ERR_INVALID_ARG, "bad argument");
    if (f->kind == SKF_FUNC_EXP_NEG)
        return fail(SKF_ERR_NOT_SUPPORTED, "exp(-z) has a complex contour rule: skf_quadrature_rule_c");
    if (!quadrature_rule(*f, ell, t_host, w_host))
        return fail(SKF_ERR_NOT_SUPPORTED, "no quadrature rule of this order for this function");
    return SKF_OK;
}

}  // extern "C"
