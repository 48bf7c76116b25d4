/*
 * skf.h -- C ABI of the GB300 sketched-Krylov f(A)b library.
 *
 * Method: Guettel & Schweitzer, "Randomized sketching for Krylov
 * approximations of large-scale matrix functions".  The library computes the
 * sketched FOM approximant (Sec. 2, eq. (sFOM) / (sFOM''')) and the sketched
 * GMRES approximant (Sec. 3, eq. (sGMRES)) of f(A)b for a sparse A in CSR
 * form and a Stieltjes function f, with the basis generated by the
 * k-truncated Arnoldi recurrence of Algorithm 2 and an s x N subspace
 * embedding S (eq. (1.1)) applied on the fly.
 *
 * Conventions for every entry point
 *   - Pointers are DEVICE pointers unless the argument says "host".
 *   - Matrices are column-major with the given leading dimension.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) and performs no host synchronisation, except
 *     skf_create_csr / skf_sketch_create, which may synchronise `stream`
 *     once while building their handle.
 *   - The return value reports argument validation and launch errors only.
 *     Numerical outcomes that are known only on the device (breakdown,
 *     branch cut, quadrature not converged, ill-conditioning) are written to
 *     skf_info::status when the stream reaches them.
 *   - On error the call returns a status != SKF_OK and skf_last_error()
 *     returns a message (thread-local, valid until the next call on the
 *     same thread).  No entry point throws across the ABI.
 *   - Handles own their device allocations; outputs are caller-allocated.
 *   - All device work runs in this library's CUDA kernels (sm_103a).  There
 *     is no CPU fallback: without a usable GPU every call returns
 *     SKF_ERR_CUDA.
 */
#ifndef SKF_H
#define SKF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *skf_stream_t; /* == cudaStream_t */

typedef enum {
    SKF_OK = 0,
    SKF_ERR_INVALID_ARG = 1,         /* bad size, null pointer, s <= m, zeta > s, ... */
    SKF_ERR_CUDA = 2,                /* a CUDA call failed (message has the CUDA error) */
    SKF_ERR_OOM = 3,                 /* device allocation failed */
    SKF_ERR_ILL_CONDITIONED = 4,     /* the estimate of cond(R) of the whitening QR passed
                                        skf_params::cond_max, or R is singular; x is still
                                        computed and written */
    SKF_ERR_BRANCH_CUT = 5,          /* a shifted system t I + M is singular for a node t */
    SKF_ERR_QUAD_NOT_CONVERGED = 6,  /* adaptive quadrature passed ell_max */
    SKF_ERR_SKETCH_TOO_SMALL = 7,    /* s < 2m is required by the GMRES reduction */
    SKF_ERR_NOT_SUPPORTED = 8,       /* valid request this build does not implement */
    SKF_ERR_ZERO_RHS = 9,            /* ||b|| = 0: x is set to 0 */
    SKF_ERR_TIMEOUT = 10             /* a bounded device-side wait (grid barrier of the
                                        persistent Arnoldi kernel) ran out; results invalid */
} skf_status;

typedef enum { SKF_F64 = 0, SKF_F32 = 1, SKF_BF16 = 2 } skf_dtype;

typedef enum {
    /* zeta nonzeros +-1/sqrt(zeta) per column, one per row stripe, rows and
       signs from SplitMix64 (see skf_sketch_create).  Not in the paper. */
    SKF_SKETCH_SPARSE_SIGN = 0,
    /* subsampled randomised Walsh-Hadamard transform (Sec. 2.2 and Sec. 5.1
       use the Fourier/DCT members of this family) */
    SKF_SKETCH_SRHT = 1,
    /* S = I (requires s == N): turns sFOM into FOM (Sec. 2, comment 1) */
    SKF_SKETCH_IDENTITY = 2,
    /* subsampled randomised discrete cosine transform, the sketch of the
       paper's experiments (Sec. 5.1, S = P F E with F a DCT) */
    SKF_SKETCH_SRDCT = 3
} skf_sketch_kind;

typedef enum { SKF_BORROW = 0, SKF_COPY = 1 } skf_copy_mode;

typedef enum {
    SKF_FUNC_INVSQRT = 0,       /* f(z) = z^(-1/2)                         */
    SKF_FUNC_LOG1P_OVER_Z = 1,  /* f(z) = log(1 + z) / z                   */
    SKF_FUNC_INV = 2,           /* f(z) = 1/z (single node t = 0): tests   */
    SKF_FUNC_INVPOW = 3,        /* f(z) = z^(-alpha), 0 < alpha < 1        */
    SKF_FUNC_EXP_NEG = 4,       /* f(z) = exp(-z): contour rule, see skf_func */
    SKF_FUNC_CUSTOM = 5         /* any Stieltjes measure: rules from skf_func::rule */
} skf_func_kind;

typedef enum { SKF_METHOD_SFOM = 0, SKF_METHOD_SGMRES = 1 } skf_method;

typedef struct skf_csr skf_csr;       /* opaque sparse operator handle */
typedef struct skf_sketch skf_sketch; /* opaque embedding handle        */

/* A Stieltjes function f(z) = int_0^inf (t + z)^-1 dmu(t) (Sec. 1) given by
 * its quadrature family.  The rule for order ell (host-generated) is
 *   INVSQRT / INVPOW: Gauss-Jacobi(-alpha, alpha-1) (Chebyshev for alpha =
 *     1/2) in x, t = scale (1-x)/(1+x)  (Sec. 5.1 uses scale = 1),
 *     w = (sin(alpha pi)/pi) 2 scale^(1-alpha) omega / (1+x) with the
 *     Gauss-Jacobi weights omega (for alpha != 1/2: Golub-Welsch, nodes by
 *     Sturm bisection of the Jacobi matrix, weights from its eigenvectors'
 *     first components; orders up to 1024),
 *   LOG1P_OVER_Z: Gauss-Legendre in x, t = 1 + scale (1-x)/(1+x),
 *   INV: t = 0, w = 1.
 *   EXP_NEG (not a Stieltjes function; Algorithm 2 with a fixed contour):
 *     Cauchy's formula in the pole variable t = -z, f(A) b =
 *     (1/(2 pi i)) oint f(-t) (t I + A)^{-1} b dt, on the parabola
 *     t(zeta) = a - c zeta^2 + i zeta (Sec. 5.2) with a = alpha and
 *     c = scale; it must enclose -Lambda (the negated spectrum and Ritz
 *     values: every -lambda left of the parabola).  Trapezoidal rule in zeta
 *     on [0, L], c L^2 = 37, h = L / (ell - 1), weights of zeta > 0 doubled
 *     (the conjugate half, real A and b), f(A) b = Re sum_k w_k (t_k I +
 *     A)^{-1} b with t_k = t(k h), w_k = (2 - [k = 0]) h e^{t_k}
 *     (i - 2 c k h) / (2 pi i).  Complex nodes: the node systems are solved
 *     through their real 2m x 2m form (requires m <= 256, ell1 >= 2).
 *   CUSTOM: the measure is the caller's, passed as a closure: for each order
 *     ell of the adaptive schedule (Sec. 4.1) the library calls
 *     rule(ell, t, w, ctx) on the calling host thread, during skf_solve and
 *     before any of its work is enqueued; the callback fills the host arrays
 *     t[ell] (nodes, t_i >= 0) and w[ell] (weights) of a rule with
 *     f(z) ~= sum_i w_i / (t_i + z) and returns 0 (nonzero: the call fails
 *     with SKF_ERR_NOT_SUPPORTED).  The rules of a (rule, ctx, schedule)
 *     triple are generated once and kept on the device for the life of the
 *     process: a different measure needs a different rule function or ctx
 *     pointer.  The library evaluates sFOM through the whitened quadrature
 *     form (eq. (sFOM) with the nodes), so no scalar f is needed.
 * If n_nodes > 0 the host arrays nodes/weights are used as the only rule
 * (no adaptivity; real rules only). */
typedef struct {
    skf_func_kind kind;
    double alpha;           /* exponent for SKF_FUNC_INVPOW (0 < alpha < 1); vertex a for EXP_NEG */
    double scale;           /* c > 0 of the Moebius map      */
    int32_t n_nodes;        /* explicit rule length, 0 = adaptive family */
    const double *nodes;    /* host, n_nodes t_i >= 0 */
    const double *weights;  /* host, n_nodes w_i      */
    int (*rule)(int32_t ell, double *t, double *w, void *ctx);   /* CUSTOM only */
    void *ctx;              /* passed to rule unchanged */
} skf_func;

/* Method parameters (inputs of Algorithms 1 and 2). */
typedef struct {
    int32_t m;              /* Krylov dimension, 1 <= m < s              */
    int32_t k;              /* truncation length of MGS, 1 <= k <= 16    */
    skf_dtype basis_dtype;  /* storage of V_m: F64 (F64 matrix values), or F32
                               or BF16 (F32 matrix values; FP32 arithmetic in
                               the Arnoldi process, FP64 tail).  F32: every
                               sketch kind; BF16: sparse-sign and identity.
                               skf_plan_basis_precision picks F32 or F64
                               per problem                                 */
    int32_t ell1, ell2;     /* first two quadrature orders (Sec. 4.1)    */
    int32_t ell_max;        /* give up past this order                   */
    double tol;             /* relative tolerance ||q1-q2|| <= tol ||q2|| */
    /* Sketched stopping criterion (Sec. 4.3), off when check_every = 0.
     * At every p = d, 2d, ... < m (d = check_every) the approximant f_p of
     * the leading p basis columns is formed in sketched form only (S f_p =
     * S V_p y_p, no N-vector) and compared with the previous checkpoint:
     *   est_p = ||S V_p (y_p - [y_{p-d}; 0])|| / sqrt(1 - eps)
     *           / (||S V_p y_p|| / sqrt(1 + eps)),
     * eps = max_{j<p} | ||S v_j||^2 - 1 |.  The first p with est_p <= stop_tol
     * ends the Arnoldi process there (m_eff = p) and f_p is returned; the
     * decision is taken on the device, so the call still needs no host
     * synchronisation.  Each checkpoint costs one dense tail (whitening QR
     * and quadrature) of order p. */
    int32_t check_every;
    double stop_tol;
    /* Two-pass truncated Arnoldi (Sec. 4.2) when nonzero: the first pass
     * keeps only the k + 2 most recent basis vectors (a ring; memory
     * N (k + 2) instead of N m) while it builds S V_m and S A V_m; after the
     * tail, a second pass repeats the same recurrence and accumulates
     * f = sum_j y_j v_j as each vector appears.  Twice the products with A.
     * The recurrence is deterministic, so the result equals the one-pass
     * result of the two-kernel form of the Arnoldi process (bit for bit with
     * an F64 basis; for F32/BF16 the one-pass recombination sums in
     * double-float, this one in FP64); the two-pass and stopping modes run
     * that form, and the persistent form that a plain F64 solve takes (see
     * skf_set_arnoldi_mode) gives the same approximant to rounding. */
    int32_t two_pass;
    /* Whitening check (Sec. 2.1 uses R^{-1}; reading of the survey: beyond
     * cond(R) ~ 1e12 in FP64 report ill-conditioning): info->status becomes
     * SKF_ERR_ILL_CONDITIONED when the estimate of cond(R) (skf_info::cond_est)
     * exceeds cond_max; x is still computed.  0 selects 1e12; a negative value
     * (or +inf) turns the test off (an exactly singular R is still reported). */
    double cond_max;
} skf_params;

/* Device-written result record.  Place it in memory the device can write
 * (cudaMalloc, or cudaHostAlloc/cudaHostRegister'd host memory) and read it
 * after synchronising the stream. */
typedef struct {
    int32_t status;         /* skf_status of the numerical outcome        */
    int32_t m_eff;          /* basis columns built (< m after breakdown)  */
    int32_t breakdown;      /* 1 if ||w|| <= 1e-12 ||A v_j|| stopped the recurrence */
    int32_t ell;            /* accepted quadrature order                  */
    double quad_err;        /* ||q_ell1 - q_ell2|| / ||q_ell2|| at acceptance */
    double beta;            /* ||b||                                      */
    double eps_est;         /* max_j | ||S v_j||^2 - 1 | (Sec. 4.3)       */
    double rdiag_ratio;     /* min |R_jj| / max |R_jj| of the whitening QR */
    int32_t nodes_fp64;     /* quadrature-node solves that needed the FP64
                               Cholesky factor (the FP32 factor with FP64
                               refinement did not converge for them)      */
    int32_t stop_m;         /* p at which the stopping criterion ended the
                               process, 0 if it did not (or was off)      */
    double err_est;         /* last relative estimate est_p (Sec. 4.3), 0
                               if no two checkpoints were compared        */
    double cond_est;        /* estimate of cond(R) = ||R|| ||R^{-1}|| of the
                               whitening factor: largest column norm times a
                               LINPACK-style ||R^{-1}|| estimate, at least
                               max|R_jj| / min|R_jj|                       */
} skf_info;

/* ---------------------------------------------------------------- misc */
const char *skf_last_error(void);
const char *skf_status_string(skf_status s);
int32_t skf_version(void);     /* major*10000 + minor*100 + patch */
/* Number of CUDA kernel launches this library has issued since it was
 * loaded, counted on the host at launch time (a diagnostic for profilers and
 * benchmarks; no device work). */
int64_t skf_kernel_launch_count(void);

/* skf_set_arnoldi_mode: which form of the FP64 Arnoldi process the library
 * launches (process-wide; a tuning and testing switch, results agree to
 * rounding between the forms):
 *   0  automatic (default): the persistent form where it applies, else the
 *      two-kernel form;
 *   1  the two-kernel form only: per step one SpMV launch and one update
 *      launch (programmatic dependents), any k, sketch kind and size;
 *   2  the persistent form only, SKF_ERR_NOT_SUPPORTED where it does not
 *      apply.
 * The persistent form runs all m steps of Algorithm 2 in one cooperative
 * launch, one CTA per SM, each CTA keeping its rows of the window vectors
 * and of A v_j in shared memory.  It applies to an F64 basis (and to an F32
 * basis with k <= 2 and slices at most 7 wide, N up to about 2e6) with a
 * sparse-sign sketch, k <= 4, one-pass storage without the stopping
 * criterion, and (k + 1) * ceil(N / SMs) * 8 bytes (plus the sketch bins)
 * within the per-CTA shared memory (N up to about 1.1e6 at k = 2 on a
 * 152-SM GB300); for k <= 2 and slices at most 7 wide it also runs with
 * A v_j in global memory (L2) when only the k window vectors fit (N up to
 * about 1.6e6).  Its grid barriers wait at most about one second each and
 * then report SKF_ERR_TIMEOUT in skf_info::status.
 * Returns INVALID_ARG for another mode. */
skf_status skf_set_arnoldi_mode(int32_t mode);

/* skf_set_block_mode: form of skf_solve_block (process-wide; results are
 * bit-identical in both): 0 (default) the columns one after another,
 * 1 the lockstep form with one SpMM per step (see skf_solve_block).
 * Returns INVALID_ARG for another mode. */
skf_status skf_set_block_mode(int32_t mode);

/* skf_set_qr_mode: form of the whitening QR of [S V_m, S A V_m] in the tail
 * (process-wide; results agree to rounding):
 *   0  automatic (default): one cooperative launch, column q updated by CTA
 *      q mod G throughout, each step starting as soon as the owner of its
 *      pivot column has published it (bounded wait: SKF_ERR_TIMEOUT in
 *      skf_info::status if it runs out);
 *   1  one launch per Householder reflector.
 * Returns INVALID_ARG for another mode. */
skf_status skf_set_qr_mode(int32_t mode);

/* skf_fp64_peak: measured FP64 FMA throughput of the current device in
 * GFLOP/s (2 flops per FMA): two CTAs of 512 threads per SM, four
 * independent accumulations x += y b per thread (the operand pattern of a dot
 * product, the fastest FMA form measured on this part), 8192 iterations,
 * timed with events on `stream` after one warm-up launch (synchronises the
 * stream).  The denominator of the FP64 roofline fraction.
 * Errors: INVALID_ARG, OOM, CUDA. */
skf_status skf_fp64_peak(double *gflops, skf_stream_t stream);

/* skf_workspace_trim: return the device memory that the library's
 * workspace pools keep mapped between calls.  Each solve takes its
 * stream-ordered workspace (about 8 m N bytes for an F64 basis, plus O(s m)
 * and O(m^2) buffers) from a per-device pool that keeps freed blocks, so
 * that repeated solves re-use them; call this (after the streams that used
 * them have finished) to release them.  Errors: CUDA. */
skf_status skf_workspace_trim(void);

/* skf_set_tail_form: what the tail factors to whiten the sketched problem
 * (Sec. 3; process-wide; results agree to rounding):
 *   0  automatic (default): with an F64 basis the relation form, the QR of
 *      the s x (m+1) matrix [S V_m, S A v_m]: the sketched Arnoldi relation
 *      S A v_j = S V_m H(1:m, j) (j < m, eq. (2.1)) gives
 *      M = [R_11 H(1:m, 1:m-1), R(1:m, m+1)] R_11^{-1} and the sGMRES term
 *      orthogonal to S V_m, R(m+1, m+1) / R(m, m) e_m^T; the same with an F32
 *      basis (its H holds the FP32 coefficients its update applied, so the
 *      relation holds for the stored columns); with a BF16 basis (whose
 *      stored columns satisfy the relation only to BF16 precision) the full
 *      form;
 *   1  the full form: the QR of the s x 2m matrix [S V_m, S A V_m].
 * The stopping criterion's checkpoints always take the full form.
 * Returns INVALID_ARG for another form. */
skf_status skf_set_tail_form(int32_t form);

/* skf_barrier_selftest: failure-detection check of the bounded grid wait
 * used by the persistent Arnoldi kernel.  Launches `ctas` co-resident CTAs
 * (1 <= ctas <= SMs) that wait at a barrier no CTA can complete, giving up
 * after budget_cycles SM clock cycles (1e3 .. 1e10); the kernel then writes
 * SKF_ERR_TIMEOUT to *status_device (device int) and returns, leaving the
 * context usable.  Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
skf_status skf_barrier_selftest(int32_t ctas, int64_t budget_cycles, int32_t *status_device, skf_stream_t stream);

/* ------------------------------------------------------------ operator */
/* skf_create_csr: wrap or copy a CSR matrix A (Sec. 2.2 assumes a sparse A
 * with O(N) nonzeros; the matrix-vector product is line "w <- A v" of
 * Algorithm 2).
 *   n       rows = columns, 1 <= n < 2^31
 *   nnz     nonzeros, 0 <= nnz < 2^31
 *   rowptr  device int64[n+1], rowptr[0] = 0, nondecreasing, rowptr[n] = nnz
 *   colind  device int32[nnz], 0 <= colind < n (any order within a row)
 *   values  device F64 or F32 array [nnz] (vdtype)
 *   mode    SKF_BORROW keeps colind/values (they must outlive the handle);
 *           SKF_COPY copies them.  The row pointer is always copied (as int32).
 * Builds the row partition used by the kernels and max_i sum_j |a_ij|.
 * May synchronise `stream`.  Errors: INVALID_ARG, OOM, CUDA. */
skf_status skf_create_csr(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                          const void *values, skf_dtype vdtype, skf_copy_mode mode,
                          skf_stream_t stream, skf_csr **A_out);
skf_status skf_destroy_csr(skf_csr *A);
/* Host copy of the matrix's max absolute row sum (an upper bound for |lambda|). */
skf_status skf_csr_norm_inf(const skf_csr *A, double *out_host);

/* skf_csr_autotune: choose the operator's slice layout by timing.  The
 * kernels read A in SELL-32 slices; rows longer than a cut leave the slices
 * and are reduced in segments of at most 1024 entries (row split), and the
 * rows may be sorted by length inside windows of 256 rows (less padding for
 * irregular row lengths).  skf_create_csr picks cut 32, unsorted.  This call
 * builds each of six
 * candidates (cut 16, 32, 64; unsorted, then sorted), times m_probe steps of
 * the truncated Arnoldi process with sketch S, truncation k and basis type
 * `basis` on a fixed probe vector (the minimum of two runs after a warm-up;
 * m_probe <= 0 selects 8), and keeps the fastest layout in A.
 * times_us (nullable, host double[6]): microseconds per step of each
 * candidate in that order; choice (nullable, host): the index kept.
 * Synchronises `stream`; A must not be in use on another stream meanwhile.
 * Results of later solves change only by the order of the long rows' sums.
 * Errors: INVALID_ARG, OOM, CUDA, NOT_SUPPORTED (as skf_arnoldi_trunc). */
skf_status skf_csr_autotune(skf_csr *A, const skf_sketch *S, int32_t k, skf_dtype basis, int32_t m_probe,
                            double *times_us, int32_t *choice, skf_stream_t stream);

/* skf_csr_set_layout: rebuild A's slice layout with rows longer than `cut`
 * entries split off (cut >= 1) and sorted = 1 (sorted slices), 0 (unsorted)
 * or -1 (sorted when that saves over a fifth of the padding, the default).
 * Synchronises `stream`.  Errors: INVALID_ARG, OOM, CUDA. */
skf_status skf_csr_set_layout(skf_csr *A, int32_t cut, int32_t sorted, skf_stream_t stream);

/* -------------------------------------------------------------- sketch */
/* skf_sketch_create: draw the embedding S in R^{s x N} (Algorithm 1, line 1;
 * eq. (1.1)).  The sparse-sign pattern is expanded once on the device from
 * its definition below (2 zeta bytes per column, plus the largest number of
 * nonzeros one kernel row block puts into one row of S, which sizes the
 * fixed-point accumulators); this call synchronises `stream`.  Definitions
 * (identical to the CPU oracle's):
 *   word(seed, i) = mix64(seed + (i+1) * 0x9E3779B97F4A7C15) (SplitMix64,
 *     Steele, Lea & Flood 2014), mix64 = xor-shift-multiply finaliser with
 *     constants 0xBF58476D1CE4E5B9, 0x94D049BB133111EB, shifts 30, 27, 31.
 *   SPARSE_SIGN: stripes q = 0..zeta-1 cover rows [floor(q s/zeta),
 *     floor((q+1) s/zeta)); column c uses words c*W + w, W = ceil(zeta/4);
 *     stripe q reads u = 16-bit chunk (q mod 4) of word (q div 4); sign is
 *     negative iff u & 1; row = start_q + ((u >> 1) * size_q) >> 15.
 *     Requires 1 <= zeta <= s, s/zeta <= 32768.
 *   SRHT: S x = s^-1/2 (H E [x; 0])[P], N' = 2^ceil(log2 N), E_c = -1 iff
 *     word(seed, c) & 1, P = first s entries of a partial Fisher-Yates
 *     shuffle of [0, N') with word(mix64(seed), i).  Requires s <= N'.
 *   SRDCT: S x = sqrt(N/s) (F E x)[P], F the orthonormal DCT-II of order N
 *     ((F y)_k = a_k sum_n y_n cos(pi k (2n+1) / (2N)), a_0 = sqrt(1/N),
 *     a_k = sqrt(2/N)), E as for SRHT, P the first s entries of the same
 *     partial Fisher-Yates shuffle, of [0, N).  Requires s <= N.  When N has
 *     no prime factor above 7 it is applied through one FFT of length N/2
 *     (even N, real input packed) or N (odd N) in FP64, O(N log N) per
 *     vector (Makhoul's reordering; creation keeps e^{-2 pi i t/N}, t < N,
 *     16 N bytes); otherwise as s direct dot products against a table of
 *     cos(pi j / (2N)), j < 4N (32 N bytes, O(s N) work per vector).
 *   IDENTITY: requires s == N.
 * Errors: INVALID_ARG, OOM, CUDA, NOT_SUPPORTED. */
skf_status skf_sketch_create(skf_sketch_kind kind, int64_t n, int32_t s, int32_t zeta, uint64_t seed,
                             skf_stream_t stream, skf_sketch **S_out);
skf_status skf_sketch_destroy(skf_sketch *S);

/* skf_sketch_apply: SX = S X for X of N rows and ncols columns (xdtype F64
 * or F32, leading dimension ldx >= N); SX is F64 s x ncols, leading
 * dimension s.  The sparse-sign sum is accumulated in 64/128-bit fixed point
 * scaled by each column's max |x|, so the result is independent of the
 * launch configuration (deterministic) and exact up to one rounding per
 * input entry at 2^-50 of the column max.  SRHT is computed the same way:
 * the Walsh-Hadamard transform runs exactly in int64 on blocks of up to 4096
 * entries (H_{N'} = H_{N'/B} (x) H_B), inputs rounded at 2^-(62 - log2 B) of
 * the column max, and the block contributions to each sampled row are summed
 * exactly.  The SRHT is available for F64 X and, in the Arnoldi process and
 * the solvers, for an F64 or F32 basis.  SRDCT sums in FP64 in a fixed order
 * (deterministic, not exact); F64 X and an F64 or F32 basis, like the SRHT.
 * Errors: INVALID_ARG, OOM, CUDA. */
skf_status skf_sketch_apply(const skf_sketch *S, const void *X, skf_dtype xdtype, int64_t ldx,
                            int32_t ncols, double *SX, skf_stream_t stream);

/* skf_sketch_apply_noalloc: the same result as skf_sketch_apply for a
 * sparse-sign sketch and F64 X, computed without allocating any device
 * memory.  The paper has no counterpart; this entry point exists for callers
 * that cannot call cudaMalloc/cudaMallocAsync at the point of use (a runtime
 * that owns and budgets every device allocation, or a path that must leave
 * the allocator and its memory pools untouched): this call makes no allocator
 * or memory-pool call at all.  Its scratch is a fixed 4 MiB array
 * inside this library, which every GPU that loads the library keeps until
 * the process exits; it must hold G * ncols * (s + 1) doubles, G being the
 * kernels' CTA count (at most 2 per SM), otherwise the call returns
 * SKF_ERR_INVALID_ARG and says how much it would need.  The first call on a
 * device looks up that array's device address (once per device), so make the
 * first call before capturing the stream into a CUDA graph.  All calls on a
 * device share the array: calls whose kernels can overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Nothing needs clearing between calls: every scratch word a call reads is
 * written by that call first.  Errors: INVALID_ARG, NOT_SUPPORTED, CUDA. */
skf_status skf_sketch_apply_noalloc(const skf_sketch *S, const void *X, skf_dtype xdtype, int64_t ldx,
                                    int32_t ncols, double *SX, skf_stream_t stream);

/* -------------------------------------------------------------- basis */
/* skf_arnoldi_trunc: the basis generation of Algorithm 2 (k-truncated
 * modified Gram-Schmidt, Sec. 2.2) with the sketches S V_m, S A V_m built on
 * the fly (Sec. 2, comment 3).  Exactly m products with A are performed.
 *   b          device F64 [N] (bdtype must be SKF_F64 in this build)
 *   V, ldv     device basis storage, N x m, type basis_dtype (F64, or F32
 *              and BF16 with F32 matrix values);
 *              column j holds a positive multiple w_j of the basis vector:
 *              v_j = vscale[j] * V[:, j], vscale[j] = 1 / ||V[:, j]||.
 *   vscale     device F64 [m]
 *   SV, SAV    device F64 s x m (ld = s): S v_j and S A v_j
 *   H          device F64 (m+1) x m (ld = m+1), zero outside the band:
 *              H[i, j] = MGS coefficient h_ij for i in the window,
 *              H[j+1, j] = ||w||; the last column holds only the window
 *              coefficients' slots as zero (no m+1-st vector is formed).
 *   info       device skf_info (m_eff, breakdown, beta, eps_est) or NULL
 * Requirements: 1 <= m < s, m <= N, 1 <= k <= 16.  Errors: INVALID_ARG, OOM, CUDA. */
skf_status skf_arnoldi_trunc(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype,
                             int32_t m, int32_t k, skf_dtype basis_dtype, void *V, int64_t ldv,
                             double *vscale, double *SV, double *SAV, double *H, skf_info *info,
                             skf_stream_t stream);

/* ------------------------------------------------------------- solvers */
/* skf_solve: the full approximant.
 *   method SFOM:   f_hat = V_m R^{-1} sum_i w_i (t_i I + M)^{-1} c, the
 *                  whitened form of eq. (sFOM) (equal to the closed form
 *                  (sFOM''') up to the quadrature error, which the adaptive
 *                  rule controls)
 *   method SGMRES: f_tilde = V_m R^{-1} sum_i w_i (t_i Q + Z)^+ S b,
 *                  eq. (sGMRES) with the quadrature (4.1)
 * where S V_m = Q R (whitening, Sec. 2.1), Z = S A V_m R^{-1}, M = Q^T Z,
 * c = Q^T S b.  Orders follow Sec. 4.1: ell1, ell2, then ell2 <-
 * floor(sqrt(2) ell2) until ||q_ell1 - q_ell2|| <= tol ||q_ell2|| or
 * ell_max is passed (info->status = QUAD_NOT_CONVERGED, x from the last
 * order).  Requires s >= 2m for SGMRES and m <= 512 (dense tail).
 * Branch cut (Sec. 2.3, Sec. 5.4): when M has an eigenvalue on the branch
 * cut of f (real and <= 0 for z^-alpha, <= -1 for log(1+z)/z) the sFOM
 * approximant (sFOM''') is undefined; its quadrature form then has a pole of
 * the integrand on the integration path, which info->status reports as
 * SKF_ERR_BRANCH_CUT (a node system singular to working precision) or
 * SKF_ERR_QUAD_NOT_CONVERGED (the rule does not settle), with x from the
 * last order.  sGMRES solves least-squares problems, which stay defined.
 *   b  device F64 [N];   x  device F64 [N] (output)
 *   workspace is taken stream-ordered from the library's pool (cached
 *   between calls, see skf_workspace_trim) and released before return; under
 *   stream capture it comes from the graph's memory nodes, so the call can be
 *   captured into a CUDA graph.
 * Errors: INVALID_ARG, OOM, CUDA, SKETCH_TOO_SMALL, NOT_SUPPORTED. */
skf_status skf_solve(skf_method method, const skf_csr *A, const skf_sketch *S, const void *b,
                     skf_dtype bdtype, const skf_func *f, const skf_params *p, void *x, skf_dtype xdtype,
                     skf_info *info, skf_stream_t stream);

/* Convenience forms of skf_solve. */
skf_status skf_sfom(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype,
                    const skf_func *f, const skf_params *p, void *x, skf_dtype xdtype, skf_info *info,
                    skf_stream_t stream);
skf_status skf_sgmres(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype,
                      const skf_func *f, const skf_params *p, void *x, skf_dtype xdtype, skf_info *info,
                      skf_stream_t stream);

/* skf_sfom_sgmres: both approximants of the same f(A) b, which share one
 * truncated Arnoldi process (V_m, S V_m, S A V_m and H are the same for the
 * two methods, Sec. 3): one Arnoldi run, one whitening QR (with M, cond(R)
 * and, in the relation form, gamma), then each method's quadrature tail, and
 * both recombinations x = V_m z in one pass over V_m.  Each result equals
 * the corresponding skf_sfom / skf_sgmres call bit for bit.  Arguments as
 * skf_solve (s >= 2m as for SGMRES); x_fom, x_gmres: device F64 [N];
 * info_fom, info_gmres nullable.  The stopping criterion (check_every > 0)
 * and the two-pass mode are not offered here (NOT_SUPPORTED).
 * Errors: INVALID_ARG, OOM, CUDA, SKETCH_TOO_SMALL, NOT_SUPPORTED. */
skf_status skf_sfom_sgmres(const skf_csr *A, const skf_sketch *S, const void *b, skf_dtype bdtype,
                           const skf_func *f, const skf_params *p, void *x_fom, void *x_gmres, skf_dtype xdtype,
                           skf_info *info_fom, skf_info *info_gmres, skf_stream_t stream);

/* ------------------------------------------------------------- batches */
/* One independent problem of a batch: the arguments of one skf_solve call. */
typedef struct {
    skf_method method;
    const skf_csr *A;
    const skf_sketch *S;
    const void *b;          /* device F64 [N] */
    skf_dtype bdtype;
    const skf_func *f;      /* host; read during the call only */
    const skf_params *p;    /* host; read during the call only */
    void *x;                /* device F64 [N] (output) */
    skf_dtype xdtype;
    skf_info *info;         /* device-writable, or NULL */
} skf_problem;

/* skf_solve_block: f(A) b_q for a block B = [b_1 .. b_nrhs] of right-hand
 * sides on one operator, with one sketch, one f, one parameter set and one
 * method (Algorithm 2 and the tail of skf_solve for every column; the paper
 * solves one right-hand side at a time).  B and X are device F64 N x nrhs,
 * column q at B + q ldb and X + q ldx (ldb, ldx >= N); info is a device
 * array of nrhs skf_info or NULL.  Every column's result is bit-identical to
 * the skf_solve call for it.  By default the columns are solved one after
 * another.  skf_set_block_mode(1) selects the lockstep form for an F32 basis
 * with one pass and no stopping criterion: the nrhs Arnoldi processes advance
 * together and each step reads A once per group of four right-hand sides (an
 * SpMM: the products of a chunk of A with the four w_j share one load of the
 * chunk); each process keeps its own update, sketch partials and tail.  It
 * applies to slices at most 8 wide without a row split, sparse-sign sketches
 * with zeta <= 8 and k <= 2 (otherwise, and for other basis types, the
 * columns go one after another).  Measured on a GB300 it is not faster than
 * the columns one after another for 7-point stencils (0.96-0.98x at
 * N = 2.4M and 16.8M): with one row per thread in 1024-thread CTAs (64
 * registers) the four columns' gathers cannot all be in flight, and the
 * kernel waits on them (27% of the DRAM peak against 72% for one column).
 * Device memory: the workspace of all nrhs processes at once in the lockstep
 * form (V_m in F32 and the sketches per column).  Errors: as skf_solve;
 * INVALID_ARG also for nrhs < 0 or ld < N. */
skf_status skf_solve_block(skf_method method, const skf_csr *A, const skf_sketch *S, const double *B, int64_t ldb,
                           int32_t nrhs, const skf_func *f, const skf_params *p, double *X, int64_t ldx,
                           skf_info *info, skf_stream_t stream);

/* skf_solve_batched: nprob independent f(A)b problems (each one exactly the
 * approximant skf_solve computes for its arguments; the paper solves one
 * f(A)b at a time, batching is a throughput form of the same computation).
 * Problems may share operators and sketches and may differ in N, m, k, s,
 * f and method.  The problems are spread over `lanes` (1..16) internal CUDA
 * streams that fork from `stream` and join it again, longest estimated work
 * first onto the least-loaded lane, so that the kernels of small problems
 * and the latency-bound tails run side by side on the GPU.  Every problem's
 * result is bit-identical to the result of its own skf_solve call (the
 * kernels' reductions have a fixed order).
 *   All problems are validated before anything is enqueued: on an argument
 *   error nothing runs and the message names the problem's index.
 *   Work is ordered after earlier work on `stream`, and later work on
 *   `stream` waits for all of it, so the whole call can be captured into
 *   one CUDA graph and replayed as one launch.  The first call on a device
 *   creates the lane streams and the first use of a quadrature rule uploads
 *   it (both synchronous, host-side): make one call outside capture first.
 *   Calls from several host threads are serialised inside the library.
 *   Outputs x must not alias each other or any input.
 *   Device memory: each running problem holds the workspace of its
 *   skf_solve (V_m and the sketches), so up to `lanes` of them are live.
 * Errors: INVALID_ARG (also nprob < 0, lanes outside 1..16), OOM, CUDA,
 *   SKETCH_TOO_SMALL, NOT_SUPPORTED. */
skf_status skf_solve_batched(int32_t nprob, const skf_problem *probs, int32_t lanes, skf_stream_t stream);

/* skf_plan_basis_precision: per problem, whether an FP32 Krylov basis is
 * expected to stay within `tol` (relative 2-norm) of the FP64-basis result.
 * This is the precision policy of the batched form; the paper has no
 * counterpart (it stores every basis in double precision).  Reasoning: an
 * FP32 basis perturbs every stored vector by a relative 2^-24, and the
 * approximant, computed from the sketched basis S V_m through its whitening
 * S V_m = Q R (Sec. 2.1, Sec. 3), moves by about 2^-24 cond(R); the rule is
 * FP32 iff cond(R) 2^-24 <= tol.  cond(R) is taken from a pilot: for each
 * distinct operator A among `probs`, the problem with the largest m runs
 * its Arnoldi process (its sketch, b, k and basis dtype, F64 or F32), and
 * for every problem r on that operator the whitening of the pilot's
 * leading m_r columns gives the estimate skf_info::cond_est describes (the
 * condition number of a sketched Krylov basis is a property of A, k and m
 * far more than of b or of the sketch's seed).  Outputs (host): cond_host[r]
 * and f32_host[r] (1: FP32 basis, 0: FP64).  The problems are validated as
 * by skf_solve_batched; their x and info are not touched.  Synchronises
 * `stream`.  Errors: INVALID_ARG, NOT_SUPPORTED (a BF16 pilot), OOM, CUDA,
 * SKETCH_TOO_SMALL. */
skf_status skf_plan_basis_precision(int32_t nprob, const skf_problem *probs, double tol, double *cond_host,
                                    int32_t *f32_host, skf_stream_t stream);

/* skf_quadrature_rule: host copy of the rule of order ell for f (the same
 * nodes and weights the solvers use).  t_host, w_host: host double[ell].
 * NOT_SUPPORTED for EXP_NEG (complex rule: skf_quadrature_rule_c). */
skf_status skf_quadrature_rule(const skf_func *f, int32_t ell, double *t_host, double *w_host);
/* skf_quadrature_rule_c: the same with real and imaginary parts (host
 * double[ell] each); for the real rules the imaginary parts are zero. */
skf_status skf_quadrature_rule_c(const skf_func *f, int32_t ell, double *t_re, double *t_im, double *w_re,
                                 double *w_im);

#ifdef __cplusplus
}
#endif
#endif /* SKF_H */
