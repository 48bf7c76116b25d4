"""Python binding of the GB300 sketched-Krylov f(A)b library (include/skf.h).

Argument marshalling only: every computation runs in the CUDA kernels of
``libskf.so`` (built in-tree by ``paper_2208_11447_gb300.build``).  Tensors are
torch CUDA tensors; the CUDA stream is torch's current stream unless one is
given.  There is no CPU fallback: if the shared library is missing or cannot
be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libskf.so")

# enums of include/skf.h
F64, F32, BF16 = 0, 1, 2
SPARSE_SIGN, SRHT, IDENTITY, SRDCT = 0, 1, 2, 3
BORROW, COPY = 0, 1
INVSQRT, LOG1P_OVER_Z, INV, INVPOW = 0, 1, 2, 3
SFOM, SGMRES = 0, 1
STATUS = {0: "SKF_OK", 1: "SKF_ERR_INVALID_ARG", 2: "SKF_ERR_CUDA", 3: "SKF_ERR_OOM",
          4: "SKF_ERR_ILL_CONDITIONED", 5: "SKF_ERR_BRANCH_CUT", 6: "SKF_ERR_QUAD_NOT_CONVERGED",
          7: "SKF_ERR_SKETCH_TOO_SMALL", 8: "SKF_ERR_NOT_SUPPORTED", 9: "SKF_ERR_ZERO_RHS",
          10: "SKF_ERR_TIMEOUT"}
# Arnoldi forms of skf_set_arnoldi_mode
ARNOLDI_AUTO, ARNOLDI_TWO_KERNEL, ARNOLDI_PERSISTENT = 0, 1, 2
EXP_NEG, CUSTOM = 4, 5
FUNC_KIND = {"invsqrt": INVSQRT, "log1p_over_z": LOG1P_OVER_Z, "inv": INV, "invpow": INVPOW, "exp_neg": EXP_NEG,
             "custom": CUSTOM}
_DTYPE = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}


class SkfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


# int rule(int32_t ell, double *t, double *w, void *ctx) of a custom Stieltjes measure
RULE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class Func(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("alpha", ctypes.c_double), ("scale", ctypes.c_double),
                ("n_nodes", ctypes.c_int32), ("nodes", ctypes.POINTER(ctypes.c_double)),
                ("weights", ctypes.POINTER(ctypes.c_double)), ("rule", RULE_FN), ("ctx", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("k", ctypes.c_int32), ("basis_dtype", ctypes.c_int),
                ("ell1", ctypes.c_int32), ("ell2", ctypes.c_int32), ("ell_max", ctypes.c_int32),
                ("tol", ctypes.c_double), ("check_every", ctypes.c_int32), ("stop_tol", ctypes.c_double),
                ("two_pass", ctypes.c_int32), ("cond_max", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("m_eff", ctypes.c_int32), ("breakdown", ctypes.c_int32),
                ("ell", ctypes.c_int32), ("quad_err", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps_est", ctypes.c_double), ("rdiag_ratio", ctypes.c_double),
                ("nodes_fp64", ctypes.c_int32), ("stop_m", ctypes.c_int32), ("err_est", ctypes.c_double),
                ("cond_est", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["status_name"] = STATUS.get(self.status, str(self.status))
        return d


class Problem(ctypes.Structure):
    """skf_problem: the arguments of one skf_solve call inside a batch."""
    _fields_ = [("method", ctypes.c_int), ("A", ctypes.c_void_p), ("S", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("bdtype", ctypes.c_int), ("f", ctypes.POINTER(Func)), ("p", ctypes.POINTER(Params)),
                ("x", ctypes.c_void_p), ("xdtype", ctypes.c_int), ("info", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libskf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found: run `python -m paper_2208_11447_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.skf_last_error.restype = ctypes.c_char_p
        L.skf_status_string.restype = ctypes.c_char_p
        L.skf_status_string.argtypes = [ctypes.c_int]
        L.skf_version.restype = i32
        L.skf_kernel_launch_count.restype = i64
        L.skf_create_csr.argtypes = [i64, i64, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.skf_destroy_csr.argtypes = [vp]
        L.skf_csr_norm_inf.argtypes = [vp, ctypes.POINTER(dbl)]
        L.skf_sketch_create.argtypes = [ctypes.c_int, i64, i32, i32, u64, vp, ctypes.POINTER(vp)]
        L.skf_sketch_destroy.argtypes = [vp]
        L.skf_sketch_apply.argtypes = [vp, vp, ctypes.c_int, i64, i32, vp, vp]
        L.skf_sketch_apply_noalloc.argtypes = [vp, vp, ctypes.c_int, i64, i32, vp, vp]
        L.skf_arnoldi_trunc.argtypes = [vp, vp, vp, ctypes.c_int, i32, i32, ctypes.c_int, vp, i64, vp, vp, vp, vp,
                                        vp, vp]
        L.skf_solve.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_int, ctypes.POINTER(Func),
                                ctypes.POINTER(Params), vp, ctypes.c_int, vp, vp]
        L.skf_sfom.argtypes = L.skf_solve.argtypes[1:]
        L.skf_sfom_sgmres.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(Func), ctypes.POINTER(Params), vp, vp,
                                      ctypes.c_int, vp, vp, vp]
        L.skf_sgmres.argtypes = L.skf_solve.argtypes[1:]
        L.skf_quadrature_rule.argtypes = [ctypes.POINTER(Func), i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        L.skf_quadrature_rule_c.argtypes = [ctypes.POINTER(Func), i32] + [ctypes.POINTER(dbl)] * 4
        L.skf_solve_batched.argtypes = [i32, ctypes.POINTER(Problem), i32, vp]
        L.skf_set_arnoldi_mode.argtypes = [i32]
        L.skf_set_qr_mode.argtypes = [i32]
        L.skf_set_tail_form.argtypes = [i32]
        L.skf_workspace_trim.argtypes = []
        L.skf_fp64_peak.argtypes = [ctypes.POINTER(dbl), vp]
        L.skf_csr_autotune.argtypes = [vp, vp, i32, ctypes.c_int, i32, ctypes.POINTER(dbl), ctypes.POINTER(i32), vp]
        L.skf_csr_set_layout.argtypes = [vp, i32, i32, vp]
        L.skf_barrier_selftest.argtypes = [i32, i64, vp, vp]
        L.skf_plan_basis_precision.argtypes = [i32, ctypes.POINTER(Problem), dbl, ctypes.POINTER(dbl),
                                               ctypes.POINTER(i32), vp]
        L.skf_set_block_mode.argtypes = [i32]
        L.skf_solve_block.argtypes = [ctypes.c_int, vp, vp, vp, i64, i32, ctypes.POINTER(Func),
                                      ctypes.POINTER(Params), vp, i64, vp, vp]
        for name in ["skf_create_csr", "skf_destroy_csr", "skf_csr_norm_inf", "skf_sketch_create",
                     "skf_sketch_destroy", "skf_sketch_apply", "skf_sketch_apply_noalloc", "skf_arnoldi_trunc",
                     "skf_solve", "skf_solve_batched", "skf_sfom", "skf_sfom_sgmres",
                     "skf_sgmres", "skf_quadrature_rule", "skf_quadrature_rule_c", "skf_set_arnoldi_mode",
                     "skf_set_qr_mode", "skf_set_tail_form", "skf_workspace_trim", "skf_fp64_peak", "skf_csr_autotune", "skf_csr_set_layout",
                     "skf_barrier_selftest", "skf_plan_basis_precision", "skf_solve_block", "skf_set_block_mode"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise SkfError(st, lib().skf_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Csr:
    """Handle of skf_create_csr; keeps the tensors it borrows alive."""

    def __init__(self, rowptr: torch.Tensor, colind: torch.Tensor, values: torch.Tensor, copy: bool = False,
                 stream=None):
        assert rowptr.is_cuda and rowptr.dtype == torch.int64 and rowptr.is_contiguous()
        assert colind.is_cuda and colind.dtype == torch.int32 and colind.is_contiguous()
        assert values.is_cuda and values.dtype in _DTYPE and values.is_contiguous()
        self.n = rowptr.numel() - 1
        self.nnz = colind.numel()
        self._keep = (rowptr, colind, values)
        h = ctypes.c_void_p()
        _check(lib().skf_create_csr(self.n, self.nnz, _ptr(rowptr), _ptr(colind), _ptr(values),
                                    _DTYPE[values.dtype], COPY if copy else BORROW, _stream(stream),
                                    ctypes.byref(h)))
        self.handle = h

    def norm_inf(self) -> float:
        v = ctypes.c_double()
        _check(lib().skf_csr_norm_inf(self.handle, ctypes.byref(v)))
        return v.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.skf_destroy_csr(self.handle)
            self.handle = None


def create_csr(rowptr, colind, values, copy=False, stream=None) -> Csr:
    return Csr(rowptr, colind, values, copy, stream)


class Sketch:
    """Handle of skf_sketch_create."""

    def __init__(self, kind: int, n: int, s: int, zeta: int = 8, seed: int = 13, stream=None):
        h = ctypes.c_void_p()
        _check(lib().skf_sketch_create(kind, n, s, zeta, seed & ((1 << 64) - 1), _stream(stream), ctypes.byref(h)))
        self.handle, self.kind, self.n, self.s, self.zeta, self.seed = h, kind, n, s, zeta, seed

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.skf_sketch_destroy(self.handle)
            self.handle = None


def sketch_create(kind, n, s, zeta=8, seed=13, stream=None) -> Sketch:
    return Sketch(kind, n, s, zeta, seed, stream)


def _column_major(X: torch.Tensor) -> torch.Tensor:
    """(ncols, N) view whose rows are the columns of X, contiguous; no copy when
    X (N,) or (N, ncols) already stores its columns one after another."""
    Xc = X.reshape(X.shape[0], -1)
    Xt = Xc.t()
    return Xt if Xt.is_contiguous() else Xt.contiguous()


def sketch_apply(S: Sketch, X: torch.Tensor, SX: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """SX = S X for X of shape (N,) or (N, ncols).  The C ABI reads X column-major
    (column c at offset c*N); a tensor already laid out that way (X.t() contiguous,
    as for X = Y.t() with Y contiguous) is passed as it is, any other is copied
    into that order first."""
    Xcm = _column_major(X)
    ncols = Xcm.shape[0]
    if SX is None:
        SX = torch.empty((ncols, S.s), dtype=torch.float64, device=X.device)
    _check(lib().skf_sketch_apply(S.handle, _ptr(Xcm), _DTYPE[X.dtype], X.shape[0], ncols, _ptr(SX),
                                  _stream(stream)))
    out = SX.t()
    return out.reshape(S.s) if X.dim() == 1 else out


def sketch_apply_noalloc(S: Sketch, X: torch.Tensor, SX: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """As sketch_apply, through the allocation-free entry point.  The library
    call allocates nothing; this binding may: it creates SX when none is given,
    and copies X into column-major order when it is not already in it (pass a
    column-major X and an SX to allocate nothing at all)."""
    Xcm = _column_major(X)
    ncols = Xcm.shape[0]
    if SX is None:
        SX = torch.empty((ncols, S.s), dtype=torch.float64, device=X.device)
    _check(lib().skf_sketch_apply_noalloc(S.handle, _ptr(Xcm), _DTYPE[X.dtype], X.shape[0], ncols, _ptr(SX),
                                          _stream(stream)))
    out = SX.t()
    return out.reshape(S.s) if X.dim() == 1 else out


def new_info(device="cuda") -> torch.Tensor:
    return torch.zeros(ctypes.sizeof(Info), dtype=torch.uint8, device=device)


def read_info(buf: torch.Tensor) -> dict:
    raw = bytes(buf.cpu().numpy().tobytes())
    return Info.from_buffer_copy(raw).as_dict()


def arnoldi_trunc(A: Csr, S: Sketch, b: torch.Tensor, m: int, k: int, basis_dtype=torch.float64, info=None,
                  stream=None, ldv: int | None = None):
    """Returns V (m x N, row j = stored column w_j; a view of an m x ldv buffer
    when ldv is given), vscale (m), SV, SAV (m x s, row j = column j), H
    ((m) x (m+1): row j = column j of the (m+1) x m H)."""
    N = A.n
    dev = b.device
    ldv = N if ldv is None else ldv
    assert ldv >= N
    V = torch.empty((m, ldv), dtype=basis_dtype, device=dev)[:, :N]
    vscale = torch.empty(m, dtype=torch.float64, device=dev)
    SV = torch.empty((m, S.s), dtype=torch.float64, device=dev)
    SAV = torch.empty((m, S.s), dtype=torch.float64, device=dev)
    H = torch.empty((m, m + 1), dtype=torch.float64, device=dev)
    _check(lib().skf_arnoldi_trunc(A.handle, S.handle, _ptr(b), _DTYPE[b.dtype], m, k, _DTYPE[basis_dtype],
                                   _ptr(V), ldv, _ptr(vscale), _ptr(SV), _ptr(SAV), _ptr(H), _ptr(info),
                                   _stream(stream)))
    return V, vscale, SV, SAV, H


def make_func(kind: str, scale: float = 1.0, alpha: float = 0.5, nodes=None, weights=None, rule=None,
              ctx: int = 0) -> Func:
    """rule (kind "custom"): a Python callable rule(ell) -> (t, w), two
    sequences of ell floats with f(z) ~= sum_i w_i / (t_i + z); it is passed
    to the library as the skf_func::rule closure (kept alive by the Func).
    The library keeps the rules it generated per (rule, ctx) pointer pair:
    give a different measure a distinct ctx (any nonzero integer tag)."""
    f = Func()
    f.kind = FUNC_KIND[kind]
    f.alpha = alpha
    f.scale = scale
    if rule is not None:
        def _cb(ell, tp, wp, ctx):
            try:
                t, w = rule(int(ell))
                if len(t) != ell or len(w) != ell:
                    return 1
                for i in range(ell):
                    tp[i] = float(t[i])
                    wp[i] = float(w[i])
                return 0
            except Exception:
                return 1
        f._cb = RULE_FN(_cb)     # keep alive
        f.rule = f._cb
        f.ctx = ctx or None
    if nodes is not None:
        import numpy as np
        t = np.ascontiguousarray(nodes, dtype=np.float64)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        f.n_nodes = t.size
        f._t, f._w = t, w        # keep alive
        f.nodes = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        f.weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        f.n_nodes = 0
    return f


def make_params(m: int, k: int, basis_dtype=torch.float64, ell1=16, ell2=22, ell_max=1024, tol=1e-10,
                check_every: int = 0, stop_tol: float = 0.0, two_pass: bool = False, cond_max: float = 0.0) -> Params:
    """check_every = d > 0 turns on the sketched stopping criterion (Sec. 4.3)
    with relative tolerance stop_tol; m is then the largest dimension.
    two_pass: the two-pass truncated Arnoldi of Sec. 4.2 (basis memory
    N (k + 2) instead of N m, twice the products with A).
    cond_max: ILL_CONDITIONED above this estimate of cond(R) (0: 1e12,
    negative: no test)."""
    return Params(m, k, _DTYPE[basis_dtype], ell1, ell2, ell_max, tol, check_every, stop_tol, 1 if two_pass else 0,
                  cond_max)


def solve(method: int, A: Csr, S: Sketch, b: torch.Tensor, f: Func, p: Params, x: torch.Tensor | None = None,
          info=None, stream=None) -> torch.Tensor:
    if x is None:
        x = torch.empty_like(b)
    _check(lib().skf_solve(method, A.handle, S.handle, _ptr(b), _DTYPE[b.dtype], ctypes.byref(f), ctypes.byref(p),
                           _ptr(x), _DTYPE[x.dtype], _ptr(info), _stream(stream)))
    return x


def solve_block(method: int, A: Csr, S: Sketch, B: torch.Tensor, f: Func, p: Params, X: torch.Tensor | None = None,
                info=None, stream=None) -> torch.Tensor:
    """skf_solve_block for B of shape (nrhs, N) (row q = right-hand side q,
    i.e. the column-major N x nrhs block); returns X of the same shape.
    info: a buffer of nrhs skf_info (new_info_block) or None."""
    assert B.dim() == 2 and B.is_contiguous()
    if X is None:
        X = torch.empty_like(B)
    nrhs, N = B.shape
    _check(lib().skf_solve_block(method, A.handle, S.handle, _ptr(B), N, nrhs, ctypes.byref(f), ctypes.byref(p),
                                 _ptr(X), N, _ptr(info), _stream(stream)))
    return X


def new_info_block(nrhs: int, device="cuda") -> torch.Tensor:
    return torch.zeros((nrhs, ctypes.sizeof(Info)), dtype=torch.uint8, device=device)


def sfom(A, S, b, f, p, x=None, info=None, stream=None):
    return solve(SFOM, A, S, b, f, p, x, info, stream)


def sgmres(A, S, b, f, p, x=None, info=None, stream=None):
    return solve(SGMRES, A, S, b, f, p, x, info, stream)


def sfom_sgmres(A, S, b, f, p, x_fom=None, x_gmres=None, info_fom=None, info_gmres=None, stream=None):
    """skf_sfom_sgmres: both approximants from one Arnoldi process.  Returns
    (x_fom, x_gmres)."""
    if x_fom is None:
        x_fom = torch.empty_like(b)
    if x_gmres is None:
        x_gmres = torch.empty_like(b)
    _check(lib().skf_sfom_sgmres(A.handle, S.handle, _ptr(b), _DTYPE[b.dtype], ctypes.byref(f), ctypes.byref(p),
                                 _ptr(x_fom), _ptr(x_gmres), _DTYPE[x_fom.dtype], _ptr(info_fom), _ptr(info_gmres),
                                 _stream(stream)))
    return x_fom, x_gmres


def _problem_array(problems):
    arr = (Problem * len(problems))()
    for i, (method, A, S, b, f, p, x, info) in enumerate(problems):
        arr[i] = Problem(method, A.handle, S.handle, b.data_ptr(), _DTYPE[b.dtype], ctypes.pointer(f),
                         ctypes.pointer(p), x.data_ptr(), _DTYPE[x.dtype], info.data_ptr() if info is not None else 0)
    return arr


def solve_batched(problems, lanes: int = 4, stream=None):
    """skf_solve_batched.  problems: sequence of (method, A, S, b, f, p, x,
    info) with x a preallocated F64 tensor and info a buffer from new_info()
    or None.  Returns the list of x."""
    arr = _problem_array(problems)
    _check(lib().skf_solve_batched(len(problems), arr, lanes, _stream(stream)))
    return [q[6] for q in problems]


def plan_basis_precision(problems, tol: float, stream=None):
    """skf_plan_basis_precision: (cond, use_f32) per problem, two lists."""
    n = len(problems)
    arr = _problem_array(problems)
    cond = (ctypes.c_double * max(n, 1))()
    f32 = (ctypes.c_int32 * max(n, 1))()
    _check(lib().skf_plan_basis_precision(n, arr, tol, cond, f32, _stream(stream)))
    return [cond[i] for i in range(n)], [bool(f32[i]) for i in range(n)]


class BatchGraph:
    """A fixed batch of problems captured once into a CUDA graph.

    The constructor runs the batch once outside capture (this creates the
    library's lane streams and uploads the quadrature rules), then captures
    one skf_solve_batched call; replay() enqueues the whole batch as one
    graph launch on the current stream.  The tensors of `problems` must stay
    alive and in place: replays read b and write x where capture found them."""

    def __init__(self, problems, lanes: int = 4):
        self.problems = list(problems)
        self.lanes = lanes
        solve_batched(self.problems, lanes)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            solve_batched(self.problems, lanes)
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()

    @classmethod
    def autotune(cls, problems, candidates=(4, 8, 16)):
        """Capture the batch once per lane count, time one replay of each
        (after a warm one) with CUDA events, and keep the fastest.  Returns
        (graph, {lanes: ms})."""
        times, best = {}, None
        for lanes in candidates:
            g = cls(problems, lanes)
            g.replay()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            g.replay()
            ev1.record()
            ev1.synchronize()
            times[lanes] = ev0.elapsed_time(ev1)
            if best is None or times[lanes] < times[best.lanes]:
                best = g
            else:
                del g
        return best, times


def set_arnoldi_mode(mode: int) -> None:
    """skf_set_arnoldi_mode: ARNOLDI_AUTO, ARNOLDI_TWO_KERNEL or ARNOLDI_PERSISTENT."""
    _check(lib().skf_set_arnoldi_mode(mode))


class arnoldi_mode:
    """Context manager: run the enclosed calls with the given Arnoldi form,
    then return to the automatic choice."""

    def __init__(self, mode: int):
        self.mode = mode

    def __enter__(self):
        set_arnoldi_mode(self.mode)
        return self

    def __exit__(self, *exc):
        set_arnoldi_mode(ARNOLDI_AUTO)
        return False


def set_qr_mode(mode: int) -> None:
    """skf_set_qr_mode: 0 one cooperative launch (default), 1 one launch per reflector."""
    _check(lib().skf_set_qr_mode(mode))


class qr_mode:
    """Context manager: run the enclosed calls with the given QR form, then
    return to the default."""

    def __init__(self, mode: int):
        self.mode = mode

    def __enter__(self):
        set_qr_mode(self.mode)
        return self

    def __exit__(self, *exc):
        set_qr_mode(0)
        return False


class block_mode:
    """Context manager: skf_set_block_mode(mode) for the enclosed calls (1: the
    lockstep SpMM form of skf_solve_block), then back to the default 0."""

    def __init__(self, mode: int):
        self.mode = mode

    def __enter__(self):
        _check(lib().skf_set_block_mode(self.mode))
        return self

    def __exit__(self, *exc):
        _check(lib().skf_set_block_mode(0))
        return False


TAIL_AUTO, TAIL_FULL = 0, 1


AUTOTUNE_CANDIDATES = [{"cut": c, "sorted": s} for s in (False, True) for c in (16, 32, 64)]


def csr_autotune(A: "Csr", S: "Sketch", k: int, basis_dtype=torch.float64, m_probe: int = 8, stream=None) -> dict:
    """skf_csr_autotune: time the six slice layouts and keep the fastest in A.
    Returns {"choice": {...}, "times_us": [...per candidate]}."""
    t = (ctypes.c_double * 6)()
    ch = ctypes.c_int32(-1)
    _check(lib().skf_csr_autotune(A.handle, S.handle, k, _DTYPE[basis_dtype], m_probe, t, ctypes.byref(ch),
                                  _stream(stream)))
    return {"choice": dict(AUTOTUNE_CANDIDATES[ch.value]), "times_us": [float(x) for x in t]}


def csr_set_layout(A: "Csr", cut: int, sorted_: int = -1, stream=None) -> None:
    """skf_csr_set_layout: rows over `cut` entries split off; sorted_ 1, 0 or -1 (automatic)."""
    _check(lib().skf_csr_set_layout(A.handle, cut, sorted_, _stream(stream)))


def fp64_peak(stream=None) -> float:
    """skf_fp64_peak: measured FP64 FMA throughput in GFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(lib().skf_fp64_peak(ctypes.byref(v), _stream(stream)))
    return v.value


def workspace_trim() -> None:
    """skf_workspace_trim: release the workspace blocks the library keeps
    mapped between calls (synchronise the streams that used them first)."""
    _check(lib().skf_workspace_trim())


def set_tail_form(form: int) -> None:
    """skf_set_tail_form: 0 automatic (relation form with an F64 basis), 1 the
    QR of [S V_m, S A V_m]."""
    _check(lib().skf_set_tail_form(form))


class tail_form:
    """Context manager: run the enclosed calls with the given tail form, then
    return to the default."""

    def __init__(self, form: int):
        self.form = form

    def __enter__(self):
        set_tail_form(self.form)
        return self

    def __exit__(self, *exc):
        set_tail_form(TAIL_AUTO)
        return False


def barrier_selftest(ctas: int, budget_cycles: int, stream=None) -> int:
    """skf_barrier_selftest: returns the status the kernel wrote (after a
    stream synchronisation)."""
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    _check(lib().skf_barrier_selftest(ctas, budget_cycles, _ptr(st), _stream(stream)))
    return int(st.item())


def kernel_launch_count() -> int:
    return int(lib().skf_kernel_launch_count())


def quadrature_rule(f: Func, ell: int):
    import numpy as np
    t = np.empty(ell)
    w = np.empty(ell)
    _check(lib().skf_quadrature_rule(ctypes.byref(f), ell, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return t, w


def quadrature_rule_c(f: Func, ell: int):
    """Complex nodes and weights (t, w) of the rule of order ell (numpy complex)."""
    import numpy as np
    arrs = [np.empty(ell) for _ in range(4)]
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib().skf_quadrature_rule_c(ctypes.byref(f), ell, *[ptr(a) for a in arrs]))
    return arrs[0] + 1j * arrs[1], arrs[2] + 1j * arrs[3]


@dataclass
class DeviceOperator:
    """A CSR operator resident on the device plus its handle."""
    rowptr: torch.Tensor
    colind: torch.Tensor
    values: torch.Tensor
    csr: Csr


def upload_csr(rowptr, colind, values, device="cuda", dtype=None) -> DeviceOperator:
    """dtype: torch.float64 or torch.float32 for the stored values (default:
    that of `values`).  An F32 operator is what the FP32/BF16-basis path takes."""
    rp = torch.as_tensor(rowptr, dtype=torch.int64).to(device)
    ci = torch.as_tensor(colind, dtype=torch.int32).to(device)
    va = torch.as_tensor(values, dtype=dtype).to(device)
    return DeviceOperator(rp, ci, va, Csr(rp, ci, va))
