"""Named workloads: operator, right-hand side, function and method parameters.

Seeds: matrix/graph 11, right-hand side 12, sketch 13, batch layout 14.

``spectrum`` is a cheap interval [lam_lo, lam_hi] enclosing the real parts of
the field of values (lam_lo = smallest eigenvalue of the symmetric part,
lam_hi = max absolute row sum).  It only sets the scale ``c`` of the
quadrature rule, which is an input of both the oracle and the CUDA path.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .operators import convdiff_2d, convdiff_3d, powerlaw_graph_operator, gaussian_rhs, upwind_2d, CSR

SEEDS = {"matrix": 11, "rhs": 12, "sketch": 13, "batch": 14}


def laplacian_lambda_min(n: int, dims: int) -> float:
    h = 1.0 / (n + 1)
    return dims * (2.0 - 2.0 * math.cos(math.pi * h)) / (h * h)


def max_abs_row_sum(A: CSR) -> float:
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return float(np.bincount(rows, weights=np.abs(A.values.astype(np.float64)), minlength=A.n).max())


def quad_scale(func: str, lam_lo: float, lam_hi: float) -> float:
    """Scale c of the Moebius map t = c(1-x)/(1+x) (or 1 + c(1-x)/(1+x))."""
    if func == "invsqrt":
        return math.sqrt(lam_lo * lam_hi)
    if func == "log1p_over_z":
        return math.sqrt(1.0 + lam_hi)
    return 1.0


@dataclass
class Workload:
    name: str
    build: callable            # () -> CSR
    func: str                  # "invsqrt" | "log1p_over_z" | "inv"
    m: int
    k: int
    s: int
    zeta: int = 8
    value_dtype: str = "f64"
    basis_dtype: str = "f64"
    lam_lo: float | None = None   # if None, computed by the caller from the matrix
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def operator(self) -> CSR:
        A = self.build()
        if self.value_dtype == "f32":
            A = A.astype(np.float32)
        return A

    def rhs(self, N: int) -> np.ndarray:
        return gaussian_rhs(N, SEEDS["rhs"], normalize=True)


def _cd(dims, n, nu):
    if dims == 2:
        return lambda: convdiff_2d(n, nu)
    return lambda: convdiff_3d(n, nu)


WORKLOADS = {
    # 2D convection-diffusion, N = 1e4, FP64, z^{-1/2}
    "cd2d_n100": Workload("cd2d_n100", _cd(2, 100, (100.0, 50.0)), "invsqrt", m=40, k=2, s=160,
                          lam_lo=laplacian_lambda_min(100, 2)),
    # same operator at m = 240, s = 960 (sGMRES reaches the true f(A)b there)
    "cd2d_n100_m240": Workload("cd2d_n100_m240", _cd(2, 100, (100.0, 50.0)), "invsqrt", m=240, k=2,
                               s=960, lam_lo=laplacian_lambda_min(100, 2)),
    # 3D convection-diffusion, N = 1e6, ~7M nnz, FP64, log(1+z)/z
    "cd3d_n100": Workload("cd3d_n100", _cd(3, 100, (50.0, 50.0, 50.0)), "log1p_over_z", m=200, k=2,
                          s=800, lam_lo=laplacian_lambda_min(100, 3)),
    # precision study: 256^3 grid, FP32 values, FP32 or BF16 basis, z^{-1/2}
    "cd3d_n256_fp32": Workload("cd3d_n256_fp32", _cd(3, 256, (50.0, 50.0, 50.0)), "invsqrt", m=120,
                               k=2, s=480, value_dtype="f32", basis_dtype="f32",
                               lam_lo=laplacian_lambda_min(256, 3)),
    # mid-size FP32 step (N = 512,000; the batched workload's sizes), for profiles
    "cd3d_n80_fp32": Workload("cd3d_n80_fp32", _cd(3, 80, (50.0, 50.0, 50.0)), "invsqrt", m=20,
                              k=2, s=80, value_dtype="f32", basis_dtype="f32",
                              lam_lo=laplacian_lambda_min(80, 3)),
    # directed power-law graph, N = 4e6, FP32, k = 3, z^{-1/2}, 128 nodes
    "graph_n4m": Workload("graph_n4m", lambda: powerlaw_graph_operator(4_000_000, 2.1, 10.0, SEEDS["matrix"]),
                          "invsqrt", m=150, k=3, s=600, value_dtype="f32", basis_dtype="f32",
                          lam_lo=0.1, extra={"ell": 128}),
    # the same graph with rows carrying the power-law out-degrees (hubs of up
    # to ~1e5 entries: the row-split SpMV)
    "graph_n4m_t": Workload("graph_n4m_t", lambda: powerlaw_graph_operator(4_000_000, 2.1, 10.0, SEEDS["matrix"],
                                                                          transpose=True),
                            "invsqrt", m=150, k=3, s=600, value_dtype="f32", basis_dtype="f32",
                            lam_lo=0.1, extra={"ell": 128}),
    # the paper's own first experiment operator (upwind, D = 1e-3), n = 100
    "upwind_n100": Workload("upwind_n100", lambda: upwind_2d(100, 1e-3), "invsqrt", m=200, k=4, s=400,
                            lam_lo=None),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
