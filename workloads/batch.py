"""Seeded layout of the batched workload: several convection-diffusion
operators of uneven size and many right-hand sides spread unevenly over them.

Layout (all draws from PCG64 with the batch-layout seed):
  * n_mats operators alternate 2D / 3D (even index 2D).  N is log-uniform in
    [n_lo, n_hi] and rounded to the nearest n^2 (2D) or n^3 (3D).
  * Each velocity component nu_d is uniform in [10, 200].
  * Right-hand-side counts per operator: a Dirichlet(0.5) weight vector, then
    a multinomial of n_rhs - n_mats over it, plus one each (every operator
    gets at least one).
  * Per right-hand side: m uniform on {m_lo, ..., m_hi}, s = 4 m, its own
    sketch seed (sketch seed + r) and right-hand-side seed
    (rhs seed * 1000 + r), b ~ N(0, 1) normalised.
The operators' values are the FP32-rounded stencil coefficients (stored as
FP32 or, exactly, as FP64), so an FP64 and an FP32 solve see the same A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .configs import SEEDS, laplacian_lambda_min, max_abs_row_sum
from .operators import CSR, convdiff_2d, convdiff_3d, gaussian_rhs


@dataclass
class BatchMatrix:
    dims: int
    n: int             # grid points per direction
    nu: tuple

    @property
    def N(self) -> int:
        return self.n ** self.dims

    def operator(self) -> CSR:
        """The stencil with FP32-rounded values (returned as FP32)."""
        A = convdiff_2d(self.n, self.nu) if self.dims == 2 else convdiff_3d(self.n, self.nu)
        return A.astype(np.float32)

    def lam_lo(self) -> float:
        return laplacian_lambda_min(self.n, self.dims)


@dataclass
class BatchRhs:
    mat: int           # index of its operator
    m: int
    s: int
    sketch_seed: int
    rhs_seed: int

    def rhs(self, N: int) -> np.ndarray:
        return gaussian_rhs(N, self.rhs_seed, normalize=True)


@dataclass
class BatchLayout:
    mats: list
    rhs: list

    def summary(self) -> dict:
        return {"n_mats": len(self.mats), "n_rhs": len(self.rhs),
                "N": [m.N for m in self.mats], "dims": [m.dims for m in self.mats],
                "rhs_per_mat": [sum(1 for r in self.rhs if r.mat == i) for i in range(len(self.mats))],
                "sum_m": int(sum(r.m for r in self.rhs))}


def batch_layout(n_mats: int = 8, n_rhs: int = 64, n_lo: float = 1e5, n_hi: float = 4e6, m_lo: int = 50,
                 m_hi: int = 400, seed: int = SEEDS["batch"]) -> BatchLayout:
    if n_rhs < n_mats:
        raise ValueError("need at least one right-hand side per operator")
    rng = np.random.Generator(np.random.PCG64(seed))
    mats = []
    for i in range(n_mats):
        dims = 2 if i % 2 == 0 else 3
        N = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        n = max(3, int(round(N ** (1.0 / dims))))
        nu = tuple(float(v) for v in rng.uniform(10.0, 200.0, size=dims))
        mats.append(BatchMatrix(dims, n, nu))
    wts = rng.dirichlet(np.full(n_mats, 0.5))
    counts = rng.multinomial(n_rhs - n_mats, wts) + 1
    rhs = []
    r = 0
    for i in range(n_mats):
        for _ in range(int(counts[i])):
            m = int(rng.integers(m_lo, m_hi + 1))
            rhs.append(BatchRhs(i, m, 4 * m, SEEDS["sketch"] + r, SEEDS["rhs"] * 1000 + r))
            r += 1
    return BatchLayout(mats, rhs)


def quad_scale_invsqrt(A: CSR, lam_lo: float) -> float:
    """c = sqrt(lam_lo * lam_hi) of the z^{-1/2} rule, lam_hi = max row sum."""
    return math.sqrt(lam_lo * max_abs_row_sum(A))
