"""Reference values of f(A) b (the "exact" result the approximants aim at).

* dense: f(A) b by Schur-based dense routines (sqrtm, logm,
  fractional_matrix_power), for N up to a few thousand;
* shifted: sum_i w_i (t_i I + A)^{-1} b with sparse LU per node (Stieltjes
  quadrature of Sec. 1), for moderate N; accurate to the rule's error.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import quadrature as quad


def fAb_dense(A: np.ndarray, b: np.ndarray, func: str, alpha: float = 0.5) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    if func == "invsqrt":
        return np.real(np.linalg.solve(sla.sqrtm(A), b))
    if func == "invpow":
        return np.real(sla.fractional_matrix_power(A, -alpha) @ b)
    if func == "log1p_over_z":
        L = sla.logm(np.eye(A.shape[0]) + A)
        return np.real(np.linalg.solve(A, L @ b))
    if func == "inv":
        return np.linalg.solve(A, b)
    if func == "exp_neg":
        return sla.expm(-A) @ b
    raise ValueError(func)


def fAb_shifted(A, b: np.ndarray, func: str, c_scale: float, ell: int) -> np.ndarray:
    A = sp.csc_matrix(A)
    N = A.shape[0]
    t, w = quad.rule(func, ell, c_scale)
    x = np.zeros(N)
    I = sp.identity(N, format="csc")
    for ti, wi in zip(t, w):
        x += wi * spla.splu((A + ti * I).tocsc()).solve(b)
    return x
