"""Sketched stopping criterion (Sec. 4.3).  Test infrastructure: plain FP64
NumPy, shared with nothing on the CUDA path.

The error of an iterate is estimated by the difference of two iterates d
steps apart, ||f_{m+d} - f_m||.  Both lie in K_{m+d}(A, b), on which S is an
eps-subspace embedding, so (eq. (sketched_err_est1))

    ||S(f_{m+d} - f_m)|| / sqrt(1 + eps)  <=  ||f_{m+d} - f_m||
                                          <=  ||S(f_{m+d} - f_m)|| / sqrt(1 - eps)

and with f_m = V_m y_m the upper side needs only sketched quantities
(eq. (sketched_err_est2)):

    ||f_{m+d} - f_m|| <= ||S V_{m+d} (y_{m+d} - [y_m; 0_d])|| / sqrt(1 - eps).

eps is unknown; Sec. 4.3 suggests tracking ||S v_j|| against ||v_j|| = 1 for
the basis vectors, which gives the lower estimate eps_hat = max_j
| ||S v_j||^2 - 1 | used here.  Reading (the paper is silent on it): the
factor 1/sqrt(1 - eps) is kept on the right-hand side of eq.
(sketched_err_est2), and the test is relative to the estimated norm of the
newer iterate, ||S f_{m+d}|| / sqrt(1 + eps).

solve_with_stopping runs the truncated Arnoldi process once up to m_max and
evaluates the estimate at p = d, 2d, ... on the leading p columns (the
recurrence is prefix-consistent: the first p columns of an m_max run are the
p-column basis); it returns the first iterate f_p whose estimate, comparing
f_p with f_{p-d}, meets the tolerance.
"""
from __future__ import annotations

import numpy as np

from . import sketched as osk
from .arnoldi import arnoldi_trunc


def eps_hat(SV: np.ndarray) -> float:
    """max_j | ||S v_j||^2 - 1 | over the columns of S V (v_j unit vectors)."""
    return float(np.max(np.abs(np.sum(SV * SV, axis=0) - 1.0))) if SV.size else 0.0


def sketched_difference(SV_full: np.ndarray, y_new: np.ndarray, y_old: np.ndarray) -> float:
    """||S V_{m+d} (y_{m+d} - [y_m; 0_d])|| for y_new of length m+d, y_old of length m."""
    dy = np.array(y_new, dtype=np.float64)
    dy[: y_old.size] -= y_old
    return float(np.linalg.norm(SV_full[:, : y_new.size] @ dy))


def error_estimate(SV_full: np.ndarray, y_new: np.ndarray, y_old: np.ndarray, eps: float):
    """(upper estimate of ||f_new - f_old||, estimated ||f_new||), eq. (sketched_err_est2)."""
    diff = sketched_difference(SV_full, y_new, y_old) / np.sqrt(1.0 - eps)
    norm_new = float(np.linalg.norm(SV_full[:, : y_new.size] @ y_new)) / np.sqrt(1.0 + eps)
    return diff, norm_new


def prefix_coefficients(ar: dict, Sb: np.ndarray, p: int, func: str, c_scale: float, method: str, tol_quad: float,
                        ell=None):
    """Coefficients y_p of the approximant built from the leading p columns."""
    W = osk.whiten(ar["SV"][:, :p], ar["SAV"][:, :p], Sb)
    if method == "sgmres":
        y, used = osk.sgmres_quadrature(W, func, c_scale, ell=ell, tol=tol_quad)
    elif method == "sfom_quad":
        y, used = osk.sfom_quadrature(W, func, c_scale, ell=ell, tol=tol_quad)
    else:
        raise ValueError(method)
    return y, used


def solve_with_stopping(A, b, func: str, m_max: int, k: int, S, c_scale: float, d: int, tol: float,
                        method: str = "sgmres", tol_quad: float = 1e-10, ell=None):
    """Returns (x, info): x = V_p y_p for the first checkpoint p (a multiple of
    d, p >= 2d) with est_p / norm_p <= tol, else the m_max iterate (checks
    at every multiple of d below m_max); info has p, the relative estimates by
    checkpoint and whether the criterion stopped the process."""
    ar = arnoldi_trunc(A, b, m_max, k, S)
    Sb = S @ np.asarray(b, dtype=np.float64)
    me = ar["m_eff"]
    prev = None
    history = []
    for p in range(d, me, d):
        y, _ = prefix_coefficients(ar, Sb, p, func, c_scale, method, tol_quad, ell)
        if prev is not None:
            eps = eps_hat(ar["SV"][:, :p])
            diff, nrm = error_estimate(ar["SV"], y, prev, eps)
            rel = diff / nrm
            history.append((p, rel))
            if rel <= tol:
                return ar["V"][:, :p] @ y, {"p": p, "stopped": True, "history": history, "y": y, "ar": ar}
        prev = y
    y, _ = prefix_coefficients(ar, Sb, me, func, c_scale, method, tol_quad, ell)
    return ar["V"] @ y, {"p": me, "stopped": False, "history": history, "y": y, "ar": ar}
