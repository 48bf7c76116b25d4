"""Sketched FOM and sketched GMRES approximants to f(A)b from the sketched
quantities S V_m, S A V_m, S b (Sec. 2 and Sec. 3).

Basis whitening (Sec. 2.1, eq. (sFOM''')): thin QR S V_m = Q R, then
Z = S A V_m R^{-1}, M = Q^T Z, c = Q^T S b; V_m R^{-1} is never formed.

* sFOM closed form (sFOM'''):   f_hat = V_m R^{-1} f(M) c
* sFOM by quadrature (eq. (sFOM) with the whitened quantities):
                                 f_hat ~= V_m R^{-1} sum_i w_i (t_i I + M)^{-1} c
* sGMRES (eq. (sGMRES), quadrature eq. (4.1)):
                                 f_tilde ~= V_m R^{-1} sum_i w_i (t_i Q + Z)^+ S b
Adaptive quadrature (Sec. 4.1): evaluate orders ell1 < ell2; while
||q_ell1 - q_ell2|| > tol, set ell1 <- ell2, ell2 <- floor(sqrt(2) ell2).
Reading: the test is relative, ||q_ell1 - q_ell2|| <= tol * ||q_ell2||, and
gives up (QuadNotConverged) once ell2 would exceed ell_max.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import quadrature as quad


class BranchCutError(ArithmeticError):
    pass


class QuadNotConverged(ArithmeticError):
    pass


def whiten(SV: np.ndarray, SAV: np.ndarray, Sb: np.ndarray):
    Q, R = np.linalg.qr(SV)
    Z = sla.solve_triangular(R, SAV.T, trans="T", lower=False).T   # Z R = SAV
    M = Q.T @ Z
    c = Q.T @ Sb
    return {"Q": Q, "R": R, "Z": Z, "M": M, "c": c, "Sb": Sb,
            "condR": float(np.linalg.cond(R))}


def matfunc_apply(func: str, M: np.ndarray, c: np.ndarray, alpha: float = 0.5) -> np.ndarray:
    """f(M) c for the principal branch, by Schur-based dense routines."""
    ev = np.linalg.eigvals(M)
    if func == "exp_neg":
        return sla.expm(-M) @ c
    if func in ("invsqrt", "invpow", "inv"):
        cut = -0.0
    elif func == "log1p_over_z":
        cut = -1.0
    else:
        raise ValueError(func)
    on_cut = (np.abs(ev.imag) <= 1e-12 * np.maximum(1.0, np.abs(ev))) & (ev.real <= cut)
    if np.any(on_cut):
        raise BranchCutError(f"eigenvalue of M on the branch cut: {ev[on_cut][:3]}")
    if func == "invsqrt":
        X = sla.sqrtm(M)
        u = np.linalg.solve(X, c)
    elif func == "invpow":
        u = sla.fractional_matrix_power(M, -alpha) @ c
    elif func == "log1p_over_z":
        L = sla.logm(np.eye(M.shape[0]) + M)
        u = np.linalg.solve(M, L @ c)
    else:
        u = np.linalg.solve(M, c)
    return np.real_if_close(u, tol=1e6).real


def adaptive(qfun, ell1: int, ell2: int, tol: float, ell_max: int):
    q1, q2 = qfun(ell1), qfun(ell2)
    while np.linalg.norm(q1 - q2) > tol * np.linalg.norm(q2):
        nxt = int(math.floor(math.sqrt(2.0) * ell2))
        if nxt > ell_max:
            raise QuadNotConverged(f"ell = {ell2} reached, next {nxt} > {ell_max}")
        q1, ell1, ell2 = q2, ell2, nxt
        q2 = qfun(ell2)
    return q2, ell2


def sfom_closed(W: dict, func: str, alpha: float = 0.5) -> np.ndarray:
    """Coefficients y with f_hat = V_m y (sFOM''')."""
    u = matfunc_apply(func, W["M"], W["c"], alpha)
    return sla.solve_triangular(W["R"], u, lower=False)


def sfom_quadrature(W: dict, func: str, c_scale: float, ell=None, ell1=16, ell2=22,
                    tol=1e-10, ell_max=1024, alpha: float = 0.5):
    M, cvec = W["M"], W["c"]
    m = M.shape[0]

    def q(ell_):
        t, w = quad.rule(func, ell_, c_scale, alpha)
        acc = np.zeros(m, dtype=np.result_type(t, w, np.float64))
        for ti, wi in zip(t, w):
            acc += wi * np.linalg.solve(ti * np.eye(m) + M, cvec)
        return acc.real   # complex contour nodes: the rule's real part (see quadrature)

    if func == "inv":
        ell = 1
    if ell is not None:
        qv, used = q(ell), ell
    else:
        qv, used = adaptive(q, ell1, ell2, tol, ell_max)
    return sla.solve_triangular(W["R"], qv, lower=False), used


def sgmres_quadrature(W: dict, func: str, c_scale: float, ell=None, ell1=16, ell2=22,
                      tol=1e-10, ell_max=1024, alpha: float = 0.5):
    Q, Z, Sb = W["Q"], W["Z"], W["Sb"]

    def q(ell_):
        t, w = quad.rule(func, ell_, c_scale, alpha)
        acc = np.zeros(Q.shape[1], dtype=np.result_type(t, w, np.float64))
        for ti, wi in zip(t, w):
            acc += wi * np.linalg.lstsq(ti * Q + Z, Sb, rcond=None)[0]
        return acc.real   # complex contour nodes: the rule's real part (see quadrature)

    if func == "inv":
        ell = 1
    if ell is not None:
        qv, used = q(ell), ell
    else:
        qv, used = adaptive(q, ell1, ell2, tol, ell_max)
    return sla.solve_triangular(W["R"], qv, lower=False), used


def solve(A, b, func: str, m: int, k: int, S, c_scale: float, method: str = "sgmres",
          ell=None, ell1=16, ell2=22, tol=1e-10, ell_max=1024, alpha: float = 0.5):
    """End-to-end O2 approximant: Algorithm 1 (sFOM) / Algorithm 2 (sGMRES).
    method in {"sgmres", "sfom", "sfom_quad"}.  Returns (x, info)."""
    from .arnoldi import arnoldi_trunc
    ar = arnoldi_trunc(A, b, m, k, S)
    Sb = S @ np.asarray(b, dtype=np.float64)
    W = whiten(ar["SV"], ar["SAV"], Sb)
    info = {"m_eff": ar["m_eff"], "condR": W["condR"], "ell": None}
    if method == "sfom":
        y = sfom_closed(W, func, alpha)
    elif method == "sfom_quad":
        y, info["ell"] = sfom_quadrature(W, func, c_scale, ell, ell1, ell2, tol, ell_max, alpha)
    elif method == "sgmres":
        y, info["ell"] = sgmres_quadrature(W, func, c_scale, ell, ell1, ell2, tol, ell_max, alpha)
    else:
        raise ValueError(method)
    info["arnoldi"] = ar
    info["whitened"] = W
    info["y"] = y
    return ar["V"] @ y, info
