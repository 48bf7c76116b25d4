"""Quadrature rules for Stieltjes integrals f(z) = int_Gamma (t + z)^{-1} dmu(t)
(Sec. 1 and Sec. 4.1, eq. (4.1)); each rule returns nodes t_i >= 0 and
weights w_i with f(z) ~= sum_i w_i / (t_i + z).

* z^-alpha, 0 < alpha < 1:  z^-alpha = (sin(alpha pi)/pi) int_0^inf t^-alpha (t+z)^-1 dt.
  With t = c(1-x)/(1+x) this is exactly
  (sin(alpha pi)/pi) 2 c^(1-alpha) int_{-1}^{1} (1-x)^-alpha (1+x)^(alpha-1)
  [c(1-x) + z(1+x)]^-1 dx, a Gauss-Jacobi(-alpha, alpha-1) integral; for
  alpha = 1/2 the weight is Chebyshev's (1-x^2)^-1/2 (the Gauss-Chebyshev rule
  after x = (1-t)/(1+t) of Sec. 5.1, which is the case c = 1).
* log(1+z)/z = int_1^inf t^-1 (t+z)^-1 dt.  With t = 1 + c(1-x)/(1+x) the
  integrand becomes 2c / ([(1+x) + c(1-x)] [(1+z)(1+x) + c(1-x)]), integrated
  by Gauss-Legendre.
* 1/z: the single node t = 0 with weight 1.
* e^{-z} (not a Stieltjes function; the contour form of Algorithm 2): by
  Cauchy's formula in the pole variable t = -z,
  f(A) b = (1/(2 pi i)) oint f(-t) (t I + A)^{-1} b dt, on a contour that
  winds once counterclockwise around the points -lambda(A).  The contour is
  the parabola t(zeta) = a - c zeta^2 + i zeta (Sec. 5.2), zeta in R, along
  which e^{t} decays like e^{-c zeta^2}; the trapezoidal rule in zeta with
  step h on [-L, L], c L^2 = 37, converges exponentially.  For real A and b
  the terms at zeta and -zeta are complex conjugates, so the rule keeps the
  nodes zeta_k = k h, k = 0 .. ell-1 (h = L / (ell - 1)), doubles the weights
  of k >= 1, and f(A) b is the real part of the sum:
      t_k = a - c zeta_k^2 + i zeta_k,
      w_k = (2 - [k = 0]) h e^{t_k} (i - 2 c zeta_k) / (2 pi i).
  Here `alpha` carries the vertex a and `c` the width parameter.

The scale c > 0 is an input (chosen from a spectral interval by the caller).
"""
from __future__ import annotations

import math

import numpy as np


def gauss_chebyshev(ell: int):
    i = np.arange(1, ell + 1)
    x = np.cos((2 * i - 1) * math.pi / (2 * ell))
    w = np.full(ell, math.pi / ell)
    return x, w


def gauss_legendre(ell: int):
    return np.polynomial.legendre.leggauss(ell)


def gauss_jacobi(ell: int, a: float, b: float):
    """Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b by Golub-Welsch: the
    nodes are the eigenvalues of the symmetric tridiagonal Jacobi matrix of
    the monic recurrence, the weights mu_0 times the squared first
    eigenvector components.  The k = 0 diagonal entry and the k = 1
    off-diagonal entry are written in cancelled form so that a + b = -1
    (the z^-alpha weight) is well defined."""
    import scipy.linalg as sla
    k = np.arange(ell, dtype=np.float64)
    ab = a + b
    diag = np.empty(ell)
    diag[0] = (b - a) / (ab + 2.0)
    kk = k[1:]
    diag[1:] = (b * b - a * a) / ((2 * kk + ab) * (2 * kk + ab + 2.0))
    off2 = np.empty(max(ell - 1, 0))
    if ell > 1:
        off2[0] = 4.0 * (1 + a) * (1 + b) / ((2.0 + ab) ** 2 * (3.0 + ab))
        kk = k[2:]
        off2[1:] = (4.0 * kk * (kk + a) * (kk + b) * (kk + ab)
                    / ((2 * kk + ab) ** 2 * (2 * kk + ab + 1.0) * (2 * kk + ab - 1.0)))
    x, vec = sla.eigh_tridiagonal(diag, np.sqrt(off2))
    mu0 = 2.0 ** (ab + 1.0) * math.exp(math.lgamma(a + 1) + math.lgamma(b + 1) - math.lgamma(ab + 2))
    w = mu0 * vec[0, :] ** 2
    return x, w


def rule_invpow(ell: int, c: float, alpha: float = 0.5):
    if alpha == 0.5:
        x, om = gauss_chebyshev(ell)
    else:
        x, om = gauss_jacobi(ell, -alpha, alpha - 1.0)
    t = c * (1.0 - x) / (1.0 + x)
    w = (math.sin(alpha * math.pi) / math.pi) * 2.0 * c ** (1.0 - alpha) * om / (1.0 + x)
    return t, w


def rule_log1p_over_z(ell: int, c: float):
    x, om = gauss_legendre(ell)
    t = 1.0 + c * (1.0 - x) / (1.0 + x)
    w = 2.0 * c * om / ((1.0 + x) ** 2 * t)
    return t, w


def rule_exp_neg(ell: int, c: float, a: float):
    if ell < 2:
        raise ValueError("the contour rule needs ell >= 2")
    L = math.sqrt(37.0 / c)
    h = L / (ell - 1)
    zeta = h * np.arange(ell)
    t = a - c * zeta ** 2 + 1j * zeta
    w = h * np.exp(t) * (1j - 2.0 * c * zeta) / (2j * math.pi)
    w[1:] *= 2.0
    return t, w


def rule(func: str, ell: int, c: float, alpha: float = 0.5):
    if func == "exp_neg":
        return rule_exp_neg(ell, c, alpha)
    if func == "invsqrt":
        return rule_invpow(ell, c, 0.5)
    if func == "invpow":
        return rule_invpow(ell, c, alpha)
    if func == "log1p_over_z":
        return rule_log1p_over_z(ell, c)
    if func == "inv":
        return np.zeros(1), np.ones(1)
    raise ValueError(func)


def fscalar(func: str, z, alpha: float = 0.5):
    """The scalar function on the principal branch."""
    z = np.asarray(z, dtype=np.complex128)
    if func == "invsqrt":
        return 1.0 / np.sqrt(z)
    if func == "invpow":
        return np.exp(-alpha * np.log(z))
    if func == "log1p_over_z":
        out = np.empty_like(z)
        small = np.abs(z) < 1e-8
        out[~small] = np.log1p(z[~small]) / z[~small]
        zs = z[small]
        out[small] = 1.0 - zs / 2.0 + zs * zs / 3.0
        return out
    if func == "inv":
        return 1.0 / z
    if func == "exp_neg":
        return np.exp(-z)
    raise ValueError(func)


def ell_schedule(ell1: int, ell2: int, ell_max: int):
    """Orders visited by the adaptive loop of Sec. 4.1: ell1 < ell2, then
    ell2 <- floor(sqrt(2) * ell2) until ell_max is passed."""
    out = [ell1, ell2]
    while out[-1] < ell_max:
        out.append(int(math.floor(math.sqrt(2.0) * out[-1])))
    return out
