"""Pins for oracle.exact: f(A)b against closed forms -- a diagonalisable
matrix with known eigenvectors, and the 2D convection-diffusion operator,
whose 1D factors tridiag(-(1+p), 2, -(1-p))/h^2 are diagonalised by a
diagonal similarity and the sine transform."""
import math

import numpy as np
import pytest

from oracle.exact import fAb_dense, fAb_shifted
from oracle import quadrature as quad
from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs


@pytest.mark.parametrize("func", ["invsqrt", "log1p_over_z", "inv"])
def test_dense_against_eigendecomposition(func):
    rng = np.random.default_rng(0)
    X = np.eye(30) + 0.1 * rng.standard_normal((30, 30))
    lam = np.geomspace(0.5, 200.0, 30)
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    b = rng.standard_normal(30)
    want = X @ (np.real(quad.fscalar(func, lam)) * np.linalg.solve(X, b))
    np.testing.assert_allclose(fAb_dense(A, b, func), want, rtol=1e-10, atol=1e-12)


def test_convdiff_closed_form():
    n, nu = 7, (10.0, 4.0)          # cell Peclet numbers p = nu h / 2 < 1
    h = 1.0 / (n + 1)
    A = csr_to_scipy(convdiff_2d(n, nu)).toarray()
    b = gaussian_rhs(n * n, 3)
    idx = np.arange(1, n + 1)
    Phi = np.sqrt(2 * h) * np.sin(np.pi * h * np.outer(idx, idx))     # orthogonal sine basis
    facs = []
    for d in range(2):
        p = nu[d] * h / 2
        rho = math.sqrt((1 + p) / (1 - p))
        D = np.diag(rho ** np.arange(n))       # T = D T_sym D^-1
        lam = (2 - 2 * math.sqrt(1 - p * p) * np.cos(np.pi * h * idx)) / h ** 2
        facs.append((D @ Phi, Phi.T @ np.linalg.inv(D), lam))
    Xx, Xxi, lx = facs[0]
    Xy, Xyi, ly = facs[1]
    X = np.kron(Xy, Xx)
    Xi = np.kron(Xyi, Xxi)
    lam = (ly[:, None] + lx[None, :]).ravel()
    np.testing.assert_allclose(X @ np.diag(lam) @ Xi, A, atol=1e-8 * np.abs(A).max())
    want = X @ (lam ** -0.5 * (Xi @ b))
    np.testing.assert_allclose(fAb_dense(A, b, "invsqrt"), want, rtol=1e-10)


def test_shifted_solves_match_dense():
    A = csr_to_scipy(convdiff_2d(9, (10.0, 5.0)))
    b = gaussian_rhs(81, 4)
    hi = float(abs(A).sum(axis=1).max())
    lo = 2 * (2 - 2 * math.cos(math.pi / 10)) * 100
    x = fAb_shifted(A, b, "invsqrt", math.sqrt(lo * hi), 120)
    np.testing.assert_allclose(x, fAb_dense(A.toarray(), b, "invsqrt"), rtol=1e-11)
    x = fAb_shifted(A, b, "log1p_over_z", math.sqrt(1 + hi), 200)
    np.testing.assert_allclose(x, fAb_dense(A.toarray(), b, "log1p_over_z"), rtol=1e-10)
