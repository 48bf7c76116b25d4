"""Pins for oracle.sketched against identities the paper states:

* S = I turns sFOM into FOM, beta V f(H_m) e_1 (Sec. 2, comment 1 after (sFOM))
* sFOM does not depend on the basis of K_m (Sec. 2.1): k = 2 equals k = m
* whitening: Q^T S b = ||b|| R_11 e_1 (proof of Cor. 2.3)
* Cortinovis et al. form V f(H_m + h x_hat e_m^T) ||b|| e_1 (Remark 2.1)
* interpolation of f at the eigenvalues of M (Cor. 2.2)
* closed form equals quadrature form (Sec. 5.1) up to the rule's error
* exactness on an invariant Krylov space
* S = I and f = 1/z: sGMRES is the GMRES iterate (Hessenberg least squares)
* residual bound (eq. (3.2)) and sFOM-FOM distance (Cor. 2.3) with the exact
  embedding constant eps of S on K_{m+1}
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import quadrature as quad
from oracle import sketched as skd
from oracle.arnoldi import arnoldi_trunc
from oracle.sketch import Sketch
from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs


def problem(n=10, nu=(30.0, 10.0)):
    A = csr_to_scipy(convdiff_2d(n, nu))
    b = gaussian_rhs(A.shape[0], 12)
    lo = 2 * (2 - 2 * math.cos(math.pi / (n + 1))) * (n + 1) ** 2
    hi = float(abs(A).sum(axis=1).max())
    return A, b, lo, hi


def f_of_small_matrix(func, H):
    """f(H) through an eigendecomposition (route independent of sqrtm/logm)."""
    lam, X = np.linalg.eig(H)
    return (X * quad.fscalar(func, lam)[None, :]) @ np.linalg.inv(X)


def exact_embedding_eps(S, A, b, m):
    K = np.empty((A.shape[0], m + 1))
    K[:, 0] = b / np.linalg.norm(b)
    for j in range(1, m + 1):
        K[:, j] = A @ K[:, j - 1]
        K[:, j] /= np.linalg.norm(K[:, j])
    U, _ = np.linalg.qr(K)
    sv = np.linalg.svd(S @ U, compute_uv=False)
    return max(sv.max() ** 2 - 1, 1 - sv.min() ** 2)


@pytest.mark.parametrize("func", ["invsqrt", "log1p_over_z"])
def test_identity_sketch_sfom_is_fom(func):
    A, b, lo, hi = problem()
    N, m = A.shape[0], 12
    S = Sketch("identity", N, N)
    x, info = skd.solve(A, b, func, m, m, S, 1.0, method="sfom")
    ar = arnoldi_trunc(A, b, m + 1, m + 1, S)     # H_m needs the m-th column of H
    fom = np.linalg.norm(b) * ar["V"][:, :m] @ f_of_small_matrix(func, ar["H"][:m, :m])[:, 0]
    np.testing.assert_allclose(x, np.real(fom), rtol=1e-10, atol=1e-12 * np.linalg.norm(fom))


@pytest.mark.parametrize("method", ["sfom", "sgmres"])
def test_basis_independence(method):
    A, b, lo, hi = problem()
    N, m = A.shape[0], 14
    S = Sketch("sparse_sign", N, 56, 4, seed=13)
    c = math.sqrt(lo * hi)
    x2, _ = skd.solve(A, b, "invsqrt", m, 2, S, c, method=method, ell=120)
    xm, _ = skd.solve(A, b, "invsqrt", m, m, S, c, method=method, ell=120)
    assert np.linalg.norm(x2 - xm) <= 1e-9 * np.linalg.norm(xm)


def test_whitening_identities():
    A, b, _, _ = problem()
    S = Sketch("sparse_sign", A.shape[0], 40, 8, seed=1)
    ar = arnoldi_trunc(A, b, 10, 2, S)
    W = skd.whiten(ar["SV"], ar["SAV"], S @ b)
    np.testing.assert_allclose(W["Q"].T @ W["Q"], np.eye(10), atol=1e-13)
    np.testing.assert_allclose(W["Q"] @ W["R"], ar["SV"], atol=1e-13)
    np.testing.assert_allclose(W["Z"] @ W["R"], ar["SAV"], rtol=1e-12, atol=1e-9)
    e = np.zeros(10)
    e[0] = np.linalg.norm(b) * W["R"][0, 0]
    np.testing.assert_allclose(W["c"], e, atol=1e-12)


def test_cortinovis_form():
    A, b, lo, hi = problem()
    N, m = A.shape[0], 9
    S = Sketch("sparse_sign", N, 40, 8, seed=7)
    x, info = skd.solve(A, b, "invsqrt", m, 2, S, 1.0, method="sfom")
    ar1 = arnoldi_trunc(A, b, m + 1, 2, S)            # gives v_{m+1} and h_{m+1,m}
    V, H = ar1["V"], ar1["H"]
    xhat = np.linalg.lstsq(ar1["SV"][:, :m], ar1["SV"][:, m], rcond=None)[0]
    Hhat = H[:m, :m].copy()
    Hhat[:, m - 1] += H[m, m - 1] * xhat
    alt = np.linalg.norm(b) * V[:, :m] @ f_of_small_matrix("invsqrt", Hhat)[:, 0]
    np.testing.assert_allclose(x, np.real(alt), rtol=1e-9, atol=1e-11 * np.linalg.norm(x))


def test_interpolation_at_sketched_ritz_values():
    A, b, _, _ = problem(6)
    N, m = A.shape[0], 5
    S = Sketch("sparse_sign", N, 20, 4, seed=2)
    x, info = skd.solve(A, b, "invsqrt", m, 2, S, 1.0, method="sfom")
    nodes = np.linalg.eigvals(info["whitened"]["M"])
    # Newton divided differences of f at the nodes, then q(A) b by Horner
    dd = quad.fscalar("invsqrt", nodes).astype(complex)
    for j in range(1, m):
        dd[j:] = (dd[j:] - dd[j - 1:-1]) / (nodes[j:] - nodes[:-j])
    Ad = A.toarray().astype(complex)
    acc = dd[m - 1] * b.astype(complex)
    for j in range(m - 2, -1, -1):
        acc = (Ad @ acc) - nodes[j] * acc + dd[j] * b
    np.testing.assert_allclose(x, acc.real, rtol=1e-8, atol=1e-10 * np.linalg.norm(x))
    assert np.abs(acc.imag).max() < 1e-8 * np.linalg.norm(x)


@pytest.mark.parametrize("func", ["invsqrt", "log1p_over_z"])
def test_closed_form_equals_quadrature(func):
    A, b, lo, hi = problem()
    S = Sketch("sparse_sign", A.shape[0], 64, 8, seed=13)
    c = quad_scale = math.sqrt(lo * hi) if func == "invsqrt" else math.sqrt(1 + hi)
    xc, _ = skd.solve(A, b, func, 16, 2, S, c, method="sfom")
    xq, info = skd.solve(A, b, func, 16, 2, S, c, method="sfom_quad", tol=1e-12)
    assert np.linalg.norm(xc - xq) <= 1e-10 * np.linalg.norm(xc)
    assert info["ell"] >= 16


@pytest.mark.parametrize("method", ["sfom", "sfom_quad", "sgmres"])
def test_exact_on_invariant_krylov_space(method):
    lam = np.repeat([1.0, 2.0, 3.5, 7.0, 11.0, 20.0], 10)
    A = np.diag(lam)
    b = np.random.default_rng(5).standard_normal(lam.size)
    S = Sketch("sparse_sign", lam.size, 30, 4, seed=13)
    x, info = skd.solve(A, b, "invsqrt", 6, 2, S, math.sqrt(20.0), method=method, tol=1e-13)
    np.testing.assert_allclose(x, b / np.sqrt(lam), rtol=1e-11, atol=1e-12)


def test_identity_sketch_inverse_is_gmres():
    A, b, _, _ = problem()
    N, m = A.shape[0], 10
    x, _ = skd.solve(A, b, "inv", m, m, Sketch("identity", N, N), 1.0, method="sgmres")
    ar = arnoldi_trunc(A, b, m + 1, m + 1, Sketch("identity", N, N))   # H-bar (m+1) x m
    rhs = np.zeros(m + 1)
    rhs[0] = np.linalg.norm(b)
    y = np.linalg.lstsq(ar["H"][: m + 1, :m], rhs, rcond=None)[0]
    np.testing.assert_allclose(x, ar["V"][:, :m] @ y, rtol=1e-9, atol=1e-12)


def test_residual_bound_per_node():
    A, b, lo, hi = problem()
    N, m = A.shape[0], 12
    S = Sketch("sparse_sign", N, 48, 4, seed=21)
    eps = exact_embedding_eps(S, A, b, m)
    assert eps < 1
    C = math.sqrt((1 + eps) / (1 - eps))
    ar = arnoldi_trunc(A, b, m, 2, S)
    W = skd.whiten(ar["SV"], ar["SAV"], S @ b)
    V = ar["V"] @ np.linalg.inv(W["R"])
    Vo = np.linalg.qr(ar["V"])[0]
    AV, AVo = A @ V, A @ Vo
    for t in [0.0, 3.0, 300.0, 3e4]:
        y_s = np.linalg.lstsq(t * W["Q"] + W["Z"], W["Sb"], rcond=None)[0]
        r_s = b - (t * V + AV) @ y_s
        y_f = np.linalg.lstsq(t * Vo + AVo, b, rcond=None)[0]
        r_f = b - (t * Vo + AVo) @ y_f
        floor = 1e-12 * np.linalg.norm(b)          # rounding level of both residuals
        assert np.linalg.norm(r_s) <= C * np.linalg.norm(r_f) * (1 + 1e-9) + floor
        assert np.linalg.norm(r_f) <= np.linalg.norm(r_s) * (1 + 1e-9) + floor


def test_sfom_fom_distance_bound():
    A, b, lo, hi = problem()
    N, m = A.shape[0], 10
    S = Sketch("sparse_sign", N, 60, 8, seed=4)
    eps = exact_embedding_eps(S, A, b, m)
    xs, info = skd.solve(A, b, "invsqrt", m, 2, S, 1.0, method="sfom")
    xf, _ = skd.solve(A, b, "invsqrt", m, m, Sketch("identity", N, N), 1.0, method="sfom")
    V = info["arnoldi"]["V"] @ np.linalg.inv(info["whitened"]["R"])   # S V orthonormal
    Vp = np.linalg.pinv(V)
    F1 = f_of_small_matrix("invsqrt", Vp @ (A @ V))
    F2 = f_of_small_matrix("invsqrt", (S @ V).T @ (S @ (A @ V)))
    bound = math.sqrt((1 + eps) / (1 - eps)) * np.linalg.norm(b) * np.linalg.norm(F1 - F2, 2)
    assert np.linalg.norm(xf - xs) <= bound * (1 + 1e-8)


def test_sgmres_converges_to_exact():
    from oracle.exact import fAb_dense
    A, b, lo, hi = problem(8)
    N = A.shape[0]
    ref = fAb_dense(A.toarray(), b, "invsqrt")
    S = Sketch("sparse_sign", N, 64, 8, seed=13)
    errs = []
    for m in [4, 8, 16, 28]:
        x, _ = skd.solve(A, b, "invsqrt", m, 2, S, math.sqrt(lo * hi), method="sgmres", tol=1e-12)
        errs.append(np.linalg.norm(x - ref) / np.linalg.norm(ref))
    assert errs[-1] < 1e-7 and all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))


def test_adaptive_quadrature_limits():
    A, b, lo, hi = problem()
    S = Sketch("sparse_sign", A.shape[0], 40, 8, seed=1)
    with pytest.raises(skd.QuadNotConverged):
        skd.solve(A, b, "invsqrt", 10, 2, S, 1e-6, method="sgmres", tol=1e-14, ell_max=40)


def test_branch_cut_detected():
    M = np.diag([2.0, -1.0, 3.0])
    with pytest.raises(skd.BranchCutError):
        skd.matfunc_apply("invsqrt", M, np.ones(3))
