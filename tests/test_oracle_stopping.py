"""Pins of the oracle's sketched stopping criterion (Sec. 4.3,
eqs. (sketched_err_est1), (sketched_err_est2)) on tiny problems where the
iterates and the exact embedding constant of S on K_{m+d}(A, b) can be formed
explicitly."""
import numpy as np
import pytest

from oracle import sketched as osk
from oracle import stopping as ost
from oracle.arnoldi import arnoldi_trunc
from oracle.sketch import Sketch
from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale


def setup(n=12, s=96, zeta=4, seed=13):
    A = convdiff_2d(n, (30.0, 10.0))
    As = csr_to_scipy(A)
    b = gaussian_rhs(A.n, 12)
    S = Sketch("sparse_sign", A.n, s, zeta, seed)
    c = quad_scale("invsqrt", laplacian_lambda_min(n, 2), float(abs(As).sum(1).max()))
    return As, b, S, c


def exact_eps(S, V):
    """Embedding constant of S on span(V): max | sigma_i(S U)^2 - 1 |, U an
    orthonormal basis of span(V)."""
    U, _ = np.linalg.qr(V)
    sv = np.linalg.svd(S @ U, compute_uv=False)
    return float(np.max(np.abs(sv ** 2 - 1.0)))


@pytest.mark.parametrize("m,d,method", [(8, 4, "sgmres"), (12, 4, "sgmres"), (10, 5, "sfom_quad")])
def test_bracket_holds_with_the_exact_embedding_constant(m, d, method):
    As, b, S, c = setup()
    ar = arnoldi_trunc(As, b, m + d, 2, S)
    Sb = S @ b
    y_m, _ = ost.prefix_coefficients(ar, Sb, m, "invsqrt", c, method, 1e-12)
    y_md, _ = ost.prefix_coefficients(ar, Sb, m + d, "invsqrt", c, method, 1e-12)
    f_m = ar["V"][:, :m] @ y_m
    f_md = ar["V"] @ y_md
    true_diff = np.linalg.norm(f_md - f_m)
    eps = exact_eps(S, ar["V"])
    assert eps < 1.0
    # the sketched difference is the sketch of the explicit difference
    sk = ost.sketched_difference(ar["SV"], y_md, y_m)
    assert abs(sk - np.linalg.norm(S @ (f_md - f_m))) <= 1e-12 * max(sk, 1e-300) + 1e-15
    lower = sk / np.sqrt(1.0 + eps)
    upper = sk / np.sqrt(1.0 - eps)
    assert lower <= true_diff * (1 + 1e-10) and true_diff <= upper * (1 + 1e-10)
    # the per-vector estimate never exceeds the exact constant
    assert ost.eps_hat(ar["SV"]) <= eps + 1e-12
    diff, nrm = ost.error_estimate(ar["SV"], y_md, y_m, ost.eps_hat(ar["SV"]))
    assert diff == pytest.approx(sk / np.sqrt(1.0 - ost.eps_hat(ar["SV"])), rel=1e-14)
    assert nrm == pytest.approx(np.linalg.norm(S @ f_md) / np.sqrt(1.0 + ost.eps_hat(ar["SV"])), rel=1e-12)


def test_stop_returns_the_iterate_of_a_fresh_solve_at_the_stopping_m():
    As, b, S, c = setup(n=14, s=120)
    x, info = ost.solve_with_stopping(As, b, "invsqrt", 40, 2, S, c, d=4, tol=1e-4)
    assert info["stopped"]
    p = info["p"]
    assert p % 4 == 0 and p >= 8
    # every earlier checkpoint missed the tolerance, the accepted one met it
    assert all(r > 1e-4 for q, r in info["history"][:-1]) and info["history"][-1][1] <= 1e-4
    xo, _ = osk.solve(As, b, "invsqrt", p, 2, S, c, method="sgmres", tol=1e-10)
    assert np.linalg.norm(x - xo) <= 1e-13 * np.linalg.norm(xo)


def test_estimate_tracks_the_true_error_decrease():
    """The estimates shrink as the iterates converge, and the estimate at the
    accepted checkpoint bounds the actual change between the two iterates."""
    As, b, S, c = setup(n=14, s=120)
    x, info = ost.solve_with_stopping(As, b, "invsqrt", 40, 2, S, c, d=4, tol=0.0)
    assert not info["stopped"] and info["p"] == 40
    rels = [r for _, r in info["history"]]
    assert rels[-1] < 1e-3 * rels[0]
    xo, _ = osk.solve(As, b, "invsqrt", 40, 2, S, c, method="sgmres", tol=1e-10)
    assert np.linalg.norm(x - xo) <= 1e-13 * np.linalg.norm(xo)
