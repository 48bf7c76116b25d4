"""Pins for oracle.quadrature: Gauss rules integrate polynomials exactly, and
the Stieltjes rules reproduce z^-alpha and log(1+z)/z (closed forms) on a
spectral interval to near machine precision once converged."""
import math

import numpy as np
import pytest

from oracle import quadrature as q


def test_gauss_chebyshev_moments():
    x, w = q.gauss_chebyshev(12)
    for j in range(12):
        # int_{-1}^{1} x^{2j} (1-x^2)^{-1/2} dx = pi (2j-1)!! / (2j)!!
        exact = math.pi * math.prod(range(1, 2 * j, 2)) / max(1, math.prod(range(2, 2 * j + 1, 2)))
        assert abs(np.sum(w * x ** (2 * j)) - exact) < 1e-13


def test_gauss_legendre_moments():
    x, w = q.gauss_legendre(10)
    for j in range(10):
        assert abs(np.sum(w * x ** (2 * j)) - 2.0 / (2 * j + 1)) < 1e-14


def test_gauss_jacobi_half_is_chebyshev():
    x1, w1 = q.gauss_chebyshev(9)
    x2, w2 = q.gauss_jacobi(9, -0.5, -0.5)
    o1, o2 = np.argsort(x1), np.argsort(x2)
    np.testing.assert_allclose(x1[o1], x2[o2], atol=1e-14)
    np.testing.assert_allclose(w1[o1], w2[o2], atol=1e-13)


def test_unscaled_map_is_papers_map():
    # c = 1: t = (1-x)/(1+x), i.e. x = (1-t)/(1+t) as in Sec. 5.1
    t, w = q.rule_invpow(7, 1.0, 0.5)
    x, _ = q.gauss_chebyshev(7)
    np.testing.assert_allclose((1 - t) / (1 + t), x, atol=1e-14)


@pytest.mark.parametrize("lo,hi", [(1.0, 1e4), (29.6, 1.2e5), (0.1, 1e5)])
def test_invsqrt_rule(lo, hi):
    c = math.sqrt(lo * hi)
    z = np.geomspace(lo, hi, 50)
    t, w = q.rule_invpow(400, c, 0.5)
    approx = (w[None, :] / (t[None, :] + z[:, None])).sum(1)
    np.testing.assert_allclose(approx, z ** -0.5, rtol=1e-13)
    # complex z in the right half plane
    zc = np.array([3 + 40j, 500 - 2000j, 1e4 + 1j])
    t, w = q.rule_invpow(400, math.sqrt(1.0 * 1e4), 0.5)
    approx = (w[None, :] / (t[None, :] + zc[:, None])).sum(1)
    np.testing.assert_allclose(approx, 1 / np.sqrt(zc), rtol=1e-11)


@pytest.mark.parametrize("alpha", [0.25, 0.7])
def test_invpow_rule(alpha):
    z = np.geomspace(1.0, 100.0, 20)
    t, w = q.rule_invpow(300, 10.0, alpha)
    approx = (w[None, :] / (t[None, :] + z[:, None])).sum(1)
    np.testing.assert_allclose(approx, z ** -alpha, rtol=1e-11)


@pytest.mark.parametrize("hi", [10.0, 1.2e5])
def test_log1p_over_z_rule(hi):
    z = np.concatenate([np.geomspace(1e-3, hi, 40), [0.0]])
    t, w = q.rule_log1p_over_z(300, math.sqrt(1 + hi))
    approx = (w[None, :] / (t[None, :] + z[:, None])).sum(1)
    exact = np.real(q.fscalar("log1p_over_z", z))
    assert exact[-1] == 1.0
    # floor ~1e-12 from rounding of 1+x at the nodes nearest x = -1
    np.testing.assert_allclose(approx, exact, rtol=5e-12)


def test_rule_nodes_nonnegative_and_weights_positive():
    for f in ["invsqrt", "log1p_over_z"]:
        t, w = q.rule(f, 37, 50.0)
        assert np.all(t >= 0) and np.all(w > 0)
    t, w = q.rule("inv", 5, 1.0)
    assert t.tolist() == [0.0] and w.tolist() == [1.0]


def test_ell_schedule():
    assert q.ell_schedule(16, 22, 300)[:9] == [16, 22, 31, 43, 60, 84, 118, 166, 234]
