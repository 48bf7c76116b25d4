"""CPU checks of the C ABI boundary: the shared library loads, exports every
function include/skf.h declares, validates arguments on the host, and its
host-side quadrature rules equal the oracle's rules (Sec. 4.1, Sec. 5.1)."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def skf():
    import paper_2208_11447_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2208_11447_gb300 import build
        build.build()
    pkg.lib()
    return pkg


def declared_functions():
    text = open(os.path.join(ROOT, "include", "skf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(skf_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(skf):
    names = declared_functions()
    assert len(names) >= 14
    L = skf.lib()
    for name in names:
        assert hasattr(L, name), name


def test_version_and_status_strings(skf):
    L = skf.lib()
    assert L.skf_version() >= 100
    for code in range(11):
        assert L.skf_status_string(code)


def test_host_side_validation(skf):
    import ctypes
    L = skf.lib()
    h = ctypes.c_void_p()
    # zeta > s, identity with s != n, unknown kind: rejected before any device work
    assert L.skf_sketch_create(skf.SPARSE_SIGN, 100, 4, 8, 1, None, ctypes.byref(h)) == 1
    assert L.skf_sketch_create(skf.IDENTITY, 100, 50, 1, 1, None, ctypes.byref(h)) == 1
    assert L.skf_sketch_create(7, 100, 50, 1, 1, None, ctypes.byref(h)) == 1
    assert L.skf_create_csr(0, 0, None, None, None, 0, 0, None, ctypes.byref(h)) == 1
    assert b"n must be" in L.skf_last_error()
    assert L.skf_sketch_destroy(None) == 0
    assert L.skf_destroy_csr(None) == 0
    assert L.skf_set_arnoldi_mode(3) == 1 and L.skf_set_arnoldi_mode(-1) == 1
    assert L.skf_set_arnoldi_mode(0) == 0
    assert L.skf_set_qr_mode(2) == 1 and L.skf_set_qr_mode(0) == 0
    assert L.skf_set_tail_form(2) == 1 and L.skf_set_tail_form(-1) == 1 and L.skf_set_tail_form(0) == 0
    assert L.skf_set_block_mode(2) == 1 and L.skf_set_block_mode(-1) == 1 and L.skf_set_block_mode(0) == 0
    assert L.skf_barrier_selftest(1, 10**6, None, None) == 1          # NULL status pointer
    # block solve and precision plan: argument checks before any device work
    assert L.skf_solve_block(1, None, None, None, 10, -1, None, None, None, 10, None, None) == 1
    assert L.skf_solve_block(1, None, None, None, 10, 0, None, None, None, 10, None, None) == 0   # empty block
    cond = (ctypes.c_double * 1)()
    f32 = (ctypes.c_int32 * 1)()
    assert L.skf_plan_basis_precision(-1, None, 1e-6, cond, f32, None) == 1
    assert L.skf_plan_basis_precision(0, None, 0.0, cond, f32, None) == 1                      # tol <= 0
    assert L.skf_plan_basis_precision(0, None, 1e-6, cond, f32, None) == 0


@pytest.mark.parametrize("func,ell,c", [("invsqrt", 45, 1.0), ("invsqrt", 300, 1885.0),
                                        ("log1p_over_z", 22, 346.4), ("log1p_over_z", 400, 30.0),
                                        ("inv", 1, 1.0)])
def test_quadrature_rule_matches_oracle(skf, func, ell, c):
    from oracle import quadrature as oq
    t, w = skf.quadrature_rule(skf.make_func(func, c), ell)
    to, wo = oq.rule(func, ell, c)
    o1, o2 = np.argsort(t), np.argsort(to)
    # the oracle forms 1 + x from x; the library from theta (x = cos theta), so
    # the nodes nearest x = +-1 differ by the oracle's rounding of 1 -+ x
    np.testing.assert_allclose(t[o1], to[o2], rtol=1e-9, atol=0)
    np.testing.assert_allclose(w[o1], wo[o2], rtol=1e-8, atol=0)
    np.testing.assert_allclose(t[o1][5:-5], to[o2][5:-5], rtol=1e-12, atol=0)


@pytest.mark.parametrize("func,lo,hi,ell", [("invsqrt", 29.6, 1.2e5, 200), ("log1p_over_z", 1e-3, 1.2e5, 300)])
def test_quadrature_rule_reproduces_f(skf, func, lo, hi, ell):
    """Sum_i w_i / (t_i + z) equals the closed form f(z) on the interval."""
    from oracle.quadrature import fscalar
    c = math.sqrt(lo * hi) if func == "invsqrt" else math.sqrt(1 + hi)
    t, w = skf.quadrature_rule(skf.make_func(func, c), ell)
    z = np.geomspace(lo, hi, 60)
    approx = (w[None, :] / (t[None, :] + z[:, None])).sum(1)
    np.testing.assert_allclose(approx, np.real(fscalar(func, z)), rtol=2e-13)


@pytest.mark.parametrize("ell,c,a", [(2, 1.0, 0.0), (64, 0.1, 0.5), (200, 0.02, -0.3)])
def test_contour_rule_matches_oracle(skf, ell, c, a):
    """exp(-z) contour rule (parabola of Sec. 5.2, trapezoidal in its
    parameter): the library's host rule equals the oracle's."""
    from oracle import quadrature as oq
    t, w = skf.quadrature_rule_c(skf.make_func("exp_neg", c, alpha=a), ell)
    to, wo = oq.rule("exp_neg", ell, c, a)
    np.testing.assert_allclose(t, to, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(w, wo, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("alpha,ell", [(0.3, 16), (0.3, 150), (0.7, 60), (0.1, 400), (0.9, 1024)])
def test_invpow_gauss_jacobi_rule(skf, alpha, ell):
    """z^-alpha, alpha != 1/2: the host Gauss-Jacobi(-alpha, alpha-1) rule
    (bisection on the Jacobi matrix, eigenvector weights) against the
    oracle's (SciPy's tridiagonal eigensolver): nodes agree away from the end
    points (both round 1 + x there), and the quadrature sums agree."""
    from oracle import quadrature as oq
    c = 7.0
    t, w = skf.quadrature_rule(skf.make_func("invpow", c, alpha=alpha), ell)
    to, wo = oq.rule("invpow", ell, c, alpha)
    o1, o2 = np.argsort(t), np.argsort(to)
    assert np.all(t > 0) and np.all(w > 0)
    # both sides form 1 -+ x from x: the nodes nearest x = +-1 carry that rounding
    np.testing.assert_allclose(t[o1], to[o2], rtol=1e-8, atol=0)
    np.testing.assert_allclose(t[o1][5:-5], to[o2][5:-5], rtol=1e-11, atol=0)
    z = np.geomspace(1e-2, 1e4, 40)
    s1 = (w[None, :] / (t[None, :] + z[:, None])).sum(1)
    s2 = (wo[None, :] / (to[None, :] + z[:, None])).sum(1)
    np.testing.assert_allclose(s1, s2, rtol=1e-11)


@pytest.mark.parametrize("alpha", [0.25, 0.6, 0.85])
def test_invpow_rule_reproduces_z_power(skf, alpha):
    """Pin to the closed form: sum_i w_i / (t_i + z) = z^-alpha on a spectral
    interval, with the scale c = sqrt(lo hi) (Sec. 4.1's rules converge
    geometrically in ell)."""
    lo, hi = 30.0, 6e4
    t, w = skf.quadrature_rule(skf.make_func("invpow", math.sqrt(lo * hi), alpha=alpha), 400)
    z = np.geomspace(lo, hi, 50)
    approx = (w[None, :] / (t[None, :] + z[:, None])).sum(1)
    np.testing.assert_allclose(approx, z ** -alpha, rtol=1e-12)


def test_invpow_rejects_alpha_outside_unit_interval(skf):
    with pytest.raises(skf.SkfError):
        skf.quadrature_rule(skf.make_func("invpow", 1.0, alpha=1.5), 10)


def test_custom_rule_closure(skf):
    """SKF_FUNC_CUSTOM: the library obtains the rule of each order from the
    caller's rule(ell, t, w, ctx) closure and uses it unchanged; a failing
    callback is reported as NOT_SUPPORTED."""
    calls = []

    def rule(ell):
        calls.append(ell)
        return np.arange(1, ell + 1, dtype=float), 1.0 / np.arange(1, ell + 1, dtype=float)

    f = skf.make_func("custom", rule=rule)
    t, w = skf.quadrature_rule(f, 7)
    assert calls == [7]
    np.testing.assert_array_equal(t, np.arange(1, 8, dtype=float))
    np.testing.assert_array_equal(w, 1.0 / np.arange(1, 8, dtype=float))
    bad = skf.make_func("custom", rule=lambda ell: ([1.0], [1.0]))      # wrong length
    with pytest.raises(skf.SkfError, match="NOT_SUPPORTED"):
        skf.quadrature_rule(bad, 3)


def test_column_major_view_without_copy(skf):
    """The sketch bindings pass X to the C ABI column-major (column c at offset
    c N): a tensor already laid out that way goes through as a view, any other
    layout is copied once."""
    import torch
    N = 7
    x = torch.arange(N, dtype=torch.float64)
    v = skf._column_major(x)
    assert v.shape == (1, N) and v.data_ptr() == x.data_ptr()
    Y = torch.arange(3 * N, dtype=torch.float64).reshape(3, N)      # rows = columns of X = Y.t()
    v = skf._column_major(Y.t())
    assert v.shape == (3, N) and v.data_ptr() == Y.data_ptr() and torch.equal(v, Y)
    X = torch.arange(3 * N, dtype=torch.float64).reshape(N, 3)      # row-major (N, 3): needs a copy
    v = skf._column_major(X)
    assert v.shape == (3, N) and v.is_contiguous() and v.data_ptr() != X.data_ptr()
    assert torch.equal(v, X.t())
