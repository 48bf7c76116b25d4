"""End-to-end parity of the GPU sFOM / sGMRES approximants with the oracle
(Algorithms 1 and 2, eqs. (sFOM), (sFOM'''), (sGMRES), adaptive quadrature
of Sec. 4.1).  FP64 path: relative 2-norm error <= 1e-10."""
import math

import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.exact import fAb_dense
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from workloads.operators import CSR
from gpu_helpers import upload, rel

pytestmark = pytest.mark.gpu

TOL = 1e-10


def gpu_solve(skf, Acsr, b, func, m, k, s, c, method, zeta=8, seed=13, tol=1e-12, kind=None, ell=(16, 22, 1024),
              nodes=None):
    op = upload(skf, Acsr)
    S = skf.Sketch(kind if kind is not None else skf.SPARSE_SIGN, Acsr.n, s, zeta, seed)
    if nodes is not None:
        f = skf.make_func(func, c, nodes=nodes[0], weights=nodes[1])
    else:
        f = skf.make_func(func, c)
    p = skf.make_params(m, k, ell1=ell[0], ell2=ell[1], ell_max=ell[2], tol=tol)
    info = skf.new_info()
    x = skf.solve(method, op.csr, S, torch.as_tensor(b, device="cuda"), f, p, info=info)
    torch.cuda.synchronize()
    return x.cpu().numpy(), skf.read_info(info)


def config1():
    A = convdiff_2d(100, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", laplacian_lambda_min(100, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    return A, b, c


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_config1_2d_invsqrt(skf, method):
    """2D convection-diffusion N = 1e4, m = 40, k = 2, s = 160, zeta = 8."""
    A, b, c = config1()
    m, k, s = 40, 2, 160
    x, info = gpu_solve(skf, A, b, "invsqrt", m, k, s, c, skf.SGMRES if method == "sgmres" else skf.SFOM)
    xo, oi = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                       method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    assert info["status"] == 0 and info["m_eff"] == m
    assert info["ell"] == oi["ell"]
    assert rel(x, xo) <= TOL
    if method == "sfom":   # quadrature form equals the closed form (sFOM''')
        xc, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                          method="sfom")
        assert rel(x, xc) <= TOL


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_3d_log1p_over_z(skf, method):
    """3D convection-diffusion (the log(1+z)/z workload) at n = 30, m = 60, s = 240."""
    A = convdiff_3d(30, (50.0, 50.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("log1p_over_z", 0.0, float(abs(csr_to_scipy(A)).sum(1).max()))
    m, k, s = 60, 2, 240
    x, info = gpu_solve(skf, A, b, "log1p_over_z", m, k, s, c, skf.SGMRES if method == "sgmres" else skf.SFOM)
    xo, oi = osk.solve(csr_to_scipy(A), b, "log1p_over_z", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                       method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    assert info["status"] == 0
    assert rel(x, xo) <= TOL


def test_identity_sketch_full_orthogonalisation_is_fom(skf):
    A = convdiff_2d(12, (30.0, 10.0))
    b = gaussian_rhs(A.n, 12)
    m = 12
    c = quad_scale("invsqrt", laplacian_lambda_min(12, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    x, info = gpu_solve(skf, A, b, "invsqrt", m, m, A.n, c, skf.SFOM, kind=skf.IDENTITY, zeta=1)
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, m, OSketch("identity", A.n, A.n), c, method="sfom")
    assert rel(x, xo) <= TOL


def test_inverse_is_sketched_gmres(skf):
    A = convdiff_2d(40, (20.0, 10.0))
    b = gaussian_rhs(A.n, 2)
    m, s = 30, 120
    x, info = gpu_solve(skf, A, b, "inv", m, 2, s, 1.0, skf.SGMRES)
    xo, _ = osk.solve(csr_to_scipy(A), b, "inv", m, 2, OSketch("sparse_sign", A.n, s, 8, 13), 1.0, method="sgmres")
    assert info["ell"] == 1 and rel(x, xo) <= TOL


def test_explicit_rule(skf):
    from oracle import quadrature as oq
    A, b, c = config1()
    t, w = oq.rule("invsqrt", 37, c)
    x, info = gpu_solve(skf, A, b, "invsqrt", 20, 2, 80, c, skf.SGMRES, nodes=(t, w))
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", 20, 2, OSketch("sparse_sign", A.n, 80, 8, 13), c,
                      method="sgmres", ell=37)
    assert info["ell"] == 37 and rel(x, xo) <= TOL


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_invariant_subspace_exact(skf, method):
    lam = np.repeat([1.0, 2.0, 3.5, 7.0, 11.0, 20.0], 400)
    N = lam.size
    A = CSR(N, np.arange(N + 1, dtype=np.int64), np.arange(N, dtype=np.int32), lam)
    b = gaussian_rhs(N, 5)
    x, info = gpu_solve(skf, A, b, "invsqrt", 10, 2, 40, math.sqrt(20.0), skf.SGMRES if method == "sgmres" else skf.SFOM,
                        tol=1e-13)
    assert info["m_eff"] == 6 and info["breakdown"] == 1
    assert rel(x, b / np.sqrt(lam)) <= 1e-11


def test_zero_rhs_and_sketch_too_small(skf):
    A = convdiff_2d(10)
    x, info = gpu_solve(skf, A, np.zeros(A.n), "invsqrt", 5, 2, 20, 10.0, skf.SGMRES)
    assert info["status_name"] == "SKF_ERR_ZERO_RHS" and np.all(x == 0)
    with pytest.raises(skf.SkfError, match="SKETCH_TOO_SMALL"):
        gpu_solve(skf, A, np.ones(A.n), "invsqrt", 12, 2, 20, 10.0, skf.SGMRES)


def test_quadrature_not_converged_reported(skf):
    A, b, c = config1()
    x, info = gpu_solve(skf, A, b, "invsqrt", 10, 2, 40, 1e-6 * c, skf.SGMRES, tol=1e-14, ell=(16, 22, 40))
    assert info["status_name"] == "SKF_ERR_QUAD_NOT_CONVERGED" and info["ell"] == 31
    assert np.all(np.isfinite(x))


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_config1_srht(skf, method):
    """Config-1 operator with the SRHT sketch (s = 160, N' = 16384)."""
    A, b, c = config1()
    m, k, s = 40, 2, 160
    x, info = gpu_solve(skf, A, b, "invsqrt", m, k, s, c, skf.SGMRES if method == "sgmres" else skf.SFOM,
                        kind=skf.SRHT, zeta=0)
    xo, oi = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("srht", A.n, s, 0, 13), c,
                       method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    assert info["status"] == 0 and info["m_eff"] == m
    assert rel(x, xo) <= TOL
