"""skf_sfom_sgmres: both approximants from one truncated Arnoldi process
(Sec. 3: sFOM and sGMRES use the same V_m, S V_m, S A V_m) equal the
separate skf_sfom / skf_sgmres results bit for bit, in both Arnoldi forms,
both tail forms, with an FP32 basis and with the complex contour rule; and
they match the oracle."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import upload, rel

pytestmark = pytest.mark.gpu


def setup(skf, n=90, m=40, k=2, func="invsqrt", basis=torch.float64):
    A = convdiff_2d(n, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    vals = A.values.astype(np.float64 if basis == torch.float64 else np.float32)   # reduced bases need F32 values
    op = skf.upload_csr(A.rowptr, A.colind, vals, device="cuda")
    s = 4 * m
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    lam = laplacian_lambda_min(n, 2)
    c = quad_scale(func, lam, float(abs(csr_to_scipy(A)).sum(1).max()))
    f = skf.make_func(func, c)
    p = skf.make_params(m, k, basis_dtype=basis, tol=1e-12 if basis == torch.float64 else 1e-10)
    return A, torch.as_tensor(b, device="cuda"), op, S, f, p, c, s


def both(skf, op, S, bt, f, p):
    i1, i2, i3, i4 = skf.new_info(), skf.new_info(), skf.new_info(), skf.new_info()
    xf = skf.sfom(op.csr, S, bt, f, p, info=i1)
    xg = skf.sgmres(op.csr, S, bt, f, p, info=i2)
    pf, pg = skf.sfom_sgmres(op.csr, S, bt, f, p, info_fom=i3, info_gmres=i4)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (xf, xg, pf, pg)], [skf.read_info(i) for i in (i1, i2, i3, i4)]


@pytest.mark.parametrize("amode", ["persistent", "two_kernel"])
@pytest.mark.parametrize("form", ["relation", "full"])
def test_pair_equals_separate_solves(skf, amode, form):
    A, bt, op, S, f, p, c, s = setup(skf)
    am = skf.ARNOLDI_PERSISTENT if amode == "persistent" else skf.ARNOLDI_TWO_KERNEL
    tf = skf.TAIL_AUTO if form == "relation" else skf.TAIL_FULL
    with skf.arnoldi_mode(am), skf.tail_form(tf):
        (xf, xg, pf, pg), (i1, i2, i3, i4) = both(skf, op, S, bt, f, p)
    assert np.array_equal(xf, pf) and np.array_equal(xg, pg)
    for a, b_ in ((i1, i3), (i2, i4)):
        for key in ("status", "m_eff", "ell", "quad_err", "beta", "cond_est", "rdiag_ratio", "eps_est", "breakdown"):
            assert a[key] == b_[key], key
    for meth, x in (("sfom_quad", pf), ("sgmres", pg)):
        xo, oi = osk.solve(csr_to_scipy(A), bt.cpu().numpy(), "invsqrt", 40, 2,
                           OSketch("sparse_sign", A.n, s, 8, 13), c, method=meth, tol=1e-12)
        assert rel(x, xo) <= 1e-10


def test_pair_fp32_basis(skf):
    A, bt, op, S, f, p, c, s = setup(skf, basis=torch.float32)
    (xf, xg, pf, pg), (i1, i2, i3, i4) = both(skf, op, S, bt, f, p)
    assert i3["status"] == 0 and i4["status"] == 0
    assert np.array_equal(xf, pf) and np.array_equal(xg, pg)


def test_pair_contour_rule(skf):
    """exp(-z): complex contour nodes (full-form tail, complex node solves),
    on the scaled operator of the contour tests (spectrum in [3.27, 23.8])."""
    import math
    A = convdiff_2d(12, (20.0, 10.0))
    op = skf.upload_csr(A.rowptr, A.colind, A.values / 50.0, device="cuda")
    bt = torch.as_tensor(np.ones(A.n) / math.sqrt(A.n), device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 160, 8, 13)
    f = skf.make_func("exp_neg", 0.1, alpha=0.5)
    p = skf.make_params(30, 2, ell1=48, ell2=64, tol=1e-12)
    (xf, xg, pf, pg), (i1, i2, i3, i4) = both(skf, op, S, bt, f, p)
    assert i3["status"] == 0 and i4["status"] == 0
    assert np.array_equal(xf, pf) and np.array_equal(xg, pg)


def test_pair_refuses_stopping_and_two_pass(skf):
    A, bt, op, S, f, p, c, s = setup(skf, n=30, m=10)
    for kw in ({"check_every": 5}, {"two_pass": True}):
        q = skf.make_params(10, 2, tol=1e-10, **kw)
        with pytest.raises(skf.SkfError, match="NOT_SUPPORTED"):
            skf.sfom_sgmres(op.csr, S, bt, f, q)
