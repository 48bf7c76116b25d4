"""Two-pass truncated Arnoldi (Sec. 4.2): the first pass keeps only a ring of
k + 2 basis vectors while it builds S V_m and S A V_m, the second repeats the
recurrence and accumulates f = sum_j y_j v_j.  The recurrence is
deterministic, so with an FP64 basis the result must equal the one-pass
result of the same (two-kernel) form of the Arnoldi process bit for bit, the
persistent form's to rounding, and the oracle's approximant to 1e-10; with an FP32 or
BF16 basis the two differ only in the recombination's summation (FP64 here,
double-float in the one-pass kernel)."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def setup(skf, dims, n, basis, kind=None, s=160):
    A = convdiff_2d(n, (100.0, 50.0)) if dims == 2 else convdiff_3d(n, (50.0, 50.0, 50.0))
    vals = A.values.astype(np.float32) if basis != torch.float64 else A.values
    op = skf.upload_csr(A.rowptr, A.colind, vals, device="cuda")
    b = torch.as_tensor(gaussian_rhs(A.n, 12), device="cuda")
    c = quad_scale("invsqrt", laplacian_lambda_min(n, dims), float(abs(csr_to_scipy(A)).sum(1).max()))
    S = skf.Sketch(kind if kind is not None else skf.SPARSE_SIGN, A.n, s, 8, 13)
    return A, op, b, c, S


def solve(skf, op, S, b, c, m, k, basis, method, two_pass, **kw):
    f = skf.make_func("invsqrt", c)
    p = skf.make_params(m, k, basis_dtype=basis, tol=1e-10, two_pass=two_pass, **kw)
    info = skf.new_info()
    x = skf.solve(method, op.csr, S, b, f, p, info=info)
    torch.cuda.synchronize()
    return x, skf.read_info(info)


@pytest.mark.parametrize("dims,n,m,k,method", [(2, 100, 40, 2, "sgmres"), (2, 100, 40, 2, "sfom"),
                                               (3, 30, 60, 3, "sgmres"), (2, 60, 33, 1, "sgmres")])
def test_fp64_two_pass_equals_one_pass_bitwise(skf, dims, n, m, k, method):
    A, op, b, c, S = setup(skf, dims, n, torch.float64, s=4 * m)
    meth = skf.SGMRES if method == "sgmres" else skf.SFOM
    with skf.arnoldi_mode(skf.ARNOLDI_TWO_KERNEL):
        x1, i1 = solve(skf, op, S, b, c, m, k, torch.float64, meth, False)
    x2, i2 = solve(skf, op, S, b, c, m, k, torch.float64, meth, True)
    assert torch.equal(x1, x2)
    assert i1 == i2
    # the default (persistent) one-pass form: the same approximant to rounding
    xp, ip = solve(skf, op, S, b, c, m, k, torch.float64, meth, False)
    assert rel(xp.cpu().numpy(), x2.cpu().numpy()) <= 1e-12 and ip["ell"] == i2["ell"]
    xo, _ = osk.solve(csr_to_scipy(A), b.cpu().numpy(), "invsqrt", m, k, OSketch("sparse_sign", A.n, 4 * m, 8, 13), c,
                      method=method if method == "sgmres" else "sfom_quad", tol=1e-10)
    assert rel(x2.cpu().numpy(), xo) <= 1e-10


def test_fp64_two_pass_srht_bitwise(skf):
    A, op, b, c, S = setup(skf, 2, 100, torch.float64, kind=skf.SRHT, s=160)
    x1, i1 = solve(skf, op, S, b, c, 40, 2, torch.float64, skf.SGMRES, False)
    x2, i2 = solve(skf, op, S, b, c, 40, 2, torch.float64, skf.SGMRES, True)
    assert torch.equal(x1, x2) and i1 == i2


@pytest.mark.parametrize("basis,tol", [(torch.float32, 1e-12), (torch.bfloat16, 1e-9)])
def test_reduced_precision_two_pass(skf, basis, tol):
    A, op, b, c, S = setup(skf, 3, 30, basis, s=240)
    # the two-pass mode runs the two-kernel Arnoldi form: compare in that form
    with skf.arnoldi_mode(skf.ARNOLDI_TWO_KERNEL):
        x1, i1 = solve(skf, op, S, b, c, 60, 2, basis, skf.SGMRES, False)
    x2, i2 = solve(skf, op, S, b, c, 60, 2, basis, skf.SGMRES, True)
    assert i1 == i2
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= tol


def test_two_pass_with_stopping_criterion(skf):
    A, op, b, c, S = setup(skf, 2, 40, torch.float64, s=480)
    x1, i1 = solve(skf, op, S, b, c, 120, 2, torch.float64, skf.SGMRES, False, check_every=10, stop_tol=1e-3)
    x2, i2 = solve(skf, op, S, b, c, 120, 2, torch.float64, skf.SGMRES, True, check_every=10, stop_tol=1e-3)
    assert i1["stop_m"] == 80 and i1 == i2
    assert torch.equal(x1, x2)


def test_two_pass_in_a_batch(skf):
    A, op, b, c, S = setup(skf, 2, 100, torch.float64, s=160)
    f = skf.make_func("invsqrt", c)
    probs, ref = [], []
    for tp in (True, False, True):
        p = skf.make_params(40, 2, tol=1e-10, two_pass=tp)
        probs.append((skf.SGMRES, op.csr, S, b, f, p, torch.empty_like(b), skf.new_info()))
        ref.append(skf.solve(skf.SGMRES, op.csr, S, b, f, p))
    skf.solve_batched(probs, lanes=3)
    torch.cuda.synchronize()
    for q, xr in zip(probs, ref):
        assert torch.equal(q[6], xr)
