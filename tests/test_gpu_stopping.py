"""The sketched stopping criterion of Sec. 4.3 on the GPU against the oracle
(oracle.stopping): the checkpoint where the process stops, the estimate
there, and the returned iterate.  Cases are chosen so that the accepted
estimate and the one before it are far from the tolerance (the decision is
not a rounding tie)."""
import numpy as np
import pytest
import torch

from oracle import stopping as ost
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu

CASES = {
    "2d": (2, 40, (100.0, 50.0), 120, 10, 1e-3, 80),
    "3d": (3, 20, (50.0, 50.0, 50.0), 120, 10, 1e-3, 60),
}


def problem(skf, key, basis):
    dims, n, nu, m, d, tol, p_expect = CASES[key]
    A = convdiff_2d(n, nu) if dims == 2 else convdiff_3d(n, nu)
    vals = A.values.astype(np.float32) if basis == torch.float32 else A.values
    op = skf.upload_csr(A.rowptr, A.colind, vals, device="cuda")
    As = csr_to_scipy(A.astype(np.float32).astype(np.float64) if basis == torch.float32 else A)
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", laplacian_lambda_min(n, dims), float(abs(As).sum(1).max()))
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 4 * m, 8, 13)
    return op, As, b, c, S, m, d, tol, p_expect


def gpu(skf, op, S, b, c, m, basis, method, check_every=0, stop_tol=0.0):
    f = skf.make_func("invsqrt", c)
    p = skf.make_params(m, 2, basis_dtype=basis, tol=1e-10, check_every=check_every, stop_tol=stop_tol)
    info = skf.new_info()
    x = skf.solve(method, op.csr, S, torch.as_tensor(b, device="cuda"), f, p, info=info)
    torch.cuda.synchronize()
    return x, skf.read_info(info)


@pytest.mark.parametrize("key,method", [("2d", "sgmres"), ("3d", "sgmres"), ("2d", "sfom")])
def test_fp64_stop_matches_oracle(skf, key, method):
    op, As, b, c, S, m, d, tol, p_expect = problem(skf, key, torch.float64)
    meth = skf.SGMRES if method == "sgmres" else skf.SFOM
    xo, oi = ost.solve_with_stopping(As, b, "invsqrt", m, 2, OSketch("sparse_sign", As.shape[0], 4 * m, 8, 13), c,
                                     d=d, tol=tol, method="sgmres" if method == "sgmres" else "sfom_quad")
    assert oi["stopped"]
    if method == "sgmres":
        assert oi["p"] == p_expect
    # the decision is not a tie: the estimates straddle the tolerance widely
    assert oi["history"][-1][1] < 0.5 * tol and all(r > 2 * tol for _, r in oi["history"][:-1])
    x, info = gpu(skf, op, S, b, c, m, torch.float64, meth, d, tol)
    assert info["status"] == 0
    assert info["stop_m"] == oi["p"] and info["m_eff"] == oi["p"] and info["breakdown"] == 0
    assert info["err_est"] == pytest.approx(oi["history"][-1][1], rel=1e-6)
    assert rel(x.cpu().numpy(), xo) <= 1e-10
    # the stopped iterate is the plain solve with m = p, bit for bit in the
    # same (two-kernel) form of the Arnoldi process (the recurrence is
    # prefix-consistent and the tail sees the same columns), and to rounding in
    # the persistent form a plain solve takes by default
    with skf.arnoldi_mode(skf.ARNOLDI_TWO_KERNEL):
        xp, ip = gpu(skf, op, S, b, c, oi["p"], torch.float64, meth)
    assert torch.equal(x, xp)
    xq, iq = gpu(skf, op, S, b, c, oi["p"], torch.float64, meth)
    assert rel(xq.cpu().numpy(), x.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("key", ["2d", "3d"])
def test_fp32_basis_stop_matches_oracle(skf, key):
    op, As, b, c, S, m, d, tol, p_expect = problem(skf, key, torch.float32)
    xo, oi = ost.solve_with_stopping(As, b, "invsqrt", m, 2, OSketch("sparse_sign", As.shape[0], 4 * m, 8, 13), c,
                                     d=d, tol=tol)
    x, info = gpu(skf, op, S, b, c, m, torch.float32, skf.SGMRES, d, tol)
    assert info["status"] == 0
    assert info["stop_m"] == oi["p"] == p_expect
    assert info["err_est"] == pytest.approx(oi["history"][-1][1], rel=1e-2)
    assert rel(x.cpu().numpy(), xo) <= 1e-5


@pytest.mark.parametrize("basis", [torch.float64, torch.float32])
def test_checks_that_never_stop_leave_the_result_unchanged(skf, basis):
    """stop_tol = 0: every checkpoint runs, none stops; the result is the plain
    m-column solve bit for bit and the last estimate is reported."""
    op, As, b, c, S, m, d, tol, p_expect = problem(skf, "3d", basis)
    x, info = gpu(skf, op, S, b, c, m, basis, skf.SGMRES, d, 0.0)
    with skf.arnoldi_mode(skf.ARNOLDI_TWO_KERNEL):       # the form the checkpoints run in
        x0, i0 = gpu(skf, op, S, b, c, m, basis, skf.SGMRES)
    assert torch.equal(x, x0)
    assert info["stop_m"] == 0 and info["m_eff"] == m
    assert 0.0 < info["err_est"] < 1e-4
    assert i0["stop_m"] == 0 and i0["err_est"] == 0.0


def test_stopping_inside_a_batch(skf):
    op, As, b, c, S, m, d, tol, p_expect = problem(skf, "2d", torch.float64)
    f = skf.make_func("invsqrt", c)
    bt = torch.as_tensor(b, device="cuda")
    probs, ref = [], []
    for ce, st in ((d, tol), (0, 0.0)):
        p = skf.make_params(m, 2, tol=1e-10, check_every=ce, stop_tol=st)
        x = torch.empty_like(bt)
        info = skf.new_info()
        probs.append((skf.SGMRES, op.csr, S, bt, f, p, x, info))
        xi = skf.solve(skf.SGMRES, op.csr, S, bt, f, p)
        ref.append(xi)
    skf.solve_batched(probs, lanes=2)
    torch.cuda.synchronize()
    for q, xi in zip(probs, ref):
        assert torch.equal(q[6], xi)
    assert skf.read_info(probs[0][7])["stop_m"] == p_expect
