"""skf_solve_block: a block of right-hand sides on one operator (Algorithm 2
and the tail for every column).  In the lockstep form (skf_set_block_mode(1))
with an FP32 basis the Arnoldi processes advance together, one SpMM per step
and group of four columns (the two-kernel Arnoldi form of each column); in
both forms every column must be bit-identical to its own skf_solve call in
the same Arnoldi form, including a zero column (stopped at step 0 while
the others go on), a block of five (groups of four and one) and both methods;
the FP32 results stay within max(1e-6, 2^-24 cond(R)) of the FP64 oracle; an
FP64 basis solves the columns one after another (also bit-identical)."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def block_case(skf, A, dims, n, nrhs, m, basis, zero_col=None):
    vals = A.values.astype(np.float32 if basis == torch.float32 else np.float64)
    op = skf.upload_csr(A.rowptr, A.colind, vals, device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 4 * m, 8, 13)
    c = quad_scale("invsqrt", laplacian_lambda_min(n, dims), float(abs(csr_to_scipy(A)).sum(1).max()))
    f = skf.make_func("invsqrt", c)
    p = skf.make_params(m, 2, basis_dtype=basis, tol=1e-12)
    Bh = np.stack([gaussian_rhs(A.n, 40 + q) for q in range(nrhs)])
    if zero_col is not None:
        Bh[zero_col] = 0.0
    B = torch.as_tensor(Bh, device="cuda").contiguous()
    return op, S, c, f, p, Bh, B


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_block_fp32_bitwise_equals_single_solves(skf, method, mode):
    n, nrhs, m = 90, 5, 40
    A = convdiff_2d(n, (100.0, 50.0)).astype(np.float32)
    op, S, c, f, p, Bh, B = block_case(skf, A, 2, n, nrhs, m, torch.float32, zero_col=2)
    meth = skf.SGMRES if method == "sgmres" else skf.SFOM
    info = skf.new_info_block(nrhs)
    with skf.block_mode(mode):
        X = skf.solve_block(meth, op.csr, S, B, f, p, info=info)
        torch.cuda.synchronize()
    OS = OSketch("sparse_sign", A.n, 4 * m, 8, 13)
    # the lockstep form runs the two-kernel Arnoldi form of every column
    form = skf.ARNOLDI_TWO_KERNEL if mode == 1 else skf.ARNOLDI_AUTO
    for q in range(nrhs):
        iq = skf.new_info()
        with skf.arnoldi_mode(form):
            xq = skf.solve(meth, op.csr, S, B[q].clone(), f, p, info=iq)
            torch.cuda.synchronize()
        bq = skf.read_info(info[q])
        sq = skf.read_info(iq)
        assert torch.equal(X[q], xq), q
        assert bq["status"] == sq["status"] and bq["m_eff"] == sq["m_eff"] and bq["ell"] == sq["ell"]
        if q == 2:
            assert bq["status_name"] == "SKF_ERR_ZERO_RHS" and not torch.any(X[q])
        else:
            assert bq["status"] == 0
            xo, _ = osk.solve(csr_to_scipy(A), Bh[q], "invsqrt", m, 2, OS, c,
                              method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
            assert rel(X[q].cpu().numpy(), xo) <= max(1e-6, 2.0 ** -24 * bq["cond_est"])


def test_block_fp32_3d_many_chunks(skf):
    """3D operator with several 1024-row chunks per CTA (N = 274625): eight
    columns, two full SpMM groups."""
    n, nrhs, m = 65, 8, 24
    A = convdiff_3d(n, (50.0, 20.0, 80.0)).astype(np.float32)
    op, S, c, f, p, Bh, B = block_case(skf, A, 3, n, nrhs, m, torch.float32)
    with skf.block_mode(1):
        X = skf.solve_block(skf.SGMRES, op.csr, S, B, f, p)
        torch.cuda.synchronize()
    for q in range(nrhs):
        with skf.arnoldi_mode(skf.ARNOLDI_TWO_KERNEL):
            xq = skf.solve(skf.SGMRES, op.csr, S, B[q].clone(), f, p)
            torch.cuda.synchronize()
        assert torch.equal(X[q], xq), q


def test_block_fp64_columns_one_after_another(skf):
    n, nrhs, m = 60, 3, 30
    A = convdiff_2d(n, (80.0, 20.0)).astype(np.float32)
    op, S, c, f, p, Bh, B = block_case(skf, A, 2, n, nrhs, m, torch.float64)
    with skf.block_mode(1):
        X = skf.solve_block(skf.SGMRES, op.csr, S, B, f, p)
        torch.cuda.synchronize()
    for q in range(nrhs):
        xq = skf.solve(skf.SGMRES, op.csr, S, B[q].clone(), f, p)
        torch.cuda.synchronize()
        assert torch.equal(X[q], xq), q


def test_block_rejects_bad_arguments(skf):
    A = convdiff_2d(20).astype(np.float32)
    op, S, c, f, p, Bh, B = block_case(skf, A, 2, 20, 2, 8, torch.float32)
    lib = skf.lib()
    X = torch.empty_like(B)
    st = lib.skf_solve_block(skf.SGMRES, op.csr.handle, S.handle, skf._ptr(B), A.n - 1, 2, skf.ctypes.byref(f),
                             skf.ctypes.byref(p), skf._ptr(X), A.n, None, None)
    assert st != 0
    assert skf.solve_block(skf.SGMRES, op.csr, S, B[:0], f, p).shape == (0, A.n)
    assert lib.skf_set_block_mode(2) != 0 and lib.skf_set_block_mode(0) == 0
