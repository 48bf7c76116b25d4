"""The library's workspace pool: repeated solves re-use cached blocks (same
results bit for bit), skf_workspace_trim releases them, and a solve after a
trim maps new blocks and still gives the same result."""
import numpy as np
import pytest
import torch

from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import upload

pytestmark = pytest.mark.gpu


def test_workspace_reuse_and_trim(skf):
    A = convdiff_2d(120, (60.0, 30.0))
    b = torch.as_tensor(gaussian_rhs(A.n, 3), device="cuda")
    op = upload(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 200, 8, 13)
    c = quad_scale("invsqrt", laplacian_lambda_min(120, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    f = skf.make_func("invsqrt", c)
    p = skf.make_params(50, 2, tol=1e-10)
    xs = []
    for i in range(4):
        if i == 2:
            torch.cuda.synchronize()
            skf.workspace_trim()
        xs.append(skf.sgmres(op.csr, S, b, f, p).cpu().numpy())
        torch.cuda.synchronize()
    for x in xs[1:]:
        assert np.array_equal(x, xs[0])
    assert np.isfinite(xs[0]).all() and np.linalg.norm(xs[0]) > 0
