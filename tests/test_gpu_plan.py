"""The precision plan of the batched form (skf_plan_basis_precision): per
problem, the condition estimate of the whitening R of a pilot basis
(S V_m = Q R, Sec. 2.1 and Sec. 3) and the choice of an FP32 basis where
cond(R) 2^-24 <= tol.

Checked here: the estimate for each problem equals the one a solve of the
pilot problem at that problem's m reports (the pilot's leading columns are
that shorter Arnoldi process); the flag follows the rule; and every problem
the plan sends to FP32 does stay within tol of its FP64-basis result."""
import numpy as np
import pytest
import torch

from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
TOL = 1e-6

# (dims, n, nu, [m of the problems on this operator])
OPERATORS = [
    (2, 60, (100.0, 50.0), [20, 45, 90]),
    (3, 16, (150.0, 20.0, 40.0), [30, 70]),
]


def build(skf, basis):
    """One problem per (operator, m): FP32-rounded operator values (FP32
    storage for an FP32 basis, the same values in FP64 otherwise)."""
    probs, meta = [], []
    for oi, (dims, n, nu, ms) in enumerate(OPERATORS):
        A = (convdiff_2d(n, nu) if dims == 2 else convdiff_3d(n, nu)).astype(np.float32)
        vals = A.values if basis == torch.float32 else A.values.astype(np.float64)
        op = skf.upload_csr(A.rowptr, A.colind, vals, device="cuda")
        c = quad_scale("invsqrt", laplacian_lambda_min(n, dims), float(abs(csr_to_scipy(A)).sum(1).max()))
        f = skf.make_func("invsqrt", c)
        for qi, m in enumerate(ms):
            S = skf.Sketch(skf.SPARSE_SIGN, A.n, 4 * m, 8, 100 + 10 * oi + qi)
            p = skf.make_params(m, 2, basis_dtype=basis, tol=1e-10)
            b = torch.as_tensor(gaussian_rhs(A.n, 50 + 10 * oi + qi), device="cuda")
            probs.append((skf.SGMRES, op.csr, S, b, f, p, torch.empty_like(b), skf.new_info()))
            meta.append((oi, m, op))
    return probs, meta


@pytest.mark.parametrize("basis", [torch.float32, torch.float64])
def test_plan_estimates_are_the_pilot_whitening(skf, basis):
    probs, meta = build(skf, basis)
    cond, f32 = skf.plan_basis_precision(probs, TOL)
    assert len(cond) == len(probs)
    for r, ((oi, m, op), cnd, fl) in enumerate(zip(meta, cond, f32)):
        assert cnd >= 1.0 and np.isfinite(cnd)
        assert fl == (cnd * U32 <= TOL)
        # the pilot of operator oi is its problem with the largest m
        grp = [i for i, mm in enumerate(meta) if mm[0] == oi]
        pl = max(grp, key=lambda i: meta[i][1])
        method, A, S, b, f, p, x, info = probs[pl]
        pm = skf.make_params(m, 2, basis_dtype=basis, tol=1e-10)
        ii = skf.new_info()
        skf.solve(method, A, S, b, f, pm, info=ii)
        torch.cuda.synchronize()
        ref = skf.read_info(ii)["cond_est"]
        print(f"op {oi} m {m}: plan cond {cnd:.4e}, pilot solve at m {ref:.4e}, f32 {fl}")
        assert abs(cnd - ref) <= 1e-3 * ref


def test_plan_fp32_choices_meet_tol(skf):
    p32, meta = build(skf, torch.float32)
    p64, _ = build(skf, torch.float64)
    cond, f32 = skf.plan_basis_precision(p32, TOL)
    assert any(f32) and not all(f32)
    for r, (q32, q64) in enumerate(zip(p32, p64)):
        x32 = skf.solve(q32[0], q32[1], q32[2], q32[3], q32[4], q32[5])
        x64 = skf.solve(q64[0], q64[1], q64[2], q64[3], q64[4], q64[5])
        torch.cuda.synchronize()
        err = rel(x32.cpu().numpy(), x64.cpu().numpy())
        print(f"problem {r} (op {meta[r][0]}, m {meta[r][1]}): cond {cond[r]:.3e}, f32 {f32[r]}, err {err:.3e}")
        if f32[r]:
            assert err <= TOL


def test_plan_rejects_bad_arguments(skf):
    probs, _ = build(skf, torch.float64)
    with pytest.raises(skf.SkfError, match="INVALID_ARG"):
        skf.plan_basis_precision(probs, 0.0)
    assert skf.plan_basis_precision([], TOL) == ([], [])
