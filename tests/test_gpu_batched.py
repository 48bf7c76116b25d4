"""Batched solves (skf_solve_batched): many independent f(A)b problems of
uneven size spread over the library's lane streams and, optionally, captured
into one CUDA graph.  Every problem's result must be bit-identical to its own
skf_solve call, and the FP64 ones agree with the oracle's approximant
(Algorithm 2, eq. (sGMRES), eq. (sFOM), quadrature of Sec. 4.1) to 1e-10."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def make_problems(skf, specs):
    """specs: (dims, n, nu, method, basis, m, s, rhs_seed, sketch_seed, func)."""
    ops, probs, keep = {}, [], []
    for dims, n, nu, method, basis, m, s, rseed, sseed, func in specs:
        key = (dims, n, nu, basis)
        if key not in ops:
            A = convdiff_2d(n, nu) if dims == 2 else convdiff_3d(n, nu)
            A32 = A.astype(np.float32)
            vals = A32.values if basis != torch.float64 else A32.values.astype(np.float64)
            ops[key] = (skf.upload_csr(A.rowptr, A.colind, vals, device="cuda"), A32)
        op, A32 = ops[key]
        lam_hi = float(abs(csr_to_scipy(A32)).sum(1).max())
        c = quad_scale(func, laplacian_lambda_min(n, dims), lam_hi)
        S = skf.Sketch(skf.SPARSE_SIGN, A32.n, s, 8, sseed)
        f = skf.make_func(func, c)
        p = skf.make_params(m, 2, basis_dtype=basis, tol=1e-11)
        b = torch.as_tensor(gaussian_rhs(A32.n, rseed), device="cuda")
        x = torch.full_like(b, float("nan"))
        info = skf.new_info()
        probs.append((method, op.csr, S, b, f, p, x, info))
        keep.append((A32, c, func, m, s, sseed, method, basis))
    return probs, ops, keep


SPECS = [
    (2, 40, (100.0, 50.0), 1, torch.float64, 30, 120, 1, 21, "invsqrt"),
    (2, 40, (100.0, 50.0), 0, torch.float64, 25, 100, 2, 22, "invsqrt"),
    (3, 12, (50.0, 50.0, 50.0), 1, torch.float64, 40, 160, 3, 23, "log1p_over_z"),
    (2, 40, (100.0, 50.0), 1, torch.float32, 45, 180, 4, 24, "invsqrt"),
    (3, 14, (20.0, 40.0, 30.0), 1, torch.float32, 60, 240, 5, 25, "invsqrt"),
    (3, 14, (20.0, 40.0, 30.0), 0, torch.float32, 20, 80, 6, 26, "invsqrt"),
    (2, 50, (30.0, 150.0), 1, torch.float32, 70, 280, 7, 27, "invsqrt"),
]


def individual(skf, probs):
    out = []
    for method, A, S, b, f, p, x, info in probs:
        xi = torch.empty_like(b)
        ii = skf.new_info()
        skf.solve(method, A, S, b, f, p, x=xi, info=ii)
        out.append((xi, ii))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("lanes", [1, 3, 16])
def test_batched_equals_individual_solves(skf, lanes):
    probs, ops, keep = make_problems(skf, SPECS)
    ref = individual(skf, probs)
    skf.solve_batched(probs, lanes=lanes)
    torch.cuda.synchronize()
    for (method, A, S, b, f, p, x, info), (xi, ii) in zip(probs, ref):
        assert torch.equal(x, xi)
        assert torch.equal(info, ii)
        assert skf.read_info(info)["status"] == 0


def test_batched_fp64_matches_oracle(skf):
    probs, ops, keep = make_problems(skf, SPECS[:3])
    skf.solve_batched(probs, lanes=3)
    torch.cuda.synchronize()
    for (method, A, S, b, f, p, x, info), (A32, c, func, m, s, sseed, _, basis) in zip(probs, keep):
        Asp = csr_to_scipy(A32.astype(np.float64))
        xo, _ = osk.solve(Asp, b.cpu().numpy(), func, m, 2, OSketch("sparse_sign", A32.n, s, 8, sseed), c,
                          method="sgmres" if method == 1 else "sfom_quad", tol=1e-11)
        assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_batch_graph_replays_with_new_right_hand_sides(skf):
    probs, ops, keep = make_problems(skf, SPECS[2:6])
    g = skf.BatchGraph(probs, lanes=2)
    for q in probs:      # new data in place; the graph reads b at replay
        q[3].copy_(torch.as_tensor(gaussian_rhs(q[3].numel(), 1000 + q[3].numel()), device="cuda"))
        q[6].fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    ref = individual(skf, probs)
    for q, (xi, ii) in zip(probs, ref):
        assert torch.equal(q[6], xi)
    g.replay()           # replays are repeatable
    torch.cuda.synchronize()
    for q, (xi, ii) in zip(probs, ref):
        assert torch.equal(q[6], xi)


def test_batched_error_names_problem_and_enqueues_nothing(skf):
    probs, ops, keep = make_problems(skf, SPECS[:2])
    bad = list(probs)
    method, A, S, b, f, p, x, info = bad[1]
    bad[1] = (method, A, S, b, f, skf.make_params(200, 2), x, info)   # m >= s
    x0 = probs[0][6]
    x0.fill_(7.0)
    with pytest.raises(skf.SkfError) as e:
        skf.solve_batched(bad, lanes=2)
    assert "problem 1" in str(e.value)
    torch.cuda.synchronize()
    assert bool((x0 == 7.0).all())
