"""Parity at the full size of the default benchmark workload, in the
configuration bench.py times: 3D convection-diffusion on a 100^3 grid
(N = 1e6, nnz = 6.94e6), f(z) = log(1+z)/z, m = 200, k = 2, sparse-sign
sketch with s = 800 and zeta = 8, FP64 basis, the adaptive quadrature with
tol = 1e-10.  The oracle runs on the same seeded inputs (its solve takes tens
of seconds on the host cores, so one method is compared at this size; both
are compared at the smaller configurations)."""
import pytest
import torch

from oracle import sketched as osk
from oracle.sketch import Sketch as OSketch
from workloads import WORKLOADS, csr_to_scipy
from workloads.configs import quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def test_default_workload_full_size_sgmres_matches_oracle(skf):
    wl = WORKLOADS["cd3d_n100"]
    A = wl.operator()
    b = wl.rhs(A.n)
    assert A.n == 1_000_000 and wl.m == 200 and wl.k == 2 and wl.s == 800 and wl.zeta == 8
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    c = quad_scale(wl.func, wl.lam_lo or 0.0, op.csr.norm_inf())
    f = skf.make_func(wl.func, c)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, wl.s, wl.zeta, 13)
    p = skf.make_params(wl.m, wl.k, tol=1e-10)
    info = skf.new_info()
    x = skf.solve(skf.SGMRES, op.csr, S, torch.as_tensor(b, device="cuda"), f, p, info=info)
    torch.cuda.synchronize()
    gi = skf.read_info(info)
    assert gi["status"] == 0 and gi["m_eff"] == wl.m
    xo, oi = osk.solve(csr_to_scipy(A), b, wl.func, wl.m, wl.k, OSketch("sparse_sign", A.n, wl.s, wl.zeta, 13), c,
                       method="sgmres", tol=1e-10)
    # FP64 path: relative 2-norm error against the oracle at most 1e-10
    assert rel(x.cpu().numpy(), xo) <= 1e-10
