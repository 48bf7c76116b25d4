"""Parity at the full size of the default benchmark workload, in the
configuration bench.py times: 3D convection-diffusion on a 100^3 grid
(N = 1e6, nnz = 6.94e6), f(z) = log(1+z)/z, m = 200, k = 2, sparse-sign
sketch with s = 800 and zeta = 8, FP64 basis, the adaptive quadrature with
tol = 1e-10.  The oracle's Arnoldi process runs once on the same seeded
inputs (tens of seconds on the host cores); its sGMRES and sFOM tails are
compared with the library's solves in both forms of the Arnoldi process (the
persistent form is the one bench.py times)."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.arnoldi import arnoldi_trunc
from oracle.sketch import Sketch as OSketch
from workloads import WORKLOADS, csr_to_scipy
from workloads.configs import quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def full(skf):
    wl = WORKLOADS["cd3d_n100"]
    A = wl.operator()
    b = wl.rhs(A.n)
    assert A.n == 1_000_000 and wl.m == 200 and wl.k == 2 and wl.s == 800 and wl.zeta == 8
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    c = quad_scale(wl.func, wl.lam_lo or 0.0, op.csr.norm_inf())
    OS = OSketch("sparse_sign", A.n, wl.s, wl.zeta, 13)
    ar = arnoldi_trunc(csr_to_scipy(A), b, wl.m, wl.k, OS)
    W = osk.whiten(ar["SV"], ar["SAV"], OS @ b)
    y_g, ell_g = osk.sgmres_quadrature(W, wl.func, c, tol=1e-10)
    y_f, ell_f = osk.sfom_quadrature(W, wl.func, c, tol=1e-10)
    ref = {"sgmres": (ar["V"] @ y_g, ell_g), "sfom": (ar["V"] @ y_f, ell_f)}
    return {"wl": wl, "A": A, "b": b, "op": op, "c": c, "ref": ref, "condR": W["condR"]}


def gpu_solve(skf, F, method, mode):
    wl = F["wl"]
    f = skf.make_func(wl.func, F["c"])
    S = skf.Sketch(skf.SPARSE_SIGN, F["A"].n, wl.s, wl.zeta, 13)
    p = skf.make_params(wl.m, wl.k, tol=1e-10)
    info = skf.new_info()
    with skf.arnoldi_mode(mode):
        x = skf.solve(skf.SGMRES if method == "sgmres" else skf.SFOM, F["op"].csr, S,
                      torch.as_tensor(F["b"], device="cuda"), f, p, info=info)
        torch.cuda.synchronize()
    return x.cpu().numpy(), skf.read_info(info)


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
@pytest.mark.parametrize("mode", ["persistent", "two_kernel"])
def test_default_workload_full_size_matches_oracle(skf, full, method, mode):
    x, gi = gpu_solve(skf, full, method,
                      skf.ARNOLDI_PERSISTENT if mode == "persistent" else skf.ARNOLDI_TWO_KERNEL)
    assert gi["status"] == 0 and gi["m_eff"] == full["wl"].m
    xo, ell = full["ref"][method]
    err = rel(x, xo)
    print(f"{method} {mode}: rel err vs oracle {err:.3e}, ell {gi['ell']} (oracle {ell}), "
          f"cond(R) {full['condR']:.3e}")
    # FP64 path: relative 2-norm error against the oracle at most 1e-10 where
    # the basis conditioning allows it (cond(V_m) u <= 1e-12; cond(R) = cond(S V_m)
    # tracks cond(V_m) within the embedding's distortion)
    assert full["condR"] * U <= 1e-12
    assert err <= 1e-10


def test_default_workload_pair_matches_oracle(skf, full):
    """The pair call bench.py times: both approximants from one Arnoldi
    process (persistent form), each against the oracle."""
    wl = full["wl"]
    f = skf.make_func(wl.func, full["c"])
    S = skf.Sketch(skf.SPARSE_SIGN, full["A"].n, wl.s, wl.zeta, 13)
    p = skf.make_params(wl.m, wl.k, tol=1e-10)
    i_f, i_g = skf.new_info(), skf.new_info()
    xf, xg = skf.sfom_sgmres(full["op"].csr, S, torch.as_tensor(full["b"], device="cuda"), f, p,
                             info_fom=i_f, info_gmres=i_g)
    torch.cuda.synchronize()
    for x, info, method in ((xf, i_f, "sfom"), (xg, i_g, "sgmres")):
        gi = skf.read_info(info)
        xo, ell = full["ref"][method]
        assert gi["status"] == 0 and gi["m_eff"] == wl.m and gi["ell"] == ell
        assert rel(x.cpu().numpy(), xo) <= 1e-10
