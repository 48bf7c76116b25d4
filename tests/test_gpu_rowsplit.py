"""Row split for skewed rows: the power-law graph operator with rows carrying
the out-degrees (Zipf(2.1), hubs of thousands of entries).  Rows longer than
32 entries leave the SELL slices and are reduced segment by segment (one
warp per <= 1024 entries); the SpMV adds their partials.  FP64 Arnoldi
columns and solves against the oracle (Algorithm 2; eq. (sGMRES), eq. (sFOM)),
and the FP32 path against the oracle at the stated tolerance of the
reduced-precision graph workload."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.arnoldi import arnoldi_trunc as o_arnoldi
from oracle.sketch import Sketch as OSketch
from workloads import csr_to_scipy, gaussian_rhs, powerlaw_graph_operator
from workloads.configs import quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu

# FP32 values and basis on the skewed graph, relative 2-norm error against
# the FP64 oracle (the reduced-precision graph workload's tolerance)
TOL_GRAPH_FP32 = 1e-6


@pytest.fixture(scope="module")
def graph():
    A = powerlaw_graph_operator(20000, seed=11, transpose=True)
    L = np.diff(A.rowptr)
    assert (L > 32).sum() > 100 and L.max() > 4 * 1024      # long rows, and hubs of several segments
    return A, gaussian_rhs(A.n, 12)


def test_rowsplit_arnoldi_columns(skf, graph):
    A, b = graph
    m, k, s = 10, 2, 40
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    info = skf.new_info()
    V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, torch.as_tensor(b, device="cuda"), m, k, info=info)
    torch.cuda.synchronize()
    g = {"V": (V.double() * vs[:, None]).cpu().numpy().T, "SV": SV.cpu().numpy().T, "SAV": SAV.cpu().numpy().T}
    ar = o_arnoldi(csr_to_scipy(A), b, m, k, OSketch("sparse_sign", A.n, s, 8, 13))
    assert skf.read_info(info)["status"] == 0
    for j in range(m):
        for key in ("V", "SV", "SAV"):
            assert rel(g[key][:, j], ar[key][:, j]) < 1e-10, (key, j)
    Hg, Ho = H.cpu().numpy().T[: m + 1, :m], ar["H"]
    assert np.abs(Hg[:, : m - 1] - Ho[:, : m - 1]).max() <= 1e-10 * np.abs(Ho).max()


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_rowsplit_solve_fp64(skf, graph, method):
    A, b = graph
    m, k, s = 10, 2, 40
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    c = quad_scale("invsqrt", 0.1, float(abs(csr_to_scipy(A)).sum(1).max()))
    f = skf.make_func("invsqrt", c)
    p = skf.make_params(m, k, tol=1e-12)
    info = skf.new_info()
    x = skf.solve(skf.SGMRES if method == "sgmres" else skf.SFOM, op.csr, S, torch.as_tensor(b, device="cuda"), f, p,
                  info=info)
    torch.cuda.synchronize()
    xo, oi = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                       method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    st = skf.read_info(info)
    assert st["status"] == 0 and st["ell"] == oi["ell"]
    assert oi["condR"] * 2.0 ** -53 <= 1e-12
    assert rel(x.cpu().numpy(), xo) <= 1e-10


@pytest.mark.parametrize("k", [2, 3])
def test_rowsplit_solve_fp32(skf, graph, k):
    A, b = graph
    m, s = 10, 40
    op = skf.upload_csr(A.rowptr, A.colind, A.values.astype(np.float32), device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    c = quad_scale("invsqrt", 0.1, float(abs(csr_to_scipy(A)).sum(1).max()))
    f = skf.make_func("invsqrt", c)
    p = skf.make_params(m, k, basis_dtype=torch.float32, tol=1e-10)
    info = skf.new_info()
    x = skf.sgmres(op.csr, S, torch.as_tensor(b, device="cuda"), f, p, info=info)
    torch.cuda.synchronize()
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                      method="sgmres", tol=1e-10)
    err = rel(x.cpu().numpy(), xo)
    print(f"graph N=20000 transpose k={k}: FP32 rel err vs oracle {err:.2e}")
    assert skf.read_info(info)["status"] == 0
    assert err <= TOL_GRAPH_FP32
