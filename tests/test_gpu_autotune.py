"""The slice layouts the autotuner chooses among (row-split cut 16, 32, 64;
unsorted and sorted slices) all give the oracle's Arnoldi process and solves
on the power-law out-degree graph (Algorithm 2; eq. (sGMRES)), in FP64 and
with an FP32 basis; the autotuner keeps one of them and the solve after it
still matches."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.sketch import Sketch as OSketch
from workloads import csr_to_scipy, gaussian_rhs, powerlaw_graph_operator
from workloads.configs import quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu

LAYOUTS = [(c, s) for s in (0, 1) for c in (16, 32, 64)]


@pytest.fixture(scope="module")
def graph():
    A = powerlaw_graph_operator(20000, seed=11, transpose=True)
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", 0.1, float(abs(csr_to_scipy(A)).sum(1).max()))
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", 10, 2, OSketch("sparse_sign", A.n, 40, 8, 13), c,
                      method="sgmres", tol=1e-12)
    return A, b, c, xo


def solve(skf, op, A, b, c, basis):
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 40, 8, 13)
    p = skf.make_params(10, 2, basis_dtype=basis, tol=1e-12 if basis == torch.float64 else 1e-10)
    info = skf.new_info()
    x = skf.sgmres(op.csr, S, torch.as_tensor(b, device="cuda"), skf.make_func("invsqrt", c), p, info=info)
    torch.cuda.synchronize()
    assert skf.read_info(info)["status"] == 0
    return x.cpu().numpy()


@pytest.mark.parametrize("basis", [torch.float64, torch.float32])
def test_every_layout_matches_oracle(skf, graph, basis):
    A, b, c, xo = graph
    vals = A.values if basis == torch.float64 else A.values.astype(np.float32)
    op = skf.upload_csr(A.rowptr, A.colind, vals, device="cuda")
    tol = 1e-10 if basis == torch.float64 else 1e-6
    for cut, srt in LAYOUTS:
        skf.csr_set_layout(op.csr, cut, srt)
        assert rel(solve(skf, op, A, b, c, basis), xo) <= tol, (cut, srt)


@pytest.mark.parametrize("basis", [torch.float64, torch.float32])
def test_autotune_keeps_a_candidate(skf, graph, basis):
    A, b, c, xo = graph
    vals = A.values if basis == torch.float64 else A.values.astype(np.float32)
    op = skf.upload_csr(A.rowptr, A.colind, vals, device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 40, 8, 13)
    r = skf.csr_autotune(op.csr, S, 2, basis_dtype=basis, m_probe=6)
    t = r["times_us"]
    assert all(np.isfinite(t)) and min(t) > 0
    assert r["choice"] in skf.AUTOTUNE_CANDIDATES
    k = skf.AUTOTUNE_CANDIDATES.index(r["choice"])
    assert t[k] == min(t)
    tol = 1e-10 if basis == torch.float64 else 1e-6
    assert rel(solve(skf, op, A, b, c, basis), xo) <= tol


def test_set_layout_rejects_bad_arguments(skf):
    A = powerlaw_graph_operator(1000, seed=11, transpose=True)
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    with pytest.raises(skf.SkfError, match="INVALID_ARG"):
        skf.csr_set_layout(op.csr, 0, 0)
    with pytest.raises(skf.SkfError, match="INVALID_ARG"):
        skf.csr_set_layout(op.csr, 32, 2)
