"""Non-Stieltjes f through a contour (Algorithm 2 with a fixed contour; the
parabola of Sec. 5.2): f(z) = exp(-z) with complex quadrature nodes, the node
systems solved through their real 2m x 2m form.  GPU against the oracle on
the same sketch and adaptive schedule (FP64: 1e-10), and convergence to
expm(-A) b."""
import math

import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.exact import fAb_dense
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, csr_to_scipy
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def problem(skf, n, scale):
    A = convdiff_2d(n, (20.0, 10.0))
    As = csr_to_scipy(A) / scale
    op = skf.upload_csr(A.rowptr, A.colind, A.values / scale, device="cuda")
    b = np.ones(A.n) / math.sqrt(A.n)
    return A, As, op, b


@pytest.mark.parametrize("m,method", [(5, "sgmres"), (10, "sgmres"), (30, "sgmres"), (10, "sfom"), (30, "sfom")])
def test_contour_matches_oracle(skf, m, method):
    A, As, op, b = problem(skf, 12, 50.0)          # real spectrum in [3.27, 23.8]
    c, a = 0.1, 0.5
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 160, 8, 13)
    f = skf.make_func("exp_neg", c, alpha=a)
    p = skf.make_params(m, 2, ell1=48, ell2=64, tol=1e-12)
    info = skf.new_info()
    meth = skf.SGMRES if method == "sgmres" else skf.SFOM
    x = skf.solve(meth, op.csr, S, torch.as_tensor(b, device="cuda"), f, p, info=info).cpu().numpy()
    xo, oi = osk.solve(As, b, "exp_neg", m, 2, OSketch("sparse_sign", A.n, 160, 8, 13), c,
                       method=method if method == "sgmres" else "sfom_quad", ell1=48, ell2=64, tol=1e-12, alpha=a)
    inf = skf.read_info(info)
    assert inf["status"] == 0 and inf["ell"] == oi["ell"]
    assert rel(x, xo) <= 1e-10


def test_contour_converges_to_expm(skf):
    A, As, op, b = problem(skf, 30, 300.0)
    ref = fAb_dense(As.toarray(), b, "exp_neg")
    ev = np.linalg.eigvals(As.toarray())
    assert ev.real.min() > 0.2 and abs(ev.imag).max() < 1e-8
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 240, 8, 13)
    f = skf.make_func("exp_neg", 0.1, alpha=0.5)
    errs = []
    for m in (10, 30, 60):
        x = skf.sgmres(op.csr, S, torch.as_tensor(b, device="cuda"), f, skf.make_params(m, 2, ell1=48, ell2=64,
                                                                                      tol=1e-12))
        errs.append(rel(x.cpu().numpy(), ref))
    # oracle on the same problem: 2.3e-2, 4.9e-5, 3.4e-14
    assert errs[2] < 1e-11 and errs[2] < 1e-9 * errs[0]
