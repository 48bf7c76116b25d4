"""SRDCT sketch (Sec. 5.1: S = P F E with a DCT) on the GPU against the oracle,
and the paper's convection-diffusion experiment (Sec. 5.1, Fig. 1: upwind
operator, n = 100, D = 1e-3, b the normalised vector of ones, k = 4,
s = 2 m_max = 400, Gauss-Chebyshev rule with 45 nodes after t = (1-x)/(1+x))
reproduced qualitatively: the sketched approximants follow the error of the
best approximation from K_m(A, b), sGMRES closely, and the sFOM quadrature
form agrees with the closed form to the rule's error."""
import numpy as np
import pytest
import torch

from oracle import quadrature as oq
from oracle import sketched as osk
from oracle.arnoldi import arnoldi_trunc
from oracle.exact import fAb_shifted
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs, upwind_2d
from workloads.configs import laplacian_lambda_min, quad_scale
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


# N with no prime factor above 7 takes the FFT form (Makhoul's reordering;
# even N packs the real input two to an entry and transforms N / 2 entries;
# Stockham passes of radices 4, 2, 3, 5, 7): 2 (one entry, no pass),
# 12 -> 6 = [2, 3], 210 -> 105 = [3, 5, 7], 1000 -> 500 = [4, 5, 5, 5],
# 125000 -> 62500 = [4, 5 x 6]; odd N transforms N entries: 7 = [7],
# 4725 = [3, 3, 3, 5, 5, 7].  1013 (prime) and 9409 = 97^2 take the direct form
@pytest.mark.parametrize("N,s,ncols", [(1, 1, 1), (2, 2, 1), (7, 5, 3), (12, 7, 2), (210, 50, 2), (1000, 200, 2),
                                       (10000, 400, 4), (4725, 300, 2), (125000, 800, 2), (1013, 300, 2),
                                       (9409, 400, 2)])
def test_srdct_apply_matches_oracle(skf, N, s, ncols):
    X = np.random.default_rng(N + s).standard_normal((N, ncols))
    S = skf.Sketch(skf.SRDCT, N, s, 0, 17)
    SX = skf.sketch_apply(S, torch.as_tensor(X, device="cuda")).cpu().numpy()
    SO = OSketch("srdct", N, s, seed=17) @ X
    for c in range(ncols):
        # N-term FP64 sums: about sqrt(N) u of the column's norm
        assert np.linalg.norm(SX[:, c] - SO[:, c]) <= 1e-13 * max(1.0, np.sqrt(N)) * np.linalg.norm(X[:, c])


def test_srdct_arnoldi_and_solve_match_oracle(skf):
    A = convdiff_2d(40, (100.0, 50.0))
    As = csr_to_scipy(A)
    b = gaussian_rhs(A.n, 12)
    m, k, s = 40, 2, 160
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    S = skf.Sketch(skf.SRDCT, A.n, s, 0, 13)
    OS = OSketch("srdct", A.n, s, seed=13)
    bt = torch.as_tensor(b, device="cuda")
    V, vsc, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, bt, m, k)
    ar = arnoldi_trunc(As, b, m, k, OS)
    assert rel(SV.cpu().numpy().T, ar["SV"]) <= 1e-12
    assert rel(SAV.cpu().numpy().T, ar["SAV"]) <= 1e-12
    c = quad_scale("invsqrt", laplacian_lambda_min(40, 2), float(abs(As).sum(1).max()))
    f = skf.make_func("invsqrt", c)
    for method, om in ((skf.SGMRES, "sgmres"), (skf.SFOM, "sfom_quad")):
        info = skf.new_info()
        x = skf.solve(method, op.csr, S, bt, f, skf.make_params(m, k, tol=1e-12), info=info)
        xo, oi = osk.solve(As, b, "invsqrt", m, k, OS, c, method=om, tol=1e-12)
        torch.cuda.synchronize()
        assert skf.read_info(info)["status"] == 0
        assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_srdct_fft_form_arnoldi_3d(skf):
    """The FFT form inside the Arnoldi process at N = 125000 (3D, n = 50):
    S v_j and S A v_j against the oracle's DCT-II sketch, then sGMRES."""
    from workloads import convdiff_3d
    A = convdiff_3d(50, (50.0, 50.0, 50.0))
    As = csr_to_scipy(A)
    b = gaussian_rhs(A.n, 4)
    m, k, s = 24, 2, 96
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    S = skf.Sketch(skf.SRDCT, A.n, s, 0, 29)
    OS = OSketch("srdct", A.n, s, seed=29)
    bt = torch.as_tensor(b, device="cuda")
    V, vsc, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, bt, m, k)
    ar = arnoldi_trunc(As, b, m, k, OS)
    assert rel(SV.cpu().numpy().T, ar["SV"]) <= 1e-12
    assert rel(SAV.cpu().numpy().T, ar["SAV"]) <= 1e-12
    c = quad_scale("invsqrt", laplacian_lambda_min(50, 3), float(abs(As).sum(1).max()))
    f = skf.make_func("invsqrt", c)
    info = skf.new_info()
    x = skf.solve(skf.SGMRES, op.csr, S, bt, f, skf.make_params(m, k, tol=1e-12), info=info)
    xo, oi = osk.solve(As, b, "invsqrt", m, k, OS, c, method="sgmres", tol=1e-12)
    torch.cuda.synchronize()
    assert skf.read_info(info)["status"] == 0
    assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_paper_convection_diffusion_experiment(skf):
    A = upwind_2d(100, 1e-3)
    As = csr_to_scipy(A)
    N = A.n
    b = np.ones(N) / np.sqrt(N)
    lam_hi = float(abs(As).sum(1).max())
    ref = fAb_shifted(As, b, "invsqrt", np.sqrt(0.1 * lam_hi), 300)
    # best approximation from K_m(A, b): orthonormal basis, two passes of CGS
    Q = np.zeros((N, 201))
    Q[:, 0] = b
    for j in range(200):
        w = As @ Q[:, j]
        for _ in range(2):
            w -= Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        Q[:, j + 1] = w / np.linalg.norm(w)
    t_, w_ = oq.rule("invsqrt", 45, 1.0)          # the paper's map: c = 1, 45 nodes
    f = skf.make_func("invsqrt", 1.0, nodes=t_, weights=w_)
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")
    S = skf.Sketch(skf.SRDCT, N, 400, 0, 13)
    bt = torch.as_tensor(b, device="cuda")
    err = lambda x: np.linalg.norm(x - ref) / np.linalg.norm(ref)
    best_40 = None
    for m in (40, 80, 120, 160, 180):
        p = skf.make_params(m, 4)
        xg = skf.solve(skf.SGMRES, op.csr, S, bt, f, p).cpu().numpy()
        xf = skf.solve(skf.SFOM, op.csr, S, bt, f, p).cpu().numpy()
        V, vsc, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, bt, m, 4)
        torch.cuda.synchronize()
        Qm = Q[:, :m]
        e_best = err(Qm @ (Qm.T @ ref))
        best_40 = best_40 or e_best
        # sGMRES follows the best approximation closely (measured ratio <= 1.9)
        assert err(xg) <= 2.5 * e_best
        # sFOM follows it less regularly (measured ratio <= 3.0)
        assert err(xf) <= 4.0 * e_best
        # sFOM by quadrature equals the closed form (sFOM''') on the same
        # sketches up to the 45-node rule's error (about 8e-8 here)
        SVn, SAVn = SV.cpu().numpy().T, SAV.cpu().numpy().T
        vs = vsc.cpu().numpy()
        W = osk.whiten(SVn, SAVn, SVn[:, 0] / vs[0])
        xc = (V.cpu().numpy() * vs[:, None]).T @ osk.sfom_closed(W, "invsqrt")
        assert rel(xf, xc) <= 1e-6
    # superlinear convergence of the best approximation, inherited by sGMRES
    assert e_best <= 1e-2 * best_40 and err(xg) <= 2.5 * e_best
