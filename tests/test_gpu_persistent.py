"""The two forms of the FP64 k-truncated Arnoldi process (Algorithm 2) against
the oracle: the persistent single-launch form (window and A v_j resident in
shared memory, S A V_m from the sketched Arnoldi relation) and the
two-kernel form.  Basis columns, S V_m, S A V_m and H per column; edge cases
(zero right-hand side, m = 1, happy breakdown, tiny N, k = 1 .. 4); the
bounded barrier wait; end-to-end solves in both forms."""
import numpy as np
import pytest
import torch

from oracle import sketched as osk
from oracle.arnoldi import arnoldi_trunc as o_arnoldi
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.configs import laplacian_lambda_min, quad_scale
from workloads.operators import CSR
from gpu_helpers import upload, rel

pytestmark = pytest.mark.gpu

MODES = ["persistent", "two_kernel"]


def mode_id(skf, mode):
    return skf.ARNOLDI_PERSISTENT if mode == "persistent" else skf.ARNOLDI_TWO_KERNEL


def gpu_arnoldi(skf, A, b, m, k, s, mode, zeta=8, seed=13):
    op = upload(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, zeta, seed)
    info = skf.new_info()
    with skf.arnoldi_mode(mode_id(skf, mode)):
        V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, torch.as_tensor(b, device="cuda"), m, k, info=info)
        torch.cuda.synchronize()
    return {"V": (V.double() * vs[:, None]).cpu().numpy().T, "Vraw": V.cpu().numpy().T, "vs": vs.cpu().numpy(),
            "SV": SV.cpu().numpy().T, "SAV": SAV.cpu().numpy().T, "H": H.cpu().numpy().T,
            "info": skf.read_info(info)}


def check_against_oracle(g, ar, m_eff, tol=1e-11):
    assert g["info"]["m_eff"] == m_eff
    for j in range(m_eff):
        assert rel(g["V"][:, j], ar["V"][:, j]) < tol, j
        assert rel(g["SV"][:, j], ar["SV"][:, j]) < tol, j
        assert rel(g["SAV"][:, j], ar["SAV"][:, j]) < tol, j
    Hg, Ho = g["H"][: m_eff + 1, :m_eff], ar["H"]
    # the last column holds only ||w_m||-free slots unless the process broke down there
    nh = m_eff if g["info"]["breakdown"] == 1 else m_eff - 1
    if nh > 0:
        assert np.abs(Hg[:, :nh] - Ho[:, :nh]).max() <= tol * np.abs(Ho).max()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_forms_match_oracle_2d(skf, mode, k):
    A = convdiff_2d(97, (100.0, 50.0))          # N = 9409: a ragged last slice and CTA
    b = gaussian_rhs(A.n, 12)
    m, s = 30, 120
    g = gpu_arnoldi(skf, A, b, m, k, s, mode)
    ar = o_arnoldi(csr_to_scipy(A), b, m, k, OSketch("sparse_sign", A.n, s, 8, 13))
    assert g["info"]["status"] == 0
    check_against_oracle(g, ar, m)
    assert abs(g["info"]["beta"] - np.linalg.norm(b)) < 1e-14


@pytest.mark.parametrize("mode", MODES)
def test_forms_match_oracle_3d_zeta4(skf, mode):
    """3D operator, zeta = 4 (the 16-bit pattern, no compact table)."""
    A = convdiff_3d(21, (50.0, 50.0, 50.0))
    b = gaussian_rhs(A.n, 7)
    m, s = 24, 100
    g = gpu_arnoldi(skf, A, b, m, 2, s, mode, zeta=4)
    ar = o_arnoldi(csr_to_scipy(A), b, m, 2, OSketch("sparse_sign", A.n, s, 4, 13))
    check_against_oracle(g, ar, m)


def test_forms_store_the_same_basis(skf):
    """Both forms perform the same recurrence; their stored bases agree to
    rounding (the dot products are summed in different orders)."""
    A = convdiff_2d(60, (80.0, 20.0))
    b = gaussian_rhs(A.n, 3)
    gp = gpu_arnoldi(skf, A, b, 25, 2, 100, "persistent")
    gt = gpu_arnoldi(skf, A, b, 25, 2, 100, "two_kernel")
    assert rel(gp["V"], gt["V"]) < 1e-12
    assert rel(gp["SV"], gt["SV"]) < 1e-12
    assert rel(gp["SAV"], gt["SAV"]) < 1e-12


@pytest.mark.parametrize("mode", MODES)
def test_edge_cases(skf, mode):
    # zero right-hand side
    A = convdiff_2d(16)
    op = upload(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 20, 4, 1)
    info = skf.new_info()
    with skf.arnoldi_mode(mode_id(skf, mode)):
        skf.arnoldi_trunc(op.csr, S, torch.zeros(A.n, dtype=torch.float64, device="cuda"), 4, 2, info=info)
        torch.cuda.synchronize()
    st = skf.read_info(info)
    assert st["status_name"] == "SKF_ERR_ZERO_RHS" and st["m_eff"] == 0
    # m = 1: one product with A, both sketches of the only column
    b = gaussian_rhs(A.n, 1)
    g = gpu_arnoldi(skf, A, b, 1, 1, 20, mode, zeta=4)
    ar = o_arnoldi(csr_to_scipy(A), b, 1, 1, OSketch("sparse_sign", A.n, 20, 4, 13))
    check_against_oracle(g, ar, 1, tol=1e-13)
    # tiny N: one CTA with a partial slice
    A = convdiff_2d(7)
    b = gaussian_rhs(A.n, 4)
    g = gpu_arnoldi(skf, A, b, 10, 2, 30, mode, zeta=4)
    ar = o_arnoldi(csr_to_scipy(A), b, 10, 2, OSketch("sparse_sign", A.n, 30, 4, 13))
    check_against_oracle(g, ar, 10)


@pytest.mark.parametrize("mode", MODES)
def test_happy_breakdown(skf, mode):
    """A diagonal operator with 5 distinct eigenvalues: the Krylov space is
    invariant after 5 steps; the last column's S A v_j is then sketched
    directly (no further vector exists for the Arnoldi relation)."""
    lam = np.repeat([1.0, 2.0, 3.5, 7.0, 11.0], 300)
    N = lam.size
    A = CSR(N, np.arange(N + 1, dtype=np.int64), np.arange(N, dtype=np.int32), lam)
    b = gaussian_rhs(N, 5)
    g = gpu_arnoldi(skf, A, b, 12, 2, 60, mode)
    ar = o_arnoldi(csr_to_scipy(A), b, 12, 2, OSketch("sparse_sign", N, 60, 8, 13))
    assert ar["m_eff"] == 5 and g["info"]["breakdown"] == 1
    check_against_oracle(g, ar, 5, tol=1e-12)


def test_persistent_form_refuses_what_it_does_not_cover(skf):
    A = convdiff_2d(20)
    op = upload(skf, A)
    b = torch.as_tensor(gaussian_rhs(A.n, 1), device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 40, 8, 13)
    with skf.arnoldi_mode(skf.ARNOLDI_PERSISTENT):
        with pytest.raises(skf.SkfError, match="NOT_SUPPORTED"):
            skf.arnoldi_trunc(op.csr, S, b, 10, 5)                 # k > 4
        Sh = skf.Sketch(skf.SRHT, A.n, 40, 0, 13)
        with pytest.raises(skf.SkfError, match="NOT_SUPPORTED"):
            skf.arnoldi_trunc(op.csr, Sh, b, 10, 2)                # SRHT
    # automatic mode takes the two-kernel form for both
    skf.arnoldi_trunc(op.csr, S, b, 10, 5)
    torch.cuda.synchronize()


def test_barrier_wait_is_bounded(skf):
    """A grid barrier that nothing completes gives up after its budget and
    reports SKF_ERR_TIMEOUT; the context stays usable afterwards."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    for ctas in (1, n_sm):
        assert skf.barrier_selftest(ctas, 2_000_000) == 10     # about 1 ms of SM cycles
    A = convdiff_2d(30)
    g = gpu_arnoldi(skf, A, gaussian_rhs(A.n, 2), 8, 2, 40, "persistent")
    assert g["info"]["status"] == 0


@pytest.mark.parametrize("method", ["sgmres", "sfom"])
def test_solves_in_both_forms_match_oracle(skf, method):
    A = convdiff_2d(100, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    c = quad_scale("invsqrt", laplacian_lambda_min(100, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    m, k, s = 40, 2, 160
    op = upload(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    f = skf.make_func("invsqrt", c)
    p = skf.make_params(m, k, tol=1e-12)
    xo, oi = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                       method="sgmres" if method == "sgmres" else "sfom_quad", tol=1e-12)
    xs = []
    for mode in MODES:
        info = skf.new_info()
        with skf.arnoldi_mode(mode_id(skf, mode)):
            x = skf.solve(skf.SGMRES if method == "sgmres" else skf.SFOM, op.csr, S,
                          torch.as_tensor(b, device="cuda"), f, p, info=info)
            torch.cuda.synchronize()
        st = skf.read_info(info)
        assert st["status"] == 0 and st["ell"] == oi["ell"]
        assert rel(x.cpu().numpy(), xo) <= 1e-10, mode
        xs.append(x.cpu().numpy())
    assert rel(xs[0], xs[1]) <= 1e-11


def test_persistent_form_with_y_in_global_memory(skf):
    """N = 1,404,225 (2D, n = 1185): 9,248 rows per CTA, so the window and A w_j
    no longer fit in the shared memory of a CTA together; the persistent form
    keeps the window on chip and A w_j in global memory (L2).  Per column
    against the oracle and the two-kernel form, and an sGMRES solve."""
    n = 1185
    A = convdiff_2d(n, (100.0, 50.0))
    b = gaussian_rhs(A.n, 5)
    m, k, s = 24, 2, 96
    gp = gpu_arnoldi(skf, A, b, m, k, s, "persistent")      # the persistent form is required here
    gt = gpu_arnoldi(skf, A, b, m, k, s, "two_kernel")
    ar = o_arnoldi(csr_to_scipy(A), b, m, k, OSketch("sparse_sign", A.n, s, 8, 13))
    check_against_oracle(gp, ar, m)
    assert rel(gp["V"], gt["V"]) < 1e-12
    assert rel(gp["SV"], gt["SV"]) < 1e-12 and rel(gp["SAV"], gt["SAV"]) < 1e-12
    c = quad_scale("invsqrt", laplacian_lambda_min(n, 2), float(abs(csr_to_scipy(A)).sum(1).max()))
    op = upload(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, s, 8, 13)
    info = skf.new_info()
    with skf.arnoldi_mode(skf.ARNOLDI_PERSISTENT):
        x = skf.sgmres(op.csr, S, torch.as_tensor(b, device="cuda"), skf.make_func("invsqrt", c),
                       skf.make_params(m, k, tol=1e-12), info=info)
        torch.cuda.synchronize()
    xo, _ = osk.solve(csr_to_scipy(A), b, "invsqrt", m, k, OSketch("sparse_sign", A.n, s, 8, 13), c,
                      method="sgmres", tol=1e-12)
    assert skf.read_info(info)["status"] == 0
    assert rel(x.cpu().numpy(), xo) <= 1e-10
