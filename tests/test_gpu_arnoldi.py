"""GPU k-truncated Arnoldi (Algorithm 2) vs the oracle's recurrence: basis,
sketches S V_m and S A V_m, and the banded H; breakdown and edge cases."""
import numpy as np
import pytest
import torch

from oracle.arnoldi import arnoldi_trunc as o_arnoldi
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, convdiff_3d, csr_to_scipy, gaussian_rhs
from workloads.operators import CSR
from gpu_helpers import upload, rel, rhs

pytestmark = pytest.mark.gpu


def run_both(skf, Acsr, b, m, k, s, zeta=8, seed=13, kind="sparse_sign"):
    op = upload(skf, Acsr)
    S = skf.Sketch({"sparse_sign": skf.SPARSE_SIGN, "identity": skf.IDENTITY, "srht": skf.SRHT}[kind], Acsr.n, s,
                   zeta, seed)
    info = skf.new_info()
    bt = torch.as_tensor(b, device="cuda")
    V, vs, SV, SAV, H = skf.arnoldi_trunc(op.csr, S, bt, m, k, info=info)
    torch.cuda.synchronize()
    st = skf.read_info(info)
    ar = o_arnoldi(csr_to_scipy(Acsr), b, m, k, OSketch(kind, Acsr.n, s, zeta, seed))
    g = {"V": (V.double() * vs[:, None]).cpu().numpy().T, "SV": SV.cpu().numpy().T, "SAV": SAV.cpu().numpy().T,
         "H": H.cpu().numpy().T, "info": st}
    return g, ar


@pytest.mark.parametrize("k", [1, 2, 3])
def test_arnoldi_matches_oracle_2d(skf, k):
    A = convdiff_2d(97, (100.0, 50.0))         # N = 9409: ragged last CTA
    b = gaussian_rhs(A.n, 12)
    m, s = 30, 120
    g, ar = run_both(skf, A, b, m, k, s)
    assert g["info"]["m_eff"] == m and g["info"]["status"] == 0
    for j in range(m):
        assert rel(g["V"][:, j], ar["V"][:, j]) < 1e-11, j
    assert rel(g["SV"], ar["SV"]) < 1e-11
    assert rel(g["SAV"], ar["SAV"]) < 1e-11
    Hg, Ho = g["H"][: m + 1, :m], ar["H"]
    assert np.abs(Hg[:, : m - 1] - Ho[:, : m - 1]).max() <= 1e-11 * np.abs(Ho).max()
    assert abs(g["info"]["beta"] - np.linalg.norm(b)) < 1e-14


def test_arnoldi_matches_oracle_3d_full_orthogonalisation(skf):
    A = convdiff_3d(21, (50.0, 50.0, 50.0))    # N = 9261
    b = gaussian_rhs(A.n, 12)
    m = 16
    g, ar = run_both(skf, A, b, m, m, 64)
    assert rel(g["V"], ar["V"]) < 1e-11
    assert rel(g["SAV"], ar["SAV"]) < 1e-11
    Vg = g["V"]
    assert np.abs(Vg.T @ Vg - np.eye(m)).max() < 1e-12


def test_arnoldi_identity_sketch(skf):
    A = convdiff_2d(20)
    b = gaussian_rhs(A.n, 3)
    g, ar = run_both(skf, A, b, 12, 2, A.n, kind="identity")
    np.testing.assert_allclose(g["SV"], g["V"], rtol=0, atol=1e-15)
    assert rel(g["SAV"], ar["SAV"]) < 1e-12


def test_arnoldi_happy_breakdown(skf):
    lam = np.repeat([1.0, 2.0, 3.5, 7.0, 11.0], 300)
    N = lam.size
    A = CSR(N, np.arange(N + 1, dtype=np.int64), np.arange(N, dtype=np.int32), lam)
    b = gaussian_rhs(N, 5)
    g, ar = run_both(skf, A, b, 12, 2, 60)
    assert ar["m_eff"] == 5
    assert g["info"]["m_eff"] == 5 and g["info"]["breakdown"] == 1
    assert rel(g["V"][:, :5], ar["V"]) < 1e-12
    assert rel(g["SAV"][:, :5], ar["SAV"]) < 1e-12


def test_arnoldi_zero_rhs_and_m1(skf):
    A = convdiff_2d(16)
    op = upload(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 20, 4, 1)
    info = skf.new_info()
    skf.arnoldi_trunc(op.csr, S, torch.zeros(A.n, dtype=torch.float64, device="cuda"), 4, 2, info=info)
    torch.cuda.synchronize()
    st = skf.read_info(info)
    assert st["status_name"] == "SKF_ERR_ZERO_RHS" and st["m_eff"] == 0
    b = gaussian_rhs(A.n, 1)
    g, ar = run_both(skf, A, b, 1, 1, 20, zeta=4)
    assert rel(g["SAV"][:, 0], ar["SAV"][:, 0]) < 1e-13
    assert rel(g["SV"][:, 0], ar["SV"][:, 0]) < 1e-13


def test_arnoldi_rejects_bad_arguments(skf):
    A = convdiff_2d(8)
    op = upload(skf, A)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, 10, 2, 1)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(skf.SkfError):
        skf.arnoldi_trunc(op.csr, S, b, 10, 2)         # m >= s
    with pytest.raises(skf.SkfError):
        skf.arnoldi_trunc(op.csr, S, b, 4, 17)         # k > 16


@pytest.mark.parametrize("k", [1, 2])
def test_arnoldi_srht_matches_oracle(skf, k):
    """SRHT sketches of w_j and A w_j, one block-transform launch per step
    (N = 9409, N' = 16384: four 4096-entry blocks)."""
    A = convdiff_2d(97, (100.0, 50.0))
    b = gaussian_rhs(A.n, 12)
    m, s = 30, 120
    g, ar = run_both(skf, A, b, m, k, s, kind="srht")
    assert g["info"]["m_eff"] == m and g["info"]["status"] == 0
    for j in range(m):
        assert rel(g["V"][:, j], ar["V"][:, j]) < 1e-11, j
    assert rel(g["SV"], ar["SV"]) < 1e-11
    assert rel(g["SAV"], ar["SAV"]) < 1e-11
