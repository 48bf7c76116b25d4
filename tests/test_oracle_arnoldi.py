"""Pins for oracle.arnoldi (Algorithm 2's truncated MGS recurrence):
full orthogonalisation reproduces the QR factor of the Krylov matrix; the
truncated basis satisfies the banded Arnoldi relation (eq. (2.1)) and local
orthogonality; the stored sketches are S applied to the stored vectors;
happy breakdown stops at the dimension of an invariant Krylov space."""
import numpy as np
import pytest

from oracle.arnoldi import arnoldi_trunc
from oracle.sketch import Sketch
from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs


def small_problem(n=12):
    A = csr_to_scipy(convdiff_2d(n, (30.0, 10.0)))
    b = gaussian_rhs(A.shape[0], 12)
    return A, b


def test_full_orthogonalisation_is_krylov_qr():
    A, b = small_problem()
    m = 8
    ar = arnoldi_trunc(A, b, m, k=m, S=Sketch("identity", A.shape[0], A.shape[0]))
    K = np.empty((A.shape[0], m))
    K[:, 0] = b
    for j in range(1, m):
        K[:, j] = A @ K[:, j - 1]
    Qk, Rk = np.linalg.qr(K)
    Qk = Qk * np.sign(np.diag(Rk))[None, :]
    np.testing.assert_allclose(ar["V"], Qk, atol=1e-9)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_truncated_arnoldi_relation_and_local_orthogonality(k):
    A, b = small_problem()
    m = 20
    S = Sketch("sparse_sign", A.shape[0], 60, 4, seed=13)
    ar = arnoldi_trunc(A, b, m, k, S)
    V, H = ar["V"], ar["H"]
    # A V_{m-1} = V_m H_{1:m, 1:m-1}: the last column has no orthogonalisation
    res = A @ V[:, : m - 1] - V @ H[:m, : m - 1]
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(A.toarray(), 2)
    np.testing.assert_allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-14)
    G = V.T @ V
    for i in range(m):
        for j in range(max(0, i - k), i):
            assert abs(G[i, j]) < 1e-13
    # H is banded: zero above the k-th superdiagonal, zero below the subdiagonal
    for j in range(m):
        for i in range(m + 1):
            if i < j - k + 1 or i > j + 1:
                assert H[i, j] == 0.0


def test_sketches_are_of_stored_vectors():
    A, b = small_problem()
    S = Sketch("sparse_sign", A.shape[0], 48, 8, seed=3)
    ar = arnoldi_trunc(A, b, 15, 2, S)
    np.testing.assert_allclose(ar["SV"], S @ ar["V"], atol=1e-14)
    np.testing.assert_allclose(ar["SAV"], S @ (A @ ar["V"]), atol=1e-9)
    assert ar["SV"].shape == (48, 15) and ar["SAV"].shape == (48, 15)


def test_happy_breakdown_at_invariant_dimension():
    lam = np.repeat([1.0, 2.0, 3.5, 7.0, 11.0], 8)
    A = np.diag(lam)
    b = np.random.default_rng(0).standard_normal(lam.size)
    ar = arnoldi_trunc(A, b, 12, 2, Sketch("identity", lam.size, lam.size))
    assert ar["m_eff"] == 5
    assert ar["V"].shape == (40, 5)


def test_zero_rhs_rejected():
    A, _ = small_problem(4)
    with pytest.raises(ValueError):
        arnoldi_trunc(A, np.zeros(16), 3, 2, Sketch("identity", 16, 16))
