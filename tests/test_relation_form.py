"""The relation form of the whitened tail (CPU, oracle data only).

With the Arnoldi relation A v_j = sum_{i <= j+1} h_ij v_i (eq. (2.1)) the
sketch of A V_m is S A v_j = S V_m H(1:m, j) for j < m, so the QR of the
s x (m+1) matrix [S V_m, S A v_m] = Q R determines the whitened quantities
of Sec. 3:
  M  = Q_1^T S A V_m R_11^{-1} = [R_11 H(1:m, 1:m-1), R(1:m, m+1)] R_11^{-1},
  (I - Q_1 Q_1^T) S A V_m R_11^{-1} = q_{m+1} gamma e_m^T,
  gamma = R(m+1, m+1) / R(m, m).
The library's FP64 tail evaluates M and the sGMRES residual term this way;
these tests check the identities on the oracle's Arnoldi output against the
oracle's own whitening (QR of S V_m, Z = S A V_m R^{-1}, M = Q^T Z)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import sketched as osk
from oracle.arnoldi import arnoldi_trunc
from oracle.sketch import Sketch as OSketch
from workloads import convdiff_2d, csr_to_scipy, gaussian_rhs


def relation_form(SV, SAV, H, k):
    m = SV.shape[1]
    Q, R = np.linalg.qr(np.column_stack([SV, SAV[:, m - 1]]))
    R11 = R[:m, :m]
    T = np.empty((m, m))
    for a in range(m):
        for j in range(m - 1):
            lo, hi = max(a, j - k + 1), min(j + 1, m - 1)
            T[a, j] = sum(R11[a, i] * H[i, j] for i in range(lo, hi + 1))
        T[a, m - 1] = R[a, m]
    M = sla.solve_triangular(R11, T.T, trans="T", lower=False).T   # M R11 = T
    gamma = R[m, m] / R[m - 1, m - 1]
    return M, gamma, Q


@pytest.mark.parametrize("k", [1, 2, 3])
def test_relation_form_matches_whitening(k):
    A = convdiff_2d(30, (40.0, 20.0))
    b = gaussian_rhs(A.n, 5)
    m, s = 16, 64
    ar = arnoldi_trunc(csr_to_scipy(A), b, m, k, OSketch("sparse_sign", A.n, s, 8, 13))
    W = osk.whiten(ar["SV"], ar["SAV"], OSketch("sparse_sign", A.n, s, 8, 13) @ b)
    M, gamma, Qr = relation_form(ar["SV"], ar["SAV"], ar["H"], k)
    # M is basis-independent up to the sign convention of the QR: compare
    # R-normalised forms (both QRs of S V_m agree up to column signs)
    D = np.sign(np.diag(W["R"])) * np.sign(np.diag(np.linalg.qr(ar["SV"])[1]))
    assert np.allclose(D, 1.0)
    Dr = np.sign(np.diag(np.linalg.qr(np.column_stack([ar["SV"], ar["SAV"][:, -1]]))[1][:m, :m]))
    Dw = np.sign(np.diag(W["R"]))
    Sg = np.diag(Dr * Dw)
    M_w = Sg @ W["M"] @ Sg
    assert np.abs(M - M_w).max() <= 1e-11 * np.abs(M_w).max()
    # the part of Z = S A V_m R^{-1} orthogonal to S V_m is q_{m+1} gamma e_m^T
    Z = W["Z"]
    Zperp = Z - W["Q"] @ (W["Q"].T @ Z)
    assert np.abs(Zperp[:, : m - 1]).max() <= 1e-10 * np.abs(Z).max()
    assert abs(np.linalg.norm(Zperp[:, m - 1]) - abs(gamma)) <= 1e-10 * np.abs(Z).max()


def test_relation_form_sgmres_residual_norms():
    """For every shift t: ||(t Q + Z) y - S b|| = ||[t I + M; gamma e_m^T] y - [c; 0]||."""
    A = convdiff_2d(25, (30.0, 10.0))
    b = gaussian_rhs(A.n, 9)
    m, s, k = 12, 48, 2
    OS = OSketch("sparse_sign", A.n, s, 8, 13)
    ar = arnoldi_trunc(csr_to_scipy(A), b, m, k, OS)
    Sb = OS @ b
    W = osk.whiten(ar["SV"], ar["SAV"], Sb)
    M, gamma, Qr = relation_form(ar["SV"], ar["SAV"], ar["H"], k)
    c = Qr[:, :m].T @ Sb
    rng = np.random.default_rng(3)
    for t in (0.01, 0.3, 2.0, 50.0):
        y = rng.standard_normal(m)
        # y in the oracle's whitened coordinates is Sg y in the relation form's
        Dr = np.sign(np.diag(np.linalg.qr(np.column_stack([ar["SV"], ar["SAV"][:, -1]]))[1][:m, :m]))
        yw = Dr * np.sign(np.diag(W["R"])) * y
        lhs = np.linalg.norm((t * W["Q"] + W["Z"]) @ yw - Sb)
        top = (t * np.eye(m) + M) @ y - c
        rhs = np.sqrt(top @ top + (gamma * y[-1]) ** 2 + (np.linalg.norm(Sb) ** 2 - c @ c))
        assert abs(lhs - rhs) <= 1e-10 * max(lhs, 1.0)


def test_fp32_update_relation_coefficients():
    """Reading 14 for an FP32 basis: an update that applies the FP32 values
    sigma~ = fl32(sigma_j) and c~_i = fl32(h_ij sigma_i),
        w_{j+1} = sigma~ y_j - sum_i c~_i w_i,
    satisfies A v_j = V H(:, j) exactly for the stored columns with
        H(j+1, j) = sigma_j ||w_{j+1}|| / sigma~,  H(i, j) = sigma_j c~_i / (sigma~ sigma_i),
    whereas the unrounded MGS coefficients h_ij leave a residual of order
    2^-24 ||A v_j||.  Checked in FP64 on a short recurrence with FP32-rounded
    coefficients (the stored columns kept in FP64 so that only the
    coefficients differ)."""
    A = csr_to_scipy(convdiff_2d(20, (30.0, 10.0)))
    b = gaussian_rhs(A.shape[0], 4)
    m, k = 12, 2
    W = [b / np.linalg.norm(b)]          # stored columns w_j (here already normalised at j = 0)
    sig = [1.0 / np.linalg.norm(W[0])]
    H_cons = np.zeros((m + 1, m))
    H_mgs = np.zeros((m + 1, m))
    for j in range(m):
        y = A @ W[j]                     # y_j = A w_j
        vj = sig[j] * y                  # A v_j
        i0 = max(0, j - k + 1)
        w = vj.copy()
        h = {}
        for i in range(i0, j + 1):       # MGS against the normalised window
            vi = sig[i] * W[i]
            h[i] = vi @ w
            w = w - h[i] * vi
        st = float(np.float32(sig[j]))
        ct = {i: float(np.float32(h[i] * sig[i])) for i in h}
        wn = st * y - sum(ct[i] * W[i] for i in h)   # the update as applied
        W.append(wn)
        sig.append(1.0 / np.linalg.norm(wn))
        for i in h:
            H_cons[i, j] = sig[j] * ct[i] / (st * sig[i])
            H_mgs[i, j] = h[i]
        H_cons[j + 1, j] = sig[j] * np.linalg.norm(wn) / st
        H_mgs[j + 1, j] = np.linalg.norm(w)     # the unrounded MGS norm
    V = np.column_stack([s_ * w_ for s_, w_ in zip(sig, W)])        # normalised stored basis, m + 1 columns
    AV = A @ V[:, :m]
    r_cons = np.linalg.norm(AV - V @ H_cons) / np.linalg.norm(AV)
    r_mgs = np.linalg.norm(AV - V @ H_mgs) / np.linalg.norm(AV)
    assert r_cons < 1e-14
    assert r_mgs > 1e-9     # the FP32 rounding of the applied coefficients shows
