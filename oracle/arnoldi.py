"""k-truncated Arnoldi with on-the-fly sketching (Algorithm 2 and Sec. 2.2).

Steps, in the paper's order:
  v_1 = b / ||b||;   w = A v_1;   sketch S v_1 and S w.
  for j = 1..m-1:
      for i = max(1, j-k+1) .. j (ascending):   h_ij = <v_i, w>;  w -= h_ij v_i
      h_{j+1,j} = ||w||;   v_{j+1} = w / h_{j+1,j}
      w = A v_{j+1};   sketch S v_{j+1} and S w.
Only m matrix-vector products are performed: Algorithm 2 as printed iterates
j = 1..m and therefore also forms v_{m+1} and A v_{m+1}, which are not part
of V_m, S V_m or S A V_m; this oracle stops after A v_m.

Happy breakdown (the paper states no criterion; this is the reading used):
if h_{j+1,j} <= 1e-12 * ||A v_j|| the Krylov space is invariant to rounding;
the recurrence stops with m_eff = j columns.  At an exactly invariant
dimension the computed ratio is at the rounding level of the k-term MGS
(about 1e-14 for N ~ 1e3), so the threshold sits two orders above it.
"""
from __future__ import annotations

import numpy as np


def arnoldi_trunc(A, b, m: int, k: int, S, breakdown_tol: float = 1e-12):
    """Returns dict with V (N x m_eff), SV, SAV (s x m_eff), H ((m_eff+1) x m_eff,
    dense, zero outside the band), beta = ||b|| and m_eff.  A is any object with
    ``A @ x``; S is an ``oracle.sketch.Sketch`` (or anything with ``S @ x``)."""
    b = np.asarray(b, dtype=np.float64)
    N = b.shape[0]
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        raise ValueError("b = 0")
    V = np.zeros((N, m))
    H = np.zeros((m + 1, m))
    V[:, 0] = b / beta
    SV_cols, SAV_cols = [S @ V[:, 0]], []
    m_eff = m
    for j in range(m):
        w = A @ V[:, j]
        SAV_cols.append(S @ w)
        if j == m - 1:
            break
        norm_y = float(np.linalg.norm(w))
        for i in range(max(0, j - k + 1), j + 1):
            H[i, j] = float(V[:, i] @ w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = float(np.linalg.norm(w))
        if H[j + 1, j] <= breakdown_tol * norm_y:
            m_eff = j + 1
            break
        V[:, j + 1] = w / H[j + 1, j]
        SV_cols.append(S @ V[:, j + 1])
    SV = np.column_stack(SV_cols[:m_eff])
    SAV = np.column_stack(SAV_cols[:m_eff])
    return {"V": V[:, :m_eff], "SV": SV, "SAV": SAV, "H": H[: m_eff + 1, :m_eff],
            "beta": beta, "m_eff": m_eff}
