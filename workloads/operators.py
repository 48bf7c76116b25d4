"""Sparse test operators (CSR, int64 row pointer, int32 column index).

* ``convdiff_2d`` / ``convdiff_3d``: centred finite differences for
  ``-Laplace(u) + nu . grad(u)`` on the unit square/cube with Dirichlet
  boundary, ``h = 1/(n+1)``, lexicographic ordering with x fastest.  With
  ``L = tridiag(-1, 2, -1)`` and ``C = tridiag(-1, 0, 1)`` the 2D operator is
  ``(1/h^2)(I(x)L + L(x)I) + nu_x/(2h) I(x)C + nu_y/(2h) C(x)I`` and the 3D one
  is its 7-point analogue.  Its symmetric part is the Laplacian, so the matrix
  is positive real (the setting of the paper's convergence theorem, Sec. 3.1).
* ``upwind_2d``: the first-order upwind convection-diffusion matrix of the
  paper's first experiment (Sec. 5.1), ``D/h^2 (I(x)L + L(x)I) + (1/h)(C (+) C^T)``
  with ``C = tridiag(-1, 1, 0)``.
* ``powerlaw_graph_operator``: ``A = D_s + 0.1 I - W^T`` for a seeded directed
  graph ``W`` with Zipf out-degrees; this equals ``L + 0.1 I + (W - W^T)/2``
  where ``L`` is the Laplacian of the symmetrised graph ``(W + W^T)/2``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray   # int64, n+1
    colind: np.ndarray   # int32, nnz
    values: np.ndarray   # float64 or float32, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.rowptr, self.colind, self.values.astype(dtype))


def _assemble(n_rows: int, cols: np.ndarray, vals: np.ndarray, valid: np.ndarray) -> CSR:
    """Compress a dense (n_rows, width) candidate table into CSR, keeping the
    candidates in their given (ascending column) order."""
    counts = valid.sum(axis=1).astype(np.int64)
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[valid].astype(np.int32)
    values = vals[valid]
    return CSR(n_rows, rowptr, colind, values)


def _stencil(n: int, dims: int, diag: float, offdiag: list[tuple[float, float]]) -> CSR:
    """Generic (2*dims+1)-point stencil on an n^dims grid, x fastest.

    ``offdiag[d] = (coef_minus, coef_plus)`` is the coupling to the neighbour at
    index -1 / +1 along dimension d (d=0 is x)."""
    N = n ** dims
    idx = np.arange(N, dtype=np.int64)
    coords = [(idx // (n ** d)) % n for d in range(dims)]
    width = 2 * dims + 1
    cols = np.empty((N, width), dtype=np.int64)
    vals = np.empty((N, width), dtype=np.float64)
    valid = np.empty((N, width), dtype=bool)
    # ascending column order: -n^(d) for d = dims-1..0, then 0, then +n^d for d = 0..dims-1
    slot = 0
    for d in reversed(range(dims)):
        stride = n ** d
        cols[:, slot] = idx - stride
        vals[:, slot] = offdiag[d][0]
        valid[:, slot] = coords[d] > 0
        slot += 1
    cols[:, slot] = idx
    vals[:, slot] = diag
    valid[:, slot] = True
    slot += 1
    for d in range(dims):
        stride = n ** d
        cols[:, slot] = idx + stride
        vals[:, slot] = offdiag[d][1]
        valid[:, slot] = coords[d] < n - 1
        slot += 1
    return _assemble(N, cols, vals, valid)


def convdiff_2d(n: int, nu=(100.0, 50.0)) -> CSR:
    h = 1.0 / (n + 1)
    ih2 = 1.0 / (h * h)
    off = [(-ih2 - nu[d] / (2 * h), -ih2 + nu[d] / (2 * h)) for d in range(2)]
    return _stencil(n, 2, 4.0 * ih2, off)


def convdiff_3d(n: int, nu=(50.0, 50.0, 50.0)) -> CSR:
    h = 1.0 / (n + 1)
    ih2 = 1.0 / (h * h)
    off = [(-ih2 - nu[d] / (2 * h), -ih2 + nu[d] / (2 * h)) for d in range(3)]
    return _stencil(n, 3, 6.0 * ih2, off)


def upwind_2d(n: int, D: float = 1e-3) -> CSR:
    """Paper Sec. 5.1 operator: D/h^2 (I(x)L + L(x)I) + (1/h) (C (+) C^T),
    C = tridiag(-1, 1, 0) (lower -1, diagonal 1).  C (+) C^T = I(x)C + C^T(x)I:
    the x-direction couples to x-1 with -1, the y-direction to y+1 with -1."""
    h = 1.0 / (n + 1)
    a = D / (h * h)
    ih = 1.0 / h
    # Kronecker sum C (+) C^T = C(x)I + I(x)C^T: with x fastest, I(x)C^T acts
    # along x (coupling -1/h to x+1) and C(x)I along y (coupling -1/h to y-1).
    diag = 4.0 * a + 2.0 * ih
    off = [(-a, -a - ih),            # x: C^T has -1 on the super-diagonal
           (-a - ih, -a)]            # y: C has -1 on the sub-diagonal
    return _stencil(n, 2, diag, off)


def ninepoint_2d(n: int, nu=(100.0, 50.0), drop_corner: bool = False) -> CSR:
    """-Delta u + nu . grad u on an n x n grid with the compact nine-point
    (Mehrstellen) Laplacian (diagonal 20, edges -4, corners -1, over 6 h^2)
    and centred first differences.  Its symmetric part is the nine-point
    Laplacian (positive definite), so the operator is positive real.  With
    ``drop_corner`` the (+1, +1) corner coupling is left out (eight entries
    per interior row); its symmetric part keeps the diagonal 20 against
    off-diagonal magnitudes 16 + 2 + 1 = 19 (over 6 h^2), so it is strictly
    diagonally dominant and the operator stays positive real."""
    h = 1.0 / (n + 1)
    N = n * n
    idx = np.arange(N, dtype=np.int64)
    x, y = idx % n, idx // n
    e, c0 = -4.0 / (6 * h * h), -1.0 / (6 * h * h)
    cx, cy = nu[0] / (2 * h), nu[1] / (2 * h)
    offs = [(-1, -1, c0), (0, -1, e - cy), (1, -1, c0), (-1, 0, e - cx), (0, 0, 20.0 / (6 * h * h)),
            (1, 0, e + cx), (-1, 1, c0), (0, 1, e + cy)]
    if not drop_corner:
        offs.append((1, 1, c0))
    width = len(offs)
    cols = np.empty((N, width), dtype=np.int64)
    vals = np.empty((N, width), dtype=np.float64)
    valid = np.empty((N, width), dtype=bool)
    for slot, (dx, dy, v) in enumerate(offs):       # ascending column order
        cols[:, slot] = idx + dx + n * dy
        vals[:, slot] = v
        valid[:, slot] = (x + dx >= 0) & (x + dx < n) & (y + dy >= 0) & (y + dy < n)
    return _assemble(N, cols, vals, valid)


def powerlaw_graph_operator(N: int, alpha: float = 2.1, mean_degree: float = 10.0,
                            seed: int = 11, d_max: int = 100_000,
                            transpose: bool = False) -> CSR:
    """``A = D_s + 0.1 I - W^T`` (rows carry in-degrees) or, with
    ``transpose=True``, ``D_s + 0.1 I - W`` (rows carry the power-law
    out-degrees).  Out-degrees are Zipf(alpha) truncated at ``d_max`` and
    rescaled to the requested mean (minimum 1); targets are uniform without
    self-loops; duplicate edges are dropped; weights are 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.zipf(alpha, size=N).astype(np.float64)
    z = np.minimum(z, d_max)
    deg = np.maximum(1, np.rint(z * (mean_degree / z.mean()))).astype(np.int64)
    deg = np.minimum(deg, N - 1)
    src = np.repeat(np.arange(N, dtype=np.int64), deg)
    dst = rng.integers(0, N - 1, size=src.size, dtype=np.int64)
    dst = dst + (dst >= src)                       # skip the self-loop
    key = np.sort(src * N + dst)                   # drop duplicates (sorted distinct keys)
    key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    src = key // N
    dst = key % N
    out_deg = np.bincount(src, minlength=N).astype(np.float64)
    in_deg = np.bincount(dst, minlength=N).astype(np.float64)
    diag = 0.5 * (out_deg + in_deg) + 0.1
    if transpose:
        rows, cols = src, dst      # row i holds -W[i, j]
    else:
        rows, cols = dst, src      # row i holds -W^T[i, j] = -W[j, i]
    # entries in (row, column) order: one sort of the distinct keys row N + col;
    # the diagonal entries carry diag, the edges -1
    diag_i = np.arange(N, dtype=np.int64)
    keys = np.sort(np.concatenate([rows * N + cols, diag_i * N + diag_i]))
    rows, cols = keys // N, keys % N
    vals = np.where(rows == cols, diag[rows], -1.0)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=N), out=rowptr[1:])
    return CSR(N, rowptr, cols.astype(np.int32), vals)


def gaussian_rhs(N: int, seed: int = 12, normalize: bool = True) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.standard_normal(N)
    if normalize:
        b /= np.linalg.norm(b)
    return b


def csr_to_scipy(A: CSR):
    import scipy.sparse as sp
    return sp.csr_matrix((A.values, A.colind, A.rowptr), shape=(A.n, A.n))
