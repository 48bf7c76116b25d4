"""Subspace embeddings S in R^{s x N} (Sec. 1, eq. (1.1)).

Sparse-sign map (not in the paper; the reading used by this library): column
c of S has zeta nonzeros +-1/sqrt(zeta).  The s rows are cut into zeta
stripes, stripe q covering rows [floor(q s/zeta), floor((q+1) s/zeta)); column
c has exactly one nonzero in each stripe.  The random bits come from the
counter-based SplitMix64 generator:

    word(seed, i) = mix64(seed + (i + 1) * 0x9E3779B97F4A7C15)  (mod 2^64)
    mix64(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
              z *= 0x94D049BB133111EB; z ^= z >> 31

Column c uses words i = c*W + w, w = 0..W-1, W = ceil(zeta/4); stripe q takes
the 16-bit chunk u = (word_{q div 4} >> 16*(q mod 4)) & 0xFFFF: the sign is
negative iff bit 0 of u is set, and the row inside the stripe is
((u >> 1) * size_q) >> 15.

SRHT (Sec. 2.2 names subsampled randomized Fourier/DCT transforms; Sec. 5.1
uses S = P F E): S x = (1/sqrt(s)) * (H E [x; 0])[P] with N' = 2^ceil(log2 N),
H the Sylvester-Hadamard matrix of order N' (entries (-1)^popcount(i&j)), E
the diagonal of signs (-1 iff bit 0 of word(seed, c) is set) and P the first
s entries of a partial Fisher-Yates shuffle of [0, N') driven by
word(mix64(seed), i): position i swaps with i + (word mod (N' - i)).
The scale makes S orthogonal when s = N' = N.

SRDCT (the sketch of the paper's experiments, Sec. 5.1: S = P F E with F a
discrete cosine transform): S x = sqrt(N/s) * (F E x)[P], F the orthonormal
DCT-II of order N, (F y)_k = a_k sum_n y_n cos(pi k (2n + 1) / (2N)) with
a_0 = sqrt(1/N), a_k = sqrt(2/N); E as for the SRHT, and P the first s entries
of the same partial Fisher-Yates shuffle, of [0, N) (no padding).  The scale
makes S orthogonal when s = N.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * M1
        z = z ^ (z >> np.uint64(27))
        z = z * M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix_word(seed: int, index) -> np.ndarray:
    """The index-th output of SplitMix64 started from state ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * GAMMA
    return mix64(state)


def mix64_scalar(z: int) -> int:
    z &= MASK64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & MASK64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & MASK64
    z ^= z >> 31
    return z


def stripe_bounds(s: int, zeta: int):
    starts = [(q * s) // zeta for q in range(zeta + 1)]
    return starts[:-1], [starts[q + 1] - starts[q] for q in range(zeta)]


def sparse_sign_pattern(N: int, s: int, zeta: int, seed: int):
    """Rows (zeta, N) int64 and signs (zeta, N) float64 of the nonzeros."""
    if not (1 <= zeta <= s) or s // zeta > 32768:
        raise ValueError("need 1 <= zeta <= s and s/zeta <= 32768")
    W = (zeta + 3) // 4
    cols = np.arange(N, dtype=np.uint64)
    starts, sizes = stripe_bounds(s, zeta)
    rows = np.empty((zeta, N), dtype=np.int64)
    signs = np.empty((zeta, N), dtype=np.float64)
    words = [splitmix_word(seed, cols * np.uint64(W) + np.uint64(w)) for w in range(W)]
    for q in range(zeta):
        u = (words[q // 4] >> np.uint64(16 * (q % 4))) & np.uint64(0xFFFF)
        signs[q] = np.where((u & np.uint64(1)) == 0, 1.0, -1.0)
        r = ((u >> np.uint64(1)) * np.uint64(sizes[q])) >> np.uint64(15)
        rows[q] = starts[q] + r.astype(np.int64)
    return rows, signs


def sparse_sign_matrix(N: int, s: int, zeta: int, seed: int) -> sp.csr_matrix:
    rows, signs = sparse_sign_pattern(N, s, zeta, seed)
    cols = np.broadcast_to(np.arange(N), rows.shape)
    vals = signs / math.sqrt(zeta)
    return sp.csr_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(s, N))


def srht_signs(N: int, seed: int) -> np.ndarray:
    w = splitmix_word(seed, np.arange(N, dtype=np.uint64))
    return np.where((w & np.uint64(1)) == 0, 1.0, -1.0)


def srht_rows(Np: int, s: int, seed: int) -> np.ndarray:
    """First s entries of a partial Fisher-Yates shuffle of range(Np)."""
    if s > Np:
        raise ValueError("s > N'")
    seed2 = mix64_scalar(seed)
    swapped: dict[int, int] = {}
    out = np.empty(s, dtype=np.int64)
    for i in range(s):
        word = int(splitmix_word(seed2, i))
        j = i + word % (Np - i)
        vi = swapped.get(i, i)
        vj = swapped.get(j, j)
        swapped[i], swapped[j] = vj, vi
        out[i] = vj
    return out


def fwht(x: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform H x (Sylvester order) along axis 0
    by the textbook butterfly; length must be a power of two."""
    y = np.array(x, dtype=np.float64, copy=True)
    n = y.shape[0]
    h = 1
    while h < n:
        y = y.reshape((n // (2 * h), 2, h) + y.shape[1:])
        a = y[:, 0].copy()
        b = y[:, 1].copy()
        y[:, 0] = a + b
        y[:, 1] = a - b
        y = y.reshape((n,) + y.shape[3:])
        h *= 2
    return y


class Sketch:
    """S as an operator: ``S @ X`` for X of shape (N,) or (N, ncols)."""

    def __init__(self, kind: str, N: int, s: int, zeta: int = 8, seed: int = 13):
        self.kind, self.N, self.s, self.zeta, self.seed = kind, N, s, zeta, seed
        if kind == "sparse_sign":
            self.mat = sparse_sign_matrix(N, s, zeta, seed)
        elif kind == "srht":
            self.Np = 1 << max(0, math.ceil(math.log2(N)))
            self.E = srht_signs(N, seed)
            self.P = srht_rows(self.Np, s, seed)
        elif kind == "srdct":
            self.E = srht_signs(N, seed)
            self.P = srht_rows(N, s, seed)
        elif kind == "identity":
            if s != N:
                raise ValueError("identity sketch needs s == N")
        else:
            raise ValueError(kind)

    def __matmul__(self, X):
        X = np.asarray(X, dtype=np.float64)
        if self.kind == "sparse_sign":
            return self.mat @ X
        if self.kind == "identity":
            return X.copy()
        if self.kind == "srdct":
            import scipy.fft
            y = self.E.reshape((-1,) + (1,) * (X.ndim - 1)) * X
            return scipy.fft.dct(y, type=2, norm="ortho", axis=0)[self.P] * math.sqrt(self.N / self.s)
        z = np.zeros((self.Np,) + X.shape[1:])
        z[: self.N] = (self.E.reshape((-1,) + (1,) * (X.ndim - 1)) * X)
        return fwht(z)[self.P] / math.sqrt(self.s)

    def dense(self) -> np.ndarray:
        return self @ np.eye(self.N)
