"""GPU sketch vs the oracle's S (eq. (1.1)): the sparse-sign pattern is
bit-exact column by column, S X agrees to FP64 rounding, and repeated calls
are bitwise identical (integer accumulation)."""
import math

import numpy as np
import pytest
import torch

from oracle.sketch import Sketch as OSketch, sparse_sign_matrix

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,s,zeta,seed", [(5000, 160, 8, 13), (9409, 800, 8, 13), (777, 50, 3, 99),
                                           (3000, 37, 16, 7)])
def test_sparse_sign_columns_bit_exact(skf, N, s, zeta, seed):
    S = skf.Sketch(skf.SPARSE_SIGN, N, s, zeta, seed)
    cols = np.unique(np.concatenate([np.arange(0, N, max(1, N // 40)), [N - 1]]))
    E = torch.zeros((N, cols.size), dtype=torch.float64, device="cuda")
    E[torch.as_tensor(cols, device="cuda"), torch.arange(cols.size, device="cuda")] = 1.0
    got = skf.sketch_apply(S, E).cpu().numpy()
    want = sparse_sign_matrix(N, s, zeta, seed)[:, cols].toarray()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("N,s,zeta", [(9409, 160, 8), (100_003, 800, 8), (50, 40, 4)])
def test_sketch_apply_matches_oracle(skf, N, s, zeta):
    rng = np.random.default_rng(N)
    X = rng.standard_normal((N, 3))
    X[:, 1] *= np.exp(rng.uniform(-20, 20, N))      # wide dynamic range
    X[:, 2] = 0.0
    X[N // 2, 2] = 1e-300
    S = skf.Sketch(skf.SPARSE_SIGN, N, s, zeta, 13)
    got = skf.sketch_apply(S, torch.as_tensor(X, device="cuda")).cpu().numpy()
    want = OSketch("sparse_sign", N, s, zeta, 13) @ X
    for c in range(2):
        assert np.linalg.norm(got[:, c] - want[:, c]) <= 1e-14 * np.linalg.norm(want[:, c])
    np.testing.assert_allclose(got[:, 2], want[:, 2], rtol=1e-13, atol=0)


def test_sketch_deterministic_and_identity(skf):
    N = 20_000
    X = torch.randn(N, 2, dtype=torch.float64, device="cuda")
    S = skf.Sketch(skf.SPARSE_SIGN, N, 300, 8, 1)
    a = skf.sketch_apply(S, X)
    b = skf.sketch_apply(S, X)
    assert torch.equal(a, b)
    I = skf.Sketch(skf.IDENTITY, N, N, 1, 0)
    assert torch.equal(skf.sketch_apply(I, X), X)


# ---------------------------------------------------------------- SRHT
# S x = s^-1/2 (H_{N'} E [x; 0])[P]: computed exactly in int64 on the GPU, in
# FP64 butterflies by the oracle, so they agree to the oracle's rounding
# (about log2(N') unit roundoffs of the output's scale).

@pytest.mark.parametrize("N,s,seed", [(1000, 64, 13), (5000, 160, 13), (100_003, 800, 7)])
def test_srht_unit_columns(skf, N, s, seed):
    """S e_c = +-1/sqrt(s) on the sampled rows: sign and row pattern exact."""
    S = skf.Sketch(skf.SRHT, N, s, 0, seed)
    cols = np.unique(np.concatenate([np.arange(0, N, max(1, N // 30)), [N - 1]]))
    E = torch.zeros((N, cols.size), dtype=torch.float64, device="cuda")
    E[torch.as_tensor(cols, device="cuda"), torch.arange(cols.size, device="cuda")] = 1.0
    got = skf.sketch_apply(S, E).cpu().numpy()
    want = OSketch("srht", N, s, 0, seed) @ np.eye(N)[:, cols]
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)
    assert np.array_equal(np.sign(got), np.sign(want))


@pytest.mark.parametrize("N,s", [(1000, 64), (5000, 160), (100_003, 800)])
def test_srht_apply_matches_oracle(skf, N, s):
    rng = np.random.default_rng(N + 1)
    X = rng.standard_normal((N, 3))
    X[:, 1] *= np.exp(rng.uniform(-20, 20, N))      # wide dynamic range
    X[:, 2] = 0.0
    S = skf.Sketch(skf.SRHT, N, s, 0, 13)
    Xt = torch.as_tensor(X, device="cuda")
    got = skf.sketch_apply(S, Xt).cpu().numpy()
    again = skf.sketch_apply(S, Xt).cpu().numpy()
    want = OSketch("srht", N, s, 0, 13) @ X
    for c in range(2):
        assert np.linalg.norm(got[:, c] - want[:, c]) <= 1e-12 * np.linalg.norm(want[:, c])
    assert np.all(got[:, 2] == 0.0)
    assert np.array_equal(got, again)   # integer accumulation: bitwise repeatable


def test_srht_full_is_orthogonal(skf):
    """s = N = N' = 4096: S = H E / sqrt(N) with rows permuted is orthogonal."""
    N = 4096
    S = skf.Sketch(skf.SRHT, N, N, 0, 3)
    D = skf.sketch_apply(S, torch.eye(N, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.abs(D.T @ D - N / N * np.eye(N)).max() < 1e-12


def test_srht_rejects_s_above_padded_length(skf):
    with pytest.raises(skf.SkfError):
        skf.Sketch(skf.SRHT, 100, 200, 0, 1)
