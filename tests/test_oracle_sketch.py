"""Pins for oracle.sketch: generator test vectors, structure of the sparse-sign
map, unbiasedness E||Sx||^2 = ||x||^2 (the expectation behind eq. (1.1)),
Walsh-Hadamard transform against the explicit Hadamard matrix, and
orthogonality of the full SRHT."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import sketch as sk


def test_splitmix64_reference_outputs():
    # First outputs of SplitMix64 from state 0, as produced by the published
    # reference generator (Steele, Lea & Flood, OOPSLA 2014; Vigna's splitmix64.c).
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [int(sk.splitmix_word(0, i)) for i in range(3)]
    assert got == want
    # the scalar and vector mixers agree
    for z in [0, 1, 12345678901234567, (1 << 64) - 1]:
        assert sk.mix64_scalar(z) == int(sk.mix64(np.uint64(z)))


@pytest.mark.parametrize("N,s,zeta", [(1000, 160, 8), (777, 50, 3), (4096, 801, 8), (300, 40, 12)])
def test_sparse_sign_structure(N, s, zeta):
    S = sk.sparse_sign_matrix(N, s, zeta, seed=13).tocsc()
    starts, sizes = sk.stripe_bounds(s, zeta)
    assert sum(sizes) == s
    for c in range(0, N, max(1, N // 97)):
        col = S[:, c]
        rows = np.sort(col.indices)
        assert rows.size == zeta
        np.testing.assert_allclose(np.abs(col.data), 1 / math.sqrt(zeta), rtol=0, atol=1e-16)
        stripe = np.searchsorted(np.array(starts + [s]), rows, side="right") - 1
        assert sorted(stripe.tolist()) == list(range(zeta))


def test_sparse_sign_rows_and_signs_balanced():
    rows, signs = sk.sparse_sign_pattern(200_000, 160, 8, seed=13)
    assert abs(signs.mean()) < 0.01
    counts = np.bincount(rows.ravel(), minlength=160)
    expected = 200_000 * 8 / 160
    # multiply-shift reduction of 15 random bits: per-row bias below size/2^15
    assert np.all(np.abs(counts / expected - 1) < 0.05)


def test_sparse_sign_unbiased_norm():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(500)
    ratios = [np.linalg.norm(sk.sparse_sign_matrix(500, 40, 4, seed) @ x) ** 2 / (x @ x)
              for seed in range(300)]
    mean = np.mean(ratios)
    sem = np.std(ratios) / math.sqrt(len(ratios))
    assert abs(mean - 1) < 4 * sem


def test_sparse_sign_is_subspace_embedding():
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((4000, 10)))
    S = sk.sparse_sign_matrix(4000, 200, 8, seed=13)
    sv = np.linalg.svd(S @ U, compute_uv=False)
    assert sv.max() ** 2 < 1.5 and sv.min() ** 2 > 0.5


@pytest.mark.parametrize("n", [1, 2, 8, 64, 256])
def test_fwht_matches_hadamard(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, 3))
    np.testing.assert_allclose(sk.fwht(x), sla.hadamard(n) @ x, rtol=1e-13, atol=1e-12)


def test_srht_orthogonal_when_full():
    S = sk.Sketch("srht", 64, 64, seed=5).dense()
    np.testing.assert_allclose(S.T @ S, np.eye(64), atol=1e-13)


def test_srht_rows_distinct_and_permutation():
    P = sk.srht_rows(1 << 12, 300, seed=9)
    assert len(set(P.tolist())) == 300 and P.min() >= 0 and P.max() < (1 << 12)
    full = sk.srht_rows(128, 128, seed=9)
    assert sorted(full.tolist()) == list(range(128))


def test_srht_unbiased_norm_and_padding():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100)            # N' = 128, zero padded
    ratios = [np.linalg.norm(sk.Sketch("srht", 100, 32, seed=s) @ x) ** 2 / (x @ x)
              for s in range(300)]
    sem = np.std(ratios) / math.sqrt(len(ratios))
    assert abs(np.mean(ratios) - 1) < 4 * sem
    # S applied to a matrix equals S applied column by column
    X = rng.standard_normal((100, 3))
    S = sk.Sketch("srht", 100, 32, seed=4)
    np.testing.assert_allclose(S @ X, np.column_stack([S @ X[:, i] for i in range(3)]), atol=1e-13)


# ---- SRDCT (Sec. 5.1: S = P F E with a discrete cosine transform)
@pytest.mark.parametrize("N", [1, 7, 12, 33])
def test_srdct_transform_is_the_textbook_dct2(N):
    """s = N, E and P undone: S equals sqrt(N/s) times the orthonormal DCT-II
    written out from its cosine sum."""
    S = sk.Sketch("srdct", N, N, seed=5)
    D = S.dense()
    F = np.empty((N, N))
    for k in range(N):
        a = math.sqrt((1.0 if k == 0 else 2.0) / N)
        for n in range(N):
            F[k, n] = a * math.cos(math.pi * k * (2 * n + 1) / (2 * N))
    expect = (F * S.E[None, :])[S.P]
    np.testing.assert_allclose(D, expect, rtol=0, atol=1e-13)


def test_srdct_orthogonal_when_full():
    S = sk.Sketch("srdct", 40, 40, seed=9)
    D = S.dense()
    np.testing.assert_allclose(D.T @ D, np.eye(40), atol=1e-13)


def test_srdct_unbiased_norm_and_rows():
    N, s = 300, 60
    x = np.random.default_rng(3).standard_normal(N)
    vals = []
    for seed in range(200):
        S = sk.Sketch("srdct", N, s, seed=seed)
        assert len(set(S.P.tolist())) == s and S.P.min() >= 0 and S.P.max() < N
        vals.append(np.sum((S @ x) ** 2))
    assert abs(np.mean(vals) / np.sum(x ** 2) - 1.0) < 0.05
