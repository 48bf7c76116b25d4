"""Host-side parts of the batched solves: the seeded layout of the batched
workload follows its stated recipe, and skf_solve_batched validates its
arguments (and every problem's) before any device work."""
import ctypes
import os

import pytest

from workloads.batch import batch_layout


def test_layout_matches_its_definition():
    L = batch_layout()
    assert len(L.mats) == 8 and len(L.rhs) == 64
    counts = L.summary()["rhs_per_mat"]
    assert min(counts) >= 1 and sum(counts) == 64
    for i, M in enumerate(L.mats):
        assert M.dims == (2 if i % 2 == 0 else 3)
        assert 0.8e5 <= M.N <= 4.4e6
        assert all(10.0 <= v <= 200.0 for v in M.nu)
        # centred differences stay positive real: cell Peclet number below 1
        assert max(M.nu) / (2.0 * (M.n + 1)) < 1.0
    for r in L.rhs:
        assert 50 <= r.m <= 400 and r.s == 4 * r.m
    assert len({r.sketch_seed for r in L.rhs}) == 64
    assert batch_layout().summary() == L.summary()     # seeded


@pytest.fixture(scope="module")
def skf():
    import paper_2208_11447_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2208_11447_gb300 import build
        build.build()
    pkg.lib()
    return pkg


def test_batched_argument_validation(skf):
    L = skf.lib()
    assert L.skf_solve_batched(0, None, 4, None) == 0
    assert L.skf_solve_batched(-1, None, 4, None) == 1
    arr = (skf.Problem * 2)()
    assert L.skf_solve_batched(2, arr, 0, None) == 1
    assert L.skf_solve_batched(2, arr, 17, None) == 1
    f = skf.make_func("invsqrt", 1.0)
    p = skf.make_params(10, 2)
    for q in arr:
        q.f = ctypes.pointer(f)
        q.p = ctypes.pointer(p)
        q.x = 16          # never dereferenced: validation fails first
    assert L.skf_solve_batched(2, arr, 2, None) == 1   # NULL operator
    assert L.skf_last_error().startswith(b"problem 0:")
