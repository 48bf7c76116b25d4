"""skf_sketch_apply_noalloc: the allocation-free sketch for callers that
cannot allocate device memory where they need S X.  Through the C ABI it must
give the same S X as skf_sketch_apply, on two calls in a row (its fixed
scratch array is reused), and it must refuse sizes its scratch cannot hold.
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice(skf):
    N, s, zeta = 9409, 160, 8
    S = skf.Sketch(skf.SPARSE_SIGN, N, s, zeta, 13)
    rng = np.random.default_rng(7)
    for call in range(2):
        X = torch.as_tensor(rng.standard_normal((N, 3)) * (1 + 100 * call), device="cuda")
        ref = skf.sketch_apply(S, X)
        got = skf.sketch_apply_noalloc(S, X)
        torch.cuda.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=1e-14, atol=0)


def test_noalloc_rejects_oversized_requests(skf):
    N = 200_000
    S = skf.Sketch(skf.SPARSE_SIGN, N, 4000, 8, 13)
    X = torch.ones((N, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(skf.SkfError, match="INVALID_ARG"):
        skf.sketch_apply_noalloc(S, X)
