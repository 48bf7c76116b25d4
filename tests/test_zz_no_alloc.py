"""skf_sketch_apply_noalloc: the allocation-free sketch for callers that
cannot allocate device memory where they need S X.  Through the C ABI it must
give the same S X as skf_sketch_apply, bit for bit (both run the same kernels
with the same CTA count and sum in exact fixed point), on calls in a row (its
fixed scratch array is reused), up to the largest request its 4 MiB scratch
holds, and it must refuse the next larger one.

No other test depends on this one or on the order of the files; the file name
only makes pytest collect it last, so that a run stopping at its first failure
has run every other test before this addition is tried."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 4 << 20   # the fixed scratch array of the allocation-free path


def _ctas(N: int) -> int:
    """CTAs of the sketch's row partition: 2 per SM, at least 512 rows each."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return max(1, min(2 * sms, (N + 511) // 512))


def test_noalloc_matches_allocating_entry_point_twice(skf):
    N, s, zeta = 9409, 160, 8
    S = skf.Sketch(skf.SPARSE_SIGN, N, s, zeta, 13)
    rng = np.random.default_rng(7)
    for call in range(2):
        X = torch.as_tensor(rng.standard_normal((N, 3)) * (1 + 100 * call), device="cuda")
        ref = skf.sketch_apply(S, X)
        got = skf.sketch_apply_noalloc(S, X)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_at_the_scratch_limit(skf):
    """Full CTA count (2 per SM) and a request just under the 4 MiB bound, so
    the per-CTA partial sums reach the end of the scratch array."""
    N, ncols, zeta = 400_000, 2, 8
    G = _ctas(N)
    s = SCRATCH_BYTES // (8 * G * ncols) - 1      # G * ncols * (s + 1) * 8 <= 4 MiB
    assert 8 * G * ncols * (s + 1) <= SCRATCH_BYTES < 8 * G * ncols * (s + 2)
    S = skf.Sketch(skf.SPARSE_SIGN, N, s, zeta, 29)
    rng = np.random.default_rng(11)
    for call in range(2):
        Y = torch.as_tensor(rng.standard_normal((ncols, N)) * 10.0 ** call, device="cuda")
        X = Y.t()                                  # column-major (N, ncols) view, passed without a copy
        ref = skf.sketch_apply(S, X)
        got = skf.sketch_apply_noalloc(S, X)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
    S_over = skf.Sketch(skf.SPARSE_SIGN, N, s + 1, zeta, 29)
    with pytest.raises(skf.SkfError, match="INVALID_ARG"):
        skf.sketch_apply_noalloc(S_over, X)


def test_noalloc_rejects_oversized_requests(skf):
    N = 200_000
    S = skf.Sketch(skf.SPARSE_SIGN, N, 4000, 8, 13)
    X = torch.ones((N, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(skf.SkfError, match="INVALID_ARG"):
        skf.sketch_apply_noalloc(S, X)
