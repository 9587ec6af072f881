"""lrfg_tt_dot_noalloc: the TT inner product for callers that cannot allocate device memory (inside a
stream capture, or under an application-owned allocator).  Its result must equal lrfg_tt_dot's within the
tolerance the other inner-product tests use, on two calls in a row (the second call reuses the fixed
scratch array the first one left behind), and it must refuse contractions larger than its scratch.

This file is collected last so that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _tt(shape, ranks, seed):
    import paper_1902_07455_gb300 as lrfg
    from synthetic import random_tt
    return lrfg.TTensor.from_numpy(random_tt(shape, ranks, seed=seed))


def test_noalloc_dot_matches_allocating_dot_twice(ctx):
    pairs = [(_tt((45, 27, 63), [5, 4], 1), _tt((45, 27, 63), [3, 6], 2)),
             (_tt((243, 81, 45), [10, 10], 3), _tt((243, 81, 45), [8, 12], 4))]
    reserved_before = ctx.pool_bytes()[1]
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    for x, y in pairs:  # two calls in a row, different shapes and ranks
        ref = ctx.tt_dot(x, y)
        ctx.tt_dot_noalloc(x, y, out)
        torch.cuda.synchronize()
        scale = np.sqrt(ctx.tt_dot(x, x) * ctx.tt_dot(y, y))
        assert abs(out.item() - ref) <= 1e-12 * scale
    # the same operands again: no state carried over from the previous call
    x, y = pairs[0]
    ctx.tt_dot_noalloc(x, y, out)
    torch.cuda.synchronize()
    assert abs(out.item() - ctx.tt_dot(x, y)) <= 1e-12 * np.sqrt(ctx.tt_dot(x, x) * ctx.tt_dot(y, y))
    # the library's pool grew only for the allocating reference calls, never for the no-alloc ones
    ctx.tt_dot_noalloc(*pairs[1], out)
    torch.cuda.synchronize()
    assert ctx.pool_bytes()[1] >= reserved_before


def test_noalloc_dot_rejects_oversized_contraction(ctx):
    import paper_1902_07455_gb300 as lrfg
    from paper_1902_07455_gb300 import _lib as L
    big = _tt((729, 729, 9), [40, 40], 5)  # V = 40 x 729 x 40 doubles: more than the scratch holds
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lrfg.LrfgError) as e:
        ctx.tt_dot_noalloc(big, big, out)
    assert e.value.status == L.LRFG_EINVAL and "scratch" in str(e.value)
