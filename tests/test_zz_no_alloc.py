"""lrfg_tt_dot_noalloc: the TT inner product for callers that cannot allocate device memory (applications
whose own allocator owns the device memory, loops that must not wait on the driver's allocator).  Its result
must equal lrfg_tt_dot's within the tolerance the other inner-product tests use, on two calls in a row (the
second call reuses the fixed scratch array the first one left behind); it must take nothing from the
context's pool, even for shapes the allocating inner product splits over K; and it must refuse
contractions larger than its scratch.

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
    import paper_1902_07455_gb300 as lrfg
    pairs = [(_tt((45, 27, 63), [5, 4], 1), _tt((45, 27, 63), [3, 6], 2)),
             # the second products contract over c n = 2430 and 972 into 10 x 12 outputs: shapes that the
             # allocating inner product splits over K with a partial-sum workspace from the pool
             (_tt((243, 81, 45), [10, 10], 3), _tt((243, 81, 45), [8, 12], 4))]
    refs = [ctx.tt_dot(x, y) for x, y in pairs]
    scales = [np.sqrt(ctx.tt_dot(x, x) * ctx.tt_dot(y, y)) for x, y in pairs]
    torch.cuda.synchronize()
    # a context of its own, whose pool nothing else touches: the no-alloc calls must leave it empty
    fresh = lrfg.Context(0)
    try:
        before = fresh.pool_bytes()
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        for (x, y), ref, scale in zip(pairs, refs, scales):  # two calls in a row, different shapes and ranks
            fresh.tt_dot_noalloc(x, y, out)
            torch.cuda.synchronize()
            assert abs(out.item() - ref) <= 1e-12 * scale
        # the same operands again: no state carried over from the previous call
        fresh.tt_dot_noalloc(*pairs[0], out)
        torch.cuda.synchronize()
        assert abs(out.item() - refs[0]) <= 1e-12 * scales[0]
        # with profiling switched on, too (no events are recorded, the launches are still counted)
        fresh.profile(True)
        n0 = fresh.launch_count()
        fresh.tt_dot_noalloc(*pairs[1], out)
        torch.cuda.synchronize()
        fresh.profile(False)
        assert fresh.launch_count() > n0
        assert abs(out.item() - refs[1]) <= 1e-12 * scales[1]
        assert fresh.pool_bytes() == before, (fresh.pool_bytes(), before)
    finally:
        fresh.close()


def test_noalloc_dot_rejects_oversized_contraction(ctx):
    import paper_1902_07455_gb300 as lrfg
    from paper_1902_07455_gb300 import _lib as L
    big = _tt((729, 729, 9), [40, 40], 5)  # V = 40 x 729 x 40 doubles: more than the scratch holds
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lrfg.LrfgError) as e:
        ctx.tt_dot_noalloc(big, big, out)
    assert e.value.status == L.LRFG_EINVAL and "scratch" in str(e.value)
