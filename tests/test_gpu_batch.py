"""Batch / serving executor (lrfg_batch_*): solves of different d, N, format and rank run concurrently on
worker streams and each result equals the same solve run alone on one context.

"The same" is bitwise: no kernel of the library accumulates with atomics (split-K products sum their
partials in a fixed order) and the launch shapes depend only on the problem and the device, so a solve
gives identical A_eff, residual and iteration count whatever runs beside it.  Against the FP64 oracle
the executor's results meet the FP64-path tolerance (1e-6 relative on A_eff)."""
import time

import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import fourier_galerkin as fg
from oracle import lowrank as lr
from synthetic import lognormal_grf, smoothed_cube, square_inclusion

pytestmark = pytest.mark.gpu


def _requests():
    """(coeff, E, fmt, kwargs) mixing d, N, coefficient format, solution format and rank."""
    reqs = []
    a2, _, _ = square_inclusion(2, 63)
    reqs.append((a2, [1.0, 0.0], lrfg.FULL, dict(tol=1e-8)))
    g3 = lognormal_grf(3, 45, seed=11)
    reqs.append((g3, [1.0, 0.0, 0.0], lrfg.FULL, dict(tol=1e-8)))
    _, t3, w3 = smoothed_cube(3, 45, contrast=10.0, full=False)
    reqs.append((lr.tt_from_separable(t3, w3), [1.0, 0.0, 0.0], lrfg.TT, dict(rank=5, maxit=30)))
    reqs.append((g3, [0.0, 1.0, 0.0], lrfg.TT, dict(rank=8, maxit=30)))
    _, t81, w81 = smoothed_cube(3, 81, contrast=20.0, full=False)
    reqs.append((lr.tt_from_separable(t81, w81), [1.0, 0.0, 0.0], lrfg.TT, dict(rank=10, maxit=25)))
    reqs.append((lr.tucker_from_separable(t3, w3), [1.0, 0.0, 0.0], lrfg.TUCKER, dict(rank=4, maxit=30)))
    _, t2, w2 = smoothed_cube(2, 63, contrast=10.0, full=False)
    reqs.append((lr.tt_from_separable(t2, w2), [1.0, 0.0], lrfg.TT, dict(rank=6, maxit=30)))
    return reqs


def _solo(ctx, coeff, E, fmt, kw):
    if isinstance(coeff, tuple):
        c = lrfg.TuckerTensor.from_numpy(*coeff)
    elif isinstance(coeff, list):
        c = lrfg.TTensor.from_numpy(coeff)
    else:
        c = coeff
    p = ctx.problem(c, fmt, **kw)
    res, _ = p.solve(E, want_field=False)
    p.free()
    return res


def test_batch_results_equal_solo(ctx):
    reqs = _requests()
    solo = [_solo(ctx, c, E, f, kw) for c, E, f, kw in reqs]
    with lrfg.Batch(0, workers=4) as B:
        # every request twice, interleaved, all submitted before the first completes
        order = list(range(len(reqs))) * 2
        tickets = [(i, B.submit(reqs[i][0], reqs[i][1], reqs[i][2], **reqs[i][3])) for i in order]
        out = [(i, B.wait(t)) for i, t in tickets]
    for i, br in out:
        s, r = solo[i], br.result
        assert r.Aeff == s.Aeff, (i, r.Aeff, s.Aeff)
        assert r.iters == s.iters and r.rel_resid == s.rel_resid, (i, r.iters, s.iters)
        assert br.total_s >= br.run_s > 0.0 and br.queue_s >= 0.0
        assert 0 <= br.worker < 4 and br.peak_bytes > 0


def test_batch_matches_oracle():
    # the executor's answer against the FP64 oracle directly (d = 2 full format, and an untruncated TT)
    a, terms, w = square_inclusion(2, 31)
    ref = fg.solve_gani(a, np.array([1.0, 0.0]), tol=1e-10)["Aeff"]
    with lrfg.Batch(0, workers=2) as B:
        t_full = B.submit(a, [1.0, 0.0], lrfg.FULL, tol=1e-10)
        t_tt = B.submit(lr.tt_from_separable(terms, w), [1.0, 0.0], lrfg.TT, rank=31, maxit=80, tol=1e-10)
        r_full, r_tt = B.wait(t_full).result, B.wait(t_tt).result
    assert abs(r_full.Aeff - ref) <= 1e-8 * ref
    assert abs(r_tt.Aeff - ref) <= 1e-6 * ref


def _intervals(subs, results):
    return [(t0 + br.queue_s, t0 + br.queue_s + br.run_s) for t0, br in zip(subs, results)]


def _max_overlap(iv):
    ev = sorted([(s, 1) for s, _ in iv] + [(e, -1) for _, e in iv], key=lambda x: (x[0], x[1]))
    cur = best = 0
    for _, k in ev:
        cur += k
        best = max(best, cur)
    return best


def test_batch_admission_by_budget():
    # a budget below any request's footprint admits one request at a time (it runs alone); no cap
    # admits as many as there are workers
    _, t3, w3 = smoothed_cube(3, 45, contrast=10.0, full=False)
    c = lr.tt_from_separable(t3, w3)
    for budget, expect_serial in [(1, True), (0, False)]:
        with lrfg.Batch(0, workers=3, budget=budget) as B:
            subs, tickets = [], []
            for k in range(6):
                subs.append(time.monotonic())
                tickets.append(B.submit(c, [1.0, 0.0, 0.0], lrfg.TT, rank=6, maxit=20))
            res = [B.wait(t) for t in tickets]
            assert B.info() == (0, 0, 0)
        iv = _intervals(subs, res)
        if expect_serial:
            assert _max_overlap(iv) == 1, iv
        else:
            assert _max_overlap(iv) >= 2, iv
        assert len({r.result.Aeff for r in res}) == 1


def test_batch_errors_and_recovery():
    a, _, _ = square_inclusion(2, 31)
    with lrfg.Batch(0, workers=2) as B:
        with pytest.raises(lrfg.LrfgError):
            B.submit(np.ones((30, 30)), [1.0, 0.0], lrfg.FULL)  # even N: rejected at submission
        bad = a.copy()
        bad[3, 4] = -1.0
        t_bad = B.submit(bad, [1.0, 0.0], lrfg.FULL)
        t_ok = B.submit(a, [1.0, 0.0], lrfg.FULL, tol=1e-8)
        with pytest.raises(lrfg.LrfgError) as e:
            B.wait(t_bad)
        assert e.value.status == 1  # LRFG_EINVAL from the solve, reported at poll with its message
        assert "positive" in str(e.value) and "index 97" in str(e.value)
        ok = B.wait(t_ok)
        assert ok.result.converged
        with pytest.raises(lrfg.LrfgError):
            B.poll(t_ok)  # retired
        # poll without waiting eventually sees completion
        t = B.submit(a, [0.0, 1.0], lrfg.FULL, tol=1e-8)
        r = None
        for _ in range(20000):
            r = B.poll(t)
            if r is not None:
                break
            time.sleep(0.001)
        assert r is not None and r.result.converged


def test_destroy_drops_queued_requests_and_releases_waiting_polls():
    """Destroying the executor while a poll waits on a request that has not started: the poll returns it
    as dropped (solve status LRFG_EINVAL), the running request finishes, nothing hangs."""
    import ctypes as C
    import threading
    from paper_1902_07455_gb300 import _lib as L
    _, t3, w3 = smoothed_cube(3, 45, contrast=10.0, full=False)
    c = lr.tt_from_separable(t3, w3)
    B = lrfg.Batch(0, workers=1)
    tickets = [B.submit(c, [1.0, 0.0, 0.0], lrfg.TT, rank=8, maxit=30) for _ in range(4)]
    out = {}

    def waiter():
        ready, sst = C.c_int(), C.c_int()
        rep = L.lrfg_batch_report()
        st = B.lib.lrfg_batch_poll(B.h, C.c_ulonglong(tickets[-1]), 1, C.byref(ready), C.byref(sst), None,
                                   C.byref(rep))
        out.update(st=st, ready=ready.value, sst=sst.value, msg=rep.message.decode())

    th = threading.Thread(target=waiter)
    th.start()
    time.sleep(0.05)
    B.close()
    th.join(timeout=120)
    assert not th.is_alive()
    assert out["st"] == 0 and out["ready"] == 1
    assert out["sst"] == 1 and "dropped" in out["msg"]


def test_batch_groups_requests_of_one_shape_in_lockstep(ctx):
    """Batching across requests: with a group size > 1 the worker takes the queued requests of one shape
    (different microstructures, same grid, coefficient ranks and options) together and solves them in lockstep
    (lrfg_problems_solve).  Each result equals its own solve up to the rounding order of the batched products;
    requests of other shapes run alone."""
    d, N = 3, 27
    coeffs = [lr.tt_svd(lognormal_grf(d, N, ell=0.2, var=0.25, seed=s), rmax=6) for s in (41, 42, 43, 44)]
    assert len({tuple(c.shape[0] for c in a) for a in coeffs}) == 1
    kw = dict(rank=12, maxit=40, tol=5e-2, stop_on_increase=False, sketch_over=6)
    Es = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]
    solo = [_solo(ctx, a, E, lrfg.TT, kw) for a, E in zip(coeffs, Es)]
    _, t2, w2 = smoothed_cube(2, 63, contrast=10.0, full=False)
    other = (lr.tt_from_separable(t2, w2), [1.0, 0.0], lrfg.TT, dict(rank=6, maxit=30))
    other_solo = _solo(ctx, *other)
    blocker = lognormal_grf(3, 81, seed=45)  # keeps the single worker busy while the rest is queued
    with lrfg.Batch(0, workers=1, group=8) as B:
        tb = B.submit(blocker, [1.0, 0.0, 0.0], lrfg.FULL, tol=1e-8)
        tickets = [B.submit(a, E, lrfg.TT, **kw) for a, E in zip(coeffs[:2], Es[:2])]
        to = B.submit(other[0], other[1], other[2], **other[3])
        tickets += [B.submit(a, E, lrfg.TT, **kw) for a, E in zip(coeffs[2:], Es[2:])]
        assert B.wait(tb).group == 1
        out = [B.wait(t) for t in tickets]
        o = B.wait(to)
    assert o.group == 1 and o.result.Aeff == other_solo.Aeff
    assert all(br.group == 4 for br in out), [br.group for br in out]
    assert len({br.run_s for br in out}) == 1  # one solve served all four
    for br, s in zip(out, solo):
        assert br.result.converged and s.converged
        assert abs(br.result.Aeff - s.Aeff) <= 1e-9 * s.Aeff, (br.result.Aeff, s.Aeff)
        assert br.result.iters == s.iters
