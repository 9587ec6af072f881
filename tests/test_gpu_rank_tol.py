"""Tolerance truncation on the GPU (rank_tol) against the oracle's tolerance rounding and solver on the
same seeded inputs.

The test tensors are sums of rank-one terms with weights 10^-i, so their singular values fall off by
about a decade each and no singular value lies near a truncation threshold: the kept ranks are unique
and must equal the oracle's exactly; the truncated tensors then agree to the Gram-SVD accuracy (1e-8
relative, as for fixed-rank truncation).  A solve with rank_tol meets the FP64-path tolerance against
the oracle's minimal-residual iteration with the same truncation rule (1e-6 on A_eff)."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import lowrank as lr
from synthetic import smoothed_cube

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def decaying_terms(shape, n_terms, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    terms = [[v / np.linalg.norm(v) for v in (rng.standard_normal(n) for n in shape)] for _ in range(n_terms)]
    return terms, 10.0 ** -np.arange(n_terms)


@pytest.mark.parametrize("shape,tol,cap", [((9, 11, 13), 1e-3, 7), ((9, 11, 13), 1e-5, 7),
                                           ((15, 13, 11), 3e-2, 5), ((21, 17), 1e-4, 6), ((9, 11, 13), 1e-5, 4)])
def test_tt_round_tol(ctx, shape, tol, cap):
    terms, w = decaying_terms(shape, 7, seed=31)
    x = lr.tt_from_separable(terms, w)
    ref = lr.tt_round(x, rmax=cap, tol=tol)
    out = ctx.tt_round(lrfg.TTensor.from_numpy(x), cap, tol=tol)
    assert out.ranks == lr.tt_ranks(ref), (out.ranks, lr.tt_ranks(ref))
    assert rel(lr.tt_full(out.numpy()), lr.tt_full(ref)) <= 1e-8


@pytest.mark.parametrize("shape,tol,cap", [((9, 11, 13), 1e-3, 7), ((15, 13, 11), 1e-5, 7), ((21, 17), 1e-4, 3)])
def test_tucker_round_tol(ctx, shape, tol, cap):
    terms, w = decaying_terms(shape, 7, seed=32)
    x = lr.tucker_from_separable(terms, w)
    ref_c, ref_f = lr.tucker_round(x, rmax=cap, tol=tol)
    out = ctx.tucker_round(lrfg.TuckerTensor.from_numpy(*x), cap, tol=tol)
    assert out.ranks == [f.shape[1] for f in ref_f]
    c, f = out.numpy()
    assert rel(lr.tucker_full(c, f), lr.tucker_full(ref_c, ref_f)) <= 1e-8


def test_tt_round_tol_zero_is_fixed_rank(ctx):
    terms, w = decaying_terms((9, 11, 13), 7, seed=33)
    x = lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w))
    a = ctx.tt_round(x, 4)
    b = ctx.tt_round(x, 4, tol=0.0)
    assert a.ranks == b.ranks == [1, 4, 4, 1]
    assert rel(lr.tt_full(a.numpy()), lr.tt_full(b.numpy())) == 0.0


@pytest.mark.parametrize("fmt,d,N,cap,rank_tol", [("tt", 2, 45, 20, 1e-4), ("tt", 2, 45, 20, 1e-6),
                                                  ("tt", 3, 27, 12, 1e-4), ("tucker", 2, 45, 16, 1e-5)])
def test_solve_rank_tol_matches_oracle(ctx, fmt, d, N, cap, rank_tol):
    _, terms, w = smoothed_cube(d, N, contrast=10.0, full=False)
    E = np.eye(d)[0]
    a_lr = lr.FORMATS[fmt].sep(terms, w)
    op = lr.LowRankGaNi(a_lr, (N,) * d, fmt=fmt, rank=cap, pinv_eps=0.1, rank_tol=rank_tol)
    ref = lr.minres(op, E, tol=1e-10, maxit=40)
    coeff = lrfg.TTensor.from_numpy(a_lr) if fmt == "tt" else lrfg.TuckerTensor.from_numpy(*a_lr)
    P = ctx.problem(coeff, lrfg.TT if fmt == "tt" else lrfg.TUCKER, rank=cap, tol=1e-10, maxit=40,
                    rank_tol=rank_tol)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    # the stop (first residual that fails to decrease, Sec. 4.3) is compared only where the oracle's rise is
    # clear: at a near-tie (a rise below 1 %) a rounding-level difference decides whether the GPU stops there
    # too or goes on; either way its best residual sits at the same truncation floor (within a factor 2)
    hist = ref["history"]
    near_tie = len(hist) >= 2 and hist[-1] <= 1.01 * min(hist[:-1])
    if not near_tie:
        assert abs(res.iters - ref["iters"]) <= 2, (res.iters, ref["iters"])
    assert res.rel_resid <= 2.0 * ref["rel_resid"], (res.rel_resid, ref["rel_resid"])
    ranks = u.info()[3]
    assert max(ranks) <= cap
    u.free()
    P.free()


def test_rank_tol_invalid(ctx):
    _, terms, w = smoothed_cube(2, 15, contrast=10.0, full=False)
    coeff = lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w))
    with pytest.raises(lrfg.LrfgError):
        ctx.problem(coeff, lrfg.TT, rank=5, rank_tol=1.5)
    with pytest.raises(lrfg.LrfgError):
        ctx.tt_round(coeff, 3, tol=-1.0)


@pytest.mark.parametrize("d,N,cap,start,step", [(2, 31, 8, 2, 2), (3, 21, 8, 2, 3)])
def test_rank_adaptive_solve_matches_oracle(ctx, d, N, cap, start, step):
    """Rank-adapting MinRes (rank_start/rank_step) against the oracle's minres_rank_adaptive: the same
    rank schedule, so A_eff agrees to the FP64-path tolerance and the returned ranks match."""
    _, terms, w = smoothed_cube(d, N, contrast=10.0, full=False)
    E = np.eye(d)[0]
    a_tt = lr.tt_from_separable(terms, w)
    op = lr.LowRankGaNi(a_tt, (N,) * d, fmt="tt", rank=cap, pinv_eps=0.1)
    ref = lr.minres_rank_adaptive(op, E, rank_start=start, rank_step=step, tol=1e-12, maxit=50)
    P = ctx.problem(lrfg.TTensor.from_numpy(a_tt), lrfg.TT, rank=cap, tol=1e-12, maxit=50, rank_start=start,
                    rank_step=step)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    assert abs(res.iters - ref["iters"]) <= 2, (res.iters, ref["iters"])
    assert u.info()[3] == lr.tt_ranks(ref["u"])
    u.free()
    # started at the cap it is the fixed-rank solve, bit for bit
    fixed, _ = ctx.problem(lrfg.TTensor.from_numpy(a_tt), lrfg.TT, rank=cap, tol=1e-12, maxit=50).solve(
        E, want_field=False)
    at_cap, _ = ctx.problem(lrfg.TTensor.from_numpy(a_tt), lrfg.TT, rank=cap, tol=1e-12, maxit=50,
                            rank_start=cap, rank_step=step).solve(E, want_field=False)
    assert at_cap.Aeff == fixed.Aeff and at_cap.iters == fixed.iters
    P.free()


@pytest.mark.parametrize("fmt,d,N,cap,start,step", [("tucker", 2, 31, 8, 2, 2), ("tucker", 3, 15, 6, 2, 2),
                                                    ("cp", 2, 31, 8, 2, 3)])
def test_rank_adaptive_tucker_cp_matches_oracle(ctx, fmt, d, N, cap, start, step):
    _, terms, w = smoothed_cube(d, N, contrast=10.0, full=False)
    E = np.eye(d)[0]
    op = lr.LowRankGaNi(lr.FORMATS[fmt].sep(terms, w), (N,) * d, fmt=fmt, rank=cap, pinv_eps=0.1)
    ref = lr.minres_rank_adaptive(op, E, rank_start=start, rank_step=step, tol=1e-12, maxit=40)
    P = ctx.problem(lrfg.TuckerTensor.from_numpy(*lr.tucker_from_separable(terms, w)),
                    lrfg.TUCKER if fmt == "tucker" else lrfg.CP, rank=cap, tol=1e-12, maxit=40, rank_start=start,
                    rank_step=step)
    res, _ = P.solve(E, want_field=False)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    # near stagnation at the cap the residual changes by parts in 1e6 per step, so "fails to decrease" may
    # fire a few steps apart on the two sides (Gram-SVD vs QR+SVD rounding).  The floor the residual stagnates
    # at is set by the truncation to the cap, which both sides share, so iterating a few steps longer moves
    # the residual reached by a modest factor either way, never by orders of magnitude
    ratio = res.rel_resid / ref["rel_resid"]
    assert 0.25 <= ratio <= 2.0, (res.rel_resid, ref["rel_resid"], res.iters, ref["iters"])
