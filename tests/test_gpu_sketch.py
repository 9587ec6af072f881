"""The randomised TT rounding on the GPU (lrfg_tt_round_sketch, lrfg_tt_hadamard_round_sketch, and the solver
option sketch_over) against the oracle's restatement (oracle/sketch.py) with the same SplitMix64 sketch.

Both sides draw the sketch from the same counter-based stream, so the comparison is element by element on the
expanded tensors.  The GPU orthonormalises the sketched unfoldings by CholeskyQR2 and finishes with its Gram-SVD
rounding, the oracle by Householder QR and QR+SVD rounding; the span is the same, so the tolerance is that of
the deterministic rounding tests (1e-8), and 1e-7 for one operator application (five truncations)."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import lowrank as lr
from oracle import sketch as sk
from synthetic import lognormal_grf, random_tt, smoothed_cube

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def full(x):
    return lr.tt_full(x.numpy() if hasattr(x, "numpy") else x)


@pytest.mark.parametrize("shape,ranks,ell,rmax,seed", [((15, 17, 19), [8, 9], 6, 4, 3), ((45, 27, 63), [12, 10], 9, 5, 8),
                                                       ((31, 29), [14], 10, 6, 5), ((7, 9, 11), [4, 5], 6, 3, 1)])
def test_round_sketch_matches_oracle(ctx, shape, ranks, ell, rmax, seed):
    x = random_tt(shape, ranks, seed=seed)
    om = sk.sketch_tt(shape, ell, seed=seed + 100)
    ref = sk.tt_round_sketch(x, om, rmax=rmax)
    got = ctx.tt_round_sketch(lrfg.TTensor.from_numpy(x), ell, seed + 100, rmax)
    assert max(got.ranks) <= rmax
    assert rel(full(got), lr.tt_full(ref)) <= 1e-8


@pytest.mark.parametrize("shape,rx,ry,ell,rmax", [((45, 27, 63), [5, 4], [6, 7], 10, 6), ((81, 45, 63), [10, 10], [9, 8], 16, 8),
                                                  ((63, 45), [6], [7], 9, 5), ((9, 11, 13), [3, 4], [2, 3], 20, 5)])
def test_hadamard_round_sketch_matches_oracle(ctx, shape, rx, ry, ell, rmax):
    x = random_tt(shape, rx, seed=11)
    y = random_tt(shape, ry, seed=12)
    om = sk.sketch_tt(shape, ell, seed=77)
    ref = sk.tt_round_sketch(lr.tt_hadamard(x, y), om, rmax=rmax)
    got = ctx.tt_hadamard_round_sketch(lrfg.TTensor.from_numpy(x), lrfg.TTensor.from_numpy(y), ell, 77, rmax)
    assert rel(full(got), lr.tt_full(ref)) <= 1e-8
    # with the tolerance: within the bound of the tolerance rounding of the product
    z = lr.tt_full(lr.tt_hadamard(x, y))
    got_t = ctx.tt_hadamard_round_sketch(lrfg.TTensor.from_numpy(x), lrfg.TTensor.from_numpy(y), ell, 77, rmax, 0.3)
    assert rel(full(got_t), z) <= 0.3 * 1.0001 or max(got_t.ranks) == rmax


def test_round_sketch_exact_when_the_sketch_covers_the_ranks(ctx):
    shape = (27, 25, 23)
    x = random_tt(shape, [4, 5], seed=2)
    got = ctx.tt_round_sketch(lrfg.TTensor.from_numpy(x), 8, 9, 4)
    det = ctx.tt_round(lrfg.TTensor.from_numpy(x), 4)
    assert rel(full(got), full(det)) <= 1e-9


@pytest.mark.parametrize("d,N,rank,rx,over", [(2, 15, 4, [3], 4), (3, 9, 3, [2, 3], 3), (3, 27, 5, [4, 4], 6),
                                              (2, 63, 6, [5], 8)])
def test_sketched_apply_and_rhs_match_oracle(ctx, d, N, rank, rx, over):
    shape = (N,) * d
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    a = lr.tt_from_separable(terms, w)
    op = lr.LowRankGaNi(a, shape, fmt="tt", rank=rank, pinv_eps=0.1, sketch=(over, 41))
    x = random_tt(shape, rx, seed=21)
    ref = np.real(lr.tt_full(lr.tt_idft(op.apply(lr.tt_dft(x)))))
    P = ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=rank, pinv_eps=0.1, sketch_over=over, sketch_seed=41)
    out = P.apply(ctx.field_from_tt(lrfg.TTensor.from_numpy(x))).full()
    assert rel(out, ref) <= 1e-7
    E = np.eye(d)[0]
    refb = np.real(lr.tt_full(lr.tt_idft(op.rhs(E))))
    assert rel(P.rhs(E).full(), refb) <= 1e-7


@pytest.mark.parametrize("d,N,rank,over,kind", [(2, 63, 10, 6, "grf"), (3, 15, 5, 5, "cube"), (3, 27, 6, 6, "grf")])
def test_sketched_solve_matches_oracle_minres(ctx, d, N, rank, over, kind):
    shape = (N,) * d
    if kind == "grf":
        a = lr.tt_svd(lognormal_grf(d, N, ell=0.2, seed=4), rmax=5)
    else:
        _, terms, w = smoothed_cube(d, N, contrast=20.0, full=False)
        a = lr.tt_from_separable(terms, w)
    E = np.eye(d)[0]
    op = lr.LowRankGaNi(a, shape, fmt="tt", rank=rank, pinv_eps=0.1, sketch=(over, 5))
    ref = lr.minres(op, E, maxit=60)
    P = ctx.problem(lrfg.TTensor.from_numpy([np.ascontiguousarray(np.real(G)) for G in a]), lrfg.TT, rank=rank,
                    pinv_eps=0.1, tol=1e-10, maxit=60, sketch_over=over, sketch_seed=5)
    res, _ = P.solve(E, want_field=False)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"], res.iters, ref["iters"])


@pytest.mark.parametrize("d,N,rank,rx,over", [(2, 15, 4, [3], 4), (3, 27, 5, [4, 4], 6), (2, 63, 6, [5], 8)])
def test_kept_sketch_rank_apply_and_rhs_match_oracle(ctx, d, N, rank, rx, over):
    # sketch_keep: the two sketched truncations return their rank + over result (no final rounding to rank)
    shape = (N,) * d
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    a = lr.tt_from_separable(terms, w)
    op = lr.LowRankGaNi(a, shape, fmt="tt", rank=rank, pinv_eps=0.1, sketch=(over, 41, True))
    x = random_tt(shape, rx, seed=21)
    ref = np.real(lr.tt_full(lr.tt_idft(op.apply(lr.tt_dft(x)))))
    P = ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=rank, pinv_eps=0.1, sketch_over=over, sketch_seed=41,
                    sketch_keep=True)
    y = P.apply(ctx.field_from_tt(lrfg.TTensor.from_numpy(x)))
    assert rel(y.full(), ref) <= 1e-7
    assert max(y.tt().ranks) <= rank + over
    E = np.eye(d)[0]
    refb = np.real(lr.tt_full(lr.tt_idft(op.rhs(E))))
    assert rel(P.rhs(E).full(), refb) <= 1e-7


# a fixed number of iterations in the range where the residual still falls at every step on both sides (near
# stagnation the truncation to rank picks among near-equal singular values, so that the stop could move)
@pytest.mark.parametrize("d,N,rank,over,kind,its", [(2, 63, 10, 6, "grf", 10), (3, 27, 6, 6, "cube", 8)])
def test_kept_sketch_rank_solve_matches_oracle(ctx, d, N, rank, over, kind, its):
    shape = (N,) * d
    if kind == "grf":
        a = lr.tt_svd(lognormal_grf(d, N, ell=0.2, seed=4), rmax=5)
    else:
        _, terms, w = smoothed_cube(d, N, contrast=20.0, full=False)
        a = lr.tt_from_separable(terms, w)
    E = np.eye(d)[0]
    op = lr.LowRankGaNi(a, shape, fmt="tt", rank=rank, pinv_eps=0.1, sketch=(over, 5, True))
    ref = lr.minres(op, E, maxit=its, tol=1e-14, stop_on_increase=False)
    assert ref["iters"] == its  # still falling at the last step
    P = ctx.problem(lrfg.TTensor.from_numpy([np.ascontiguousarray(np.real(G)) for G in a]), lrfg.TT, rank=rank,
                    pinv_eps=0.1, tol=1e-14, maxit=its, stop_on_increase=False, sketch_over=over, sketch_seed=5,
                    sketch_keep=True)
    res, _ = P.solve(E, want_field=False)
    assert res.iters == its
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"], res.iters, ref["iters"])
    # the residual norm, near the truncation floor, follows the rounding order more than A_eff (quadratic in it)
    assert abs(res.rel_resid - ref["rel_resid"]) <= 5e-2 * ref["rel_resid"]


def test_sketch_keep_needs_the_sketch(ctx):
    A = lognormal_grf(2, 15, ell=0.2, seed=3)
    a = lr.tt_svd(A, rmax=4)
    with pytest.raises(lrfg.LrfgError):
        ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=4, sketch_keep=True)


def test_sketch_option_rejected_outside_tt_gani(ctx):
    A = lognormal_grf(2, 15, ell=0.2, seed=3)
    with pytest.raises(lrfg.LrfgError):
        ctx.problem(A, lrfg.FULL, sketch_over=4)
