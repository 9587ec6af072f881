"""Several macroscopic fields E of one TT problem solved in lockstep (lrfg_problem_solve_many), and the homogenised
tensor through it: each right-hand side against the same solve run alone and against the oracle's
minimal-residual solve; launches shared (fewer launches than the separate solves)."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import lowrank as lr
from synthetic import lognormal_grf, smoothed_cube

pytestmark = pytest.mark.gpu


def _coeff(d, N, kind):
    if kind == "grf":
        # variance 1/4: contrast ~20 (as the inclusions), so that the iterations converge well above their floor
        a = lr.tt_svd(lognormal_grf(d, N, ell=0.2, var=0.25, seed=7), rmax=8)
        assert np.real(lr.tt_full(a)).min() > 0.0  # the compressed coefficient stays positive
        return a
    _, terms, w = smoothed_cube(d, N, contrast=20.0, full=False)
    return lr.tt_from_separable(terms, w)


# tol: a residual each right-hand side reaches well above its truncation floor, where the iterates depend smoothly
# on the rounding order (stagnating near the floor, the "best iterate" can move with it; see the oracle test below)
@pytest.mark.parametrize("d,N,rank,over,kind,tol,keep", [(3, 27, 12, 6, "grf", 5e-2, False),
                                                         (3, 15, 5, 0, "cube", 5e-2, False),
                                                         (2, 45, 8, 8, "grf", 5e-2, False),
                                                         (2, 31, 6, 0, "cube", 5e-2, False),
                                                         (2, 45, 8, 8, "grf", 5e-2, True)])
def test_lockstep_equals_separate_solves(ctx, d, N, rank, over, kind, tol, keep):
    a = _coeff(d, N, kind)
    Es = np.eye(d).tolist() + [[1.0] * d, [0.0] * d]
    kw = dict(rank=rank, pinv_eps=0.1, tol=tol, maxit=40, stop_on_increase=False, sketch_over=over, sketch_keep=keep)
    P = ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, **kw)
    n0 = ctx.launch_count()
    many = P.solve_many(Es)
    n_many = ctx.launch_count() - n0
    n0 = ctx.launch_count()
    alone = [P.solve(E, want_field=False)[0] for E in Es]
    n_alone = ctx.launch_count() - n0
    for m, s, E in zip(many, alone, Es):
        if not any(E):
            assert m.Aeff == 0.0 and s.Aeff == 0.0
            continue
        assert s.converged and m.converged
        assert abs(m.Aeff - s.Aeff) <= 1e-9 * s.Aeff, (E, m.Aeff, s.Aeff, m.iters, s.iters)
        assert m.iters == s.iters
    assert n_many < 0.75 * n_alone, (n_many, n_alone)
    P.free()


# a fixed number of iterations on both sides (no stopping test that a rounding-level difference could move), few
# enough that the residual still falls monotonically: at the truncation floor it rises and falls (Sec. 4.3), and
# which iterate is the best there moves with the rounding order
@pytest.mark.parametrize("d,N,rank,over", [(3, 21, 5, 5), (2, 45, 8, 0), (3, 15, 4, 0)])
def test_lockstep_matches_oracle(ctx, d, N, rank, over):
    a = _coeff(d, N, "grf")
    Es = np.eye(d).tolist() + [[1.0, 1.0] + [0.0] * (d - 2)]
    sketch = (over, 0) if over else None
    op = lr.LowRankGaNi(a, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.1, sketch=sketch)
    P = ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=rank, pinv_eps=0.1, tol=1e-14, maxit=6,
                    stop_on_increase=False, sketch_over=over)
    many = P.solve_many(Es)
    for m, E in zip(many, Es):
        ref = lr.minres(op, np.asarray(E), tol=1e-14, maxit=6, stop_on_increase=False)
        assert abs(m.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (E, m.Aeff, ref["Aeff"], m.iters, ref["iters"])
    P.free()


def test_tt_homogenised_tensor_in_lockstep(ctx):
    d, N, rank = 3, 21, 5
    a = _coeff(d, N, "grf")
    op = lr.LowRankGaNi(a, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.1, sketch=(5, 0))
    P = ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=rank, pinv_eps=0.1, tol=1e-14, maxit=12,
                    stop_on_increase=False, sketch_over=5)
    T, results = P.aeff_tensor(with_results=True)
    assert len(results) == 6
    eye = np.eye(d)
    mr = dict(tol=1e-14, maxit=12, stop_on_increase=False)
    q = {a_: lr.minres(op, eye[a_], **mr)["Aeff"] for a_ in range(d)}
    for i in range(d):
        assert abs(T[i, i] - q[i]) <= 1e-6 * q[i]
    s01 = lr.minres(op, eye[0] + eye[1], **mr)["Aeff"]
    assert abs(T[0, 1] - 0.5 * (s01 - q[0] - q[1])) <= 1e-6 * q[0]
    assert np.array_equal(T, T.T)
    P.free()


# rank adaptation in lockstep: each item follows the rank-adapting iteration of its own solve (frozen while
# others still improve at the current rank, restarted from its best iterate at every rise).  Batched and single
# launches round differently, and a rise is decided by "the residual fails to decrease", which can be a near-tie
# (rises below 1 % occur here): the counts may differ by a step or two, A_eff (deep below the tolerance) may not.
@pytest.mark.parametrize("d,N,rank,start,step,over", [(2, 31, 8, 2, 2, 0), (3, 21, 8, 2, 3, 0), (3, 21, 8, 2, 3, 4)])
def test_rank_adaptive_lockstep_equals_separate_solves(ctx, d, N, rank, start, step, over):
    # the axis fields of the symmetric cube: items of like behaviour, which is where lockstep pays (unlike items
    # wait for one another at each rise); and one E = 0
    a = _coeff(d, N, "cube")
    Es = np.eye(d).tolist() + [[0.0] * d]
    P = ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=rank, pinv_eps=0.1, tol=1e-12, maxit=50,
                    rank_start=start, rank_step=step, sketch_over=over)
    n0 = ctx.launch_count()
    many = P.solve_many(Es)
    n_many = ctx.launch_count() - n0
    n0 = ctx.launch_count()
    alone = [P.solve(E, want_field=False)[0] for E in Es]
    n_alone = ctx.launch_count() - n0
    for m, s, E in zip(many, alone, Es):
        if not any(E):
            assert m.Aeff == 0.0 and s.Aeff == 0.0
            continue
        assert abs(m.Aeff - s.Aeff) <= 1e-7 * s.Aeff, (E, m.Aeff, s.Aeff, m.iters, s.iters)
        assert abs(m.iters - s.iters) <= 2 and m.ranks == s.ranks, (E, m.iters, s.iters, m.ranks, s.ranks)
    # fewer launches than the separate solves (by less than at a fixed rank: the items wait for one another at
    # each rise, and without the sketch the P~^-1 truncation runs item by item)
    assert n_many < n_alone, (n_many, n_alone)
    P.free()


@pytest.mark.parametrize("d,N,rank,start,step", [(2, 31, 8, 2, 2), (3, 21, 8, 2, 3)])
def test_rank_adaptive_lockstep_matches_oracle(ctx, d, N, rank, start, step):
    a = _coeff(d, N, "cube")
    Es = [np.eye(d)[0], np.eye(d)[1]]
    op = lr.LowRankGaNi(a, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.1)
    P = ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=rank, pinv_eps=0.1, tol=1e-12, maxit=50,
                    rank_start=start, rank_step=step)
    many = P.solve_many([list(E) for E in Es])
    for m, E in zip(many, Es):
        ref = lr.minres_rank_adaptive(op, E, start, step, tol=1e-12, maxit=50)
        assert abs(m.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (E, m.Aeff, ref["Aeff"], m.iters, ref["iters"])
        assert list(m.ranks[:d + 1]) == lr.tt_ranks(ref["u"])
    P.free()
