"""A batch of microstructures of one shape solved together (lrfg_problems_solve): each problem's minimal-residual
iteration (Sec. 4.3) in lockstep with the others, item i with its own coefficient in the material product and the
right-hand side.  Each result against the same problem solved alone and against the oracle's solve of it; launches
shared; problems of different shapes fall back to separate solves."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import lowrank as lr
from synthetic import lognormal_grf

pytestmark = pytest.mark.gpu


def _coeffs(d, N, rmax, seeds, var=0.25):
    out = []
    for s in seeds:
        a = lr.tt_svd(lognormal_grf(d, N, ell=0.2, var=var, seed=s), rmax=rmax)
        assert np.real(lr.tt_full(a)).min() > 0.0
        out.append(a)
    ranks = {tuple(c.shape[0] for c in a) for a in out}
    assert len(ranks) == 1, ranks  # one shape: the same coefficient TT ranks
    return out


@pytest.mark.parametrize("d,N,rank,over,adapt", [(3, 27, 10, 6, False), (2, 45, 8, 8, False), (3, 21, 12, 0, False),
                                                  (3, 27, 10, 6, True)])
def test_microstructures_together_equal_separate_solves(ctx, d, N, rank, over, adapt):
    coeffs = _coeffs(d, N, 6, seeds=[11, 12, 13, 14])
    Es = [np.eye(d)[i % d] for i in range(len(coeffs))]
    kw = dict(rank=rank, pinv_eps=0.1, tol=5e-2, maxit=40, stop_on_increase=False, sketch_over=over)
    if adapt:
        kw.update(rank_start=rank // 2, rank_step=rank // 4)
    Ps = [ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, **kw) for a in coeffs]
    n0 = ctx.launch_count()
    together = lrfg.Problem.solve_together(Ps, Es)
    n_together = ctx.launch_count() - n0
    n0 = ctx.launch_count()
    alone = [P.solve(E, want_field=False)[0] for P, E in zip(Ps, Es)]
    n_alone = ctx.launch_count() - n0
    for m, s in zip(together, alone):
        assert s.converged and m.converged
        assert abs(m.Aeff - s.Aeff) <= 1e-9 * s.Aeff, (m.Aeff, s.Aeff, m.iters, s.iters)
        assert m.iters == s.iters
    assert n_together < 0.75 * n_alone, (n_together, n_alone)
    # the coefficients differ, so do the results
    assert len({round(m.Aeff, 6) for m in together}) == len(together)
    for P in Ps:
        P.free()


# a fixed number of iterations on both sides, few enough that the residual still falls monotonically (at the
# truncation floor the best iterate moves with the rounding order)
@pytest.mark.parametrize("d,N,rank,over", [(3, 21, 5, 5), (2, 45, 8, 0)])
def test_microstructures_together_match_oracle(ctx, d, N, rank, over):
    coeffs = _coeffs(d, N, 5, seeds=[21, 22, 23])
    Es = [np.eye(d)[0], np.eye(d)[1], np.ones(d)]
    sketch = (over, 0) if over else None
    Ps = [ctx.problem(lrfg.TTensor.from_numpy(a), lrfg.TT, rank=rank, pinv_eps=0.1, tol=1e-14, maxit=6,
                      stop_on_increase=False, sketch_over=over) for a in coeffs]
    together = lrfg.Problem.solve_together(Ps, Es)
    for a, m, E in zip(coeffs, together, Es):
        op = lr.LowRankGaNi(a, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.1, sketch=sketch)
        ref = lr.minres(op, np.asarray(E), tol=1e-14, maxit=6, stop_on_increase=False)
        assert abs(m.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (E, m.Aeff, ref["Aeff"], m.iters, ref["iters"])
    for P in Ps:
        P.free()


def test_problems_of_different_shapes_run_one_after_the_other(ctx):
    # different grids (and different coefficient ranks): no lockstep, every result that of its own solve
    d = 2
    a0 = _coeffs(d, 31, 5, seeds=[31])[0]
    a1 = _coeffs(d, 45, 7, seeds=[32])[0]
    kw = dict(rank=6, pinv_eps=0.1, tol=5e-2, maxit=30, stop_on_increase=False)
    Ps = [ctx.problem(lrfg.TTensor.from_numpy(a0), lrfg.TT, **kw), ctx.problem(lrfg.TTensor.from_numpy(a1), lrfg.TT, **kw)]
    Es = [[1.0, 0.0], [0.0, 1.0]]
    together = lrfg.Problem.solve_together(Ps, Es)
    for P, E, m in zip(Ps, Es, together):
        s = P.solve(E, want_field=False)[0]
        assert m.Aeff == s.Aeff and m.iters == s.iters
    for P in Ps:
        P.free()
