"""Tucker format on the GPU (App. A.2) against the oracle's Tucker path (Fourier-space, complex) on the
same seeded inputs: truncation, one operator application, right-hand side, and the minimal-residual
solve.  Tolerances as for the TT path: a truncation is Gram/Cholesky-based (error ~ eps sigma_1^2 /
(sigma_k gap)), 1e-8 on the expanded result; one operator application contains five truncations,
1e-7; A_eff after a solve 1e-6 (the FP64-path target); the laminate's closed form 1e-9."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import lowrank as lr
from synthetic import laminate, smoothed_cube, square_inclusion

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def random_tucker(shape, ranks, seed):
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(ranks))
    factors = [rng.standard_normal((n, r)) / np.sqrt(n) for n, r in zip(shape, ranks)]
    return core, factors


def real_full(xh):
    return np.real(lr.tucker_full(*lr.tucker_idft(xh)))


@pytest.mark.parametrize("shape,ranks,rmax", [((15, 13, 11), (6, 5, 4), 3), ((21, 17), (7, 6), 4),
                                              ((9, 9, 9), (12, 12, 12), 5)])
def test_tucker_round(ctx, shape, ranks, rmax):
    core, factors = random_tucker(shape, ranks, seed=7)
    ref = lr.tucker_full(*lr.tucker_round((core, factors), rmax=rmax))
    out = ctx.tucker_round(lrfg.TuckerTensor.from_numpy(core, factors), rmax)
    c, f = out.numpy()
    assert out.ranks == [min(rmax, r) for r in ranks]
    assert rel(lr.tucker_full(c, f), ref) <= 1e-8
    # the factors come out orthonormal (where the input has full column rank)
    for F in f:
        assert np.abs(F.T @ F - np.eye(F.shape[1])).max() <= 1e-8


def test_tucker_round_rank_deficient_sum(ctx):
    core, factors = random_tucker((11, 9, 7), (3, 3, 2), seed=3)
    x = (core, factors)
    s = lr.tucker_add(x, x)  # twice x, in a rank-doubled frame
    out = ctx.tucker_round(lrfg.TuckerTensor.from_numpy(*s), 4)
    assert rel(lr.tucker_full(*out.numpy()), 2.0 * lr.tucker_full(core, factors)) <= 1e-12


def _oracle_op(terms, w, shape, rank):
    return lr.LowRankGaNi(lr.tucker_from_separable(terms, w), shape, fmt="tucker", rank=rank, pinv_eps=0.1)


@pytest.mark.parametrize("d,N,rank,rx", [(3, 15, 4, (3, 3, 2)), (2, 45, 6, (5, 4)), (3, 27, 5, (4, 4, 4))])
def test_tucker_apply_and_rhs(ctx, d, N, rank, rx):
    shape = (N,) * d
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    op = _oracle_op(terms, w, shape, rank)
    core, factors = random_tucker(shape, rx, seed=21)
    ref = real_full(op.apply(lr.tucker_dft((core, factors))))
    a_tk = lrfg.TuckerTensor.from_numpy(*lr.tucker_from_separable(terms, w))
    P = ctx.problem(a_tk, lrfg.TUCKER, rank=rank, pinv_eps=0.1)
    out = P.apply(ctx.field_from_tucker(lrfg.TuckerTensor.from_numpy(core, factors))).full()
    # The Gram-SVD truncation drops the pivots of a factor's Gram matrix below eps = 1e-16 of its largest
    # diagonal, i.e. directions of norm up to sqrt(eps) = 1e-8 of a column (the oracle's QR+SVD keeps them).
    # The P~^-1 product's factors [G_1 B .. G_R B] are R r nearly collinear columns (R = 8 here), so the
    # operator carries such differences from up to R r dropped directions: 7e-9..3e-7 across rounding orders
    # of the same build for (2, 45, 6) — a bound of 1e-6, not a rounding-level one.
    assert rel(out, ref) <= 1e-6
    E = np.eye(d)[0]
    assert rel(P.rhs(E).full(), real_full(op.rhs(E))) <= 1e-7


@pytest.mark.parametrize("d,N,rank,kind", [(2, 45, 8, "square"), (3, 15, 5, "square"), (3, 27, 6, "cube")])
def test_tucker_solve_matches_oracle_minres(ctx, d, N, rank, kind):
    shape = (N,) * d
    _, terms, w = square_inclusion(d, N) if kind == "square" else smoothed_cube(d, N, contrast=10.0)
    op = _oracle_op(terms, w, shape, rank)
    E = np.eye(d)[0]
    ref = lr.minres(op, E, tol=1e-10, maxit=60)
    P = ctx.problem(lrfg.TuckerTensor.from_numpy(*lr.tucker_from_separable(terms, w)), lrfg.TUCKER, rank=rank,
                    pinv_eps=0.1, tol=1e-10, maxit=60)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"]
    # near a residual plateau the stop iteration depends on rounding; A_eff does not
    assert abs(res.iters - ref["iters"]) <= 3
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-12 * res.Aeff


def test_tucker_laminate_is_harmonic_mean(ctx):
    d, N = 3, 81
    A, terms, w = laminate(d, N, contrast=10.0)
    harm = 1.0 / np.mean(1.0 / A[:, 0, 0])
    P = ctx.problem(lrfg.TuckerTensor.from_numpy(*lr.tucker_from_separable(terms, w)), lrfg.TUCKER, rank=3,
                    tol=1e-12, maxit=200)
    res, _ = P.solve(np.eye(d)[0])
    assert abs(res.Aeff - harm) <= 1e-9 * harm


def test_tucker_coefficient_from_grid(ctx):
    # a separable rank-2 coefficient given as grid values: the HOSVD compression is exact
    d, N, rank = 3, 15, 5
    A, terms, w = square_inclusion(d, N)
    E = np.eye(d)[0]
    ref = lr.minres(_oracle_op(terms, w, (N,) * d, rank), E, tol=1e-10, maxit=60)
    P = ctx.problem(A, lrfg.TUCKER, rank=rank, pinv_eps=0.1, tol=1e-10, maxit=60)
    assert P.coeff_ranks()[:3] == [2, 2, 2]
    res, _ = P.solve(E, want_field=False)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"]


# ---- canonical (CP) format, d = 2 (App. A.1): the oracle's CP path against LRFG_CP --------------------
def _cp_as_tucker(c, B1, B2):
    return lrfg.TuckerTensor.from_numpy(np.diag(np.asarray(c, dtype=np.float64)), [B1, B2])


@pytest.mark.parametrize("N,rank,kind", [(45, 6, "square"), (63, 8, "cube"), (31, 4, "cube")])
def test_cp_solve_matches_oracle_minres(ctx, N, rank, kind):
    d = 2
    _, terms, w = square_inclusion(d, N) if kind == "square" else smoothed_cube(d, N, contrast=10.0)
    op = lr.LowRankGaNi(lr.cp_from_separable(terms, w), (N, N), fmt="cp", rank=rank, pinv_eps=0.1)
    E = np.eye(d)[0]
    ref = lr.minres(op, E, tol=1e-10, maxit=60)
    P = ctx.problem(_cp_as_tucker(*lr.cp_from_separable(terms, w)), lrfg.CP, rank=rank, pinv_eps=0.1, tol=1e-10,
                    maxit=60)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"]
    # fields agree up to a constant (P~^-1 does not vanish at k = 0, so rounding noise there can leave a
    # tiny mean); compare the zero-mean parts
    g, h = u.full(), np.real(lr.cp_full(lr.cp_idft(ref["u"])))
    # the field carries the truncations' sqrt(eps)-level differences (see test_tucker_apply_and_rhs) through the
    # iterations; A_eff, quadratic in the field's error, is the tight check above
    assert rel(g - g.mean(), h - h.mean()) <= 1e-5


def test_cp_apply_matches_oracle(ctx):
    N, rank = 45, 5
    _, terms, w = smoothed_cube(2, N, contrast=10.0)
    op = lr.LowRankGaNi(lr.cp_from_separable(terms, w), (N, N), fmt="cp", rank=rank, pinv_eps=0.1)
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(3), rng.standard_normal((N, 3)), rng.standard_normal((N, 3)))
    ref = np.real(lr.cp_full(lr.cp_idft(op.apply(lr.cp_dft(x)))))
    P = ctx.problem(_cp_as_tucker(*lr.cp_from_separable(terms, w)), lrfg.CP, rank=rank, pinv_eps=0.1)
    out = P.apply(ctx.field_from_tucker(_cp_as_tucker(*x))).full()
    assert rel(out, ref) <= 1e-7


def test_cp_three_dimensional_is_not_supported(ctx):
    from paper_1902_07455_gb300 import _lib as L
    with pytest.raises(lrfg.LrfgError) as e:
        ctx.problem(np.ones((9, 9, 9)), lrfg.CP, rank=2)
    assert e.value.status == L.LRFG_ENOTSUP
