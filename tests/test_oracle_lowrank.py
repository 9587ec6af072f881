"""Pins of the low-rank FP64 oracle (CP, Tucker, TT) against brute force, closed forms and the
full-format solve.

* every format operation against the same operation on the expanded full tensor (brute force);
* truncation error bounds of App. A.1.3 (Eckart–Young for d=2), A.2.3 (HOSVD) and A.3.3 (TT-SVD and
  rounding), and orthonormality of the truncated bases;
* rank 2 of the inclusion coefficient in all formats (Sec. 4.1);
* the exponential-sum inverse against 1/x on every integer k.k of the grid;
* the untruncated low-rank minimal-residual solve against the full PCG solve (to 1e-10);
* the rank-1 laminate: the low-rank solver must give the harmonic mean exactly at any N;
* the energy identity A_{N,r} - A_N = ||u_N - u_{N,r}||_A^2 >= 0 (Sec. 4.3).
"""
import numpy as np
import pytest

from oracle import expsum
from oracle import fourier_galerkin as fg
from oracle import lowrank as lr
from synthetic import laminate, lognormal_grf, random_tt, smoothed_cube, square_inclusion


def _rand_lr(fmt, shape, r, seed):
    rng = np.random.default_rng(seed)
    d = len(shape)
    if fmt == "tt":
        return random_tt(shape, [r] * (d - 1), seed=seed)
    if fmt == "tucker":
        return rng.standard_normal((r,) * d), [rng.standard_normal((n, r)) for n in shape]
    return rng.standard_normal(r), rng.standard_normal((shape[0], r)), rng.standard_normal((shape[1], r))


FMTS = [("tt", (5, 7, 9)), ("tt", (7, 9)), ("tucker", (5, 7, 9)), ("tucker", (7, 9)), ("cp", (7, 9))]


@pytest.mark.parametrize("fmt,shape", FMTS)
def test_format_ops_match_full(fmt, shape):
    f = lr.FORMATS[fmt]
    x = _rand_lr(fmt, shape, 3, 1)
    y = _rand_lr(fmt, shape, 2, 2)
    X, Y = f.full(x), f.full(y)
    assert np.allclose(f.full(f.add(x, y)), X + Y, atol=1e-12)
    assert np.allclose(f.full(f.had(x, y)), X * Y, atol=1e-12)
    assert np.allclose(f.full(f.scale(x, -2.5)), -2.5 * X, atol=1e-12)
    d = len(shape)
    assert np.allclose(f.full(f.dft(x)), fg.dft(X, d), atol=1e-12)
    assert np.allclose(f.full(f.idft(f.dft(x))), X, atol=1e-11)
    m = np.arange(shape[1]) + 0.5
    ref = X * m.reshape((1, -1) + (1,) * (d - 2))
    assert np.allclose(f.full(f.mmul(x, 1, m)), ref, atol=1e-12)
    assert np.isclose(f.dot(x, y), np.vdot(X, Y), rtol=1e-12)
    assert np.isclose(f.norm(x), np.linalg.norm(X), rtol=1e-12)


@pytest.mark.parametrize("fmt,shape", FMTS)
def test_round_without_loss_is_exact(fmt, shape):
    f = lr.FORMATS[fmt]
    x = f.add(_rand_lr(fmt, shape, 2, 3), _rand_lr(fmt, shape, 2, 4))  # rank 4 frame
    y = f.round(x, rmax=None, tol=1e-14)
    assert np.allclose(f.full(y), f.full(x), atol=1e-11)


def test_cp_truncation_is_eckart_young():
    x = _rand_lr("cp", (11, 13), 6, 5)
    X = lr.cp_full(x)
    s = np.linalg.svd(X, compute_uv=False)
    for k in [1, 2, 4]:
        y = lr.cp_round(x, rmax=k)
        err = np.linalg.norm(lr.cp_full(y) - X)
        assert np.isclose(err, np.sqrt(np.sum(s[k:] ** 2)), rtol=1e-10)


def test_tt_rounding_bound_and_orthonormality():
    shape = (7, 8, 9)
    x = random_tt(shape, [6, 6], seed=9)
    X = lr.tt_full(x)
    best = []
    for j in range(2):  # best rank-k error of each unfolding
        s = np.linalg.svd(X.reshape(int(np.prod(shape[: j + 1])), -1), compute_uv=False)
        best.append(s)
    for k in [2, 3, 5]:
        y = lr.tt_round(x, rmax=k)
        err = np.linalg.norm(lr.tt_full(y) - X)
        # quasi-optimality of TT-SVD truncation: err <= sqrt(sum_j eps_j^2), eps_j best error of unfolding j
        bound = np.sqrt(sum(np.sum(s[k:] ** 2) for s in best))
        assert err <= bound * (1 + 1e-10)
        assert err >= np.sqrt(np.sum(best[0][k:] ** 2)) * (1 - 1e-10)  # cannot beat the best unfolding
        for G in y[:-1]:
            M = G.reshape(-1, G.shape[2])
            assert np.abs(M.conj().T @ M - np.eye(M.shape[1])).max() <= 1e-13


def test_tt_svd_and_hosvd_error_bounds():
    A = lognormal_grf(3, 9, ell=0.2, seed=4)
    for tol in [1e-2, 1e-4, 1e-8]:
        t = lr.tt_svd(A, tol=tol)
        assert np.linalg.norm(lr.tt_full(t) - A) <= tol * np.linalg.norm(A) * (1 + 1e-10)
        c, F = lr.tucker_hosvd(A, tol=tol)
        assert np.linalg.norm(lr.tucker_full(c, F) - A) <= tol * np.linalg.norm(A) * (1 + 1e-10)
        for B in F:
            assert np.abs(B.T @ B - np.eye(B.shape[1])).max() <= 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_inclusion_coefficient_has_rank_two(d):
    """Sec. 4.1: the inclusion material has rank 2 in all three formats."""
    A = square_inclusion(d, 15)[0]
    t = lr.tt_svd(A, tol=1e-13)
    assert max(lr.tt_ranks(t)) == 2
    c, F = lr.tucker_hosvd(A, tol=1e-13)
    assert c.shape == (2,) * d
    if d == 2:
        assert len(lr.compress(A, "cp", tol=1e-13)[0]) == 2


@pytest.mark.parametrize("N,d", [(9, 3), (63, 2), (243, 3)])
@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-6])
def test_expsum_inverse_accuracy(N, d, eps):
    X = d * ((N - 1) // 2) ** 2
    t, w = expsum.expsum_inverse(X, eps)
    x = np.arange(1, X + 1, dtype=np.float64)
    assert np.max(np.abs(x * expsum.expsum_eval(x, t, w) - 1.0)) <= eps


def _solve_pair(A, terms, weights, fmt, d, N, rank, rank_tol, maxit, stop_on_increase=True, tol=1e-13):
    E = np.eye(d)[0]
    full = fg.solve_gani(A, E, tol=1e-13, maxit=3000)
    a_lr = lr.FORMATS[fmt].sep(terms, weights)
    op = lr.LowRankGaNi(a_lr, (N,) * d, fmt=fmt, rank=rank, pinv_eps=0.1, rank_tol=rank_tol)
    out = lr.minres(op, E, tol=tol, maxit=maxit, stop_on_increase=stop_on_increase)
    return full, op, out


@pytest.mark.parametrize("fmt,d,N", [("tt", 2, 15), ("cp", 2, 15), ("tucker", 2, 15), ("tt", 3, 9),
                                     ("tucker", 3, 9)])
def test_untruncated_lowrank_equals_full(fmt, d, N):
    A, terms, weights = square_inclusion(d, N)
    full, op, out = _solve_pair(A, terms, weights, fmt, d, N, rank=None, rank_tol=1e-15, maxit=400,
                                stop_on_increase=False)
    assert lr.relative_error(full["Aeff"], out["Aeff"]) <= 1e-10
    u_full = np.real(fg.idft(full["uh"], d))
    assert np.abs(op.full_field(out["u"]) - u_full).max() <= 1e-10 * np.abs(u_full).max()


@pytest.mark.parametrize("fmt,d,N", [("tt", 3, 45), ("tucker", 3, 45), ("cp", 2, 243), ("tt", 2, 243)])
def test_lowrank_laminate_is_harmonic_mean(fmt, d, N):
    A, terms, weights = laminate(d, N, contrast=10.0)
    f = A[(slice(None),) + (0,) * (d - 1)]
    harm = 1.0 / np.mean(1.0 / f)
    a_lr = lr.FORMATS[fmt].sep(terms, weights)
    op = lr.LowRankGaNi(a_lr, (N,) * d, fmt=fmt, rank=3, pinv_eps=0.1)
    out = lr.minres(op, np.eye(d)[0], tol=1e-12, maxit=300)
    assert abs(out["Aeff"] - harm) <= 1e-9 * harm


def test_energy_identity_and_rank_monotonicity():
    d, N = 2, 45
    A, terms, weights = smoothed_cube(d, N, contrast=10.0)
    E = np.eye(d)[0]
    full = fg.solve_gani(A, E, tol=1e-12)
    errs = []
    for r in [1, 2, 4, 8]:
        op = lr.LowRankGaNi(lr.tt_from_separable(terms, weights), (N,) * d, rank=r, pinv_eps=0.1)
        out = lr.minres(op, E, maxit=200)
        # A_{N,r} - A_N = ||u_N - u_{N,r}||_A^2 >= 0 for any admissible field
        assert out["Aeff"] >= full["Aeff"] * (1 - 1e-12)
        errs.append(lr.relative_error(full["Aeff"], out["Aeff"]))
    assert errs[-1] < errs[0]
    assert errs[-1] < 1e-3


def test_energy_identity_exact_for_any_field():
    """A(u) - A(u_N) = a(grad(u - u_N), grad(u - u_N)) for any trigonometric polynomial u (Sec. 4.3)."""
    d, N = 2, 21
    A = lognormal_grf(d, N, seed=2)
    E = np.array([1.0, 0.0])
    full = fg.solve_gani(A, E, tol=1e-14)
    rng = np.random.default_rng(0)
    pert = fg.dft(rng.standard_normal((N, N)), d)
    uh = full["uh"] + 0.1 * pert
    lhs = fg.homogenised_coefficient(uh, A, E) - full["Aeff"]
    e = np.real(fg.idft(fg.grad_hat(uh - full["uh"]), d))
    rhs = float(np.mean(A * np.sum(e * e, axis=0)))
    assert np.isclose(lhs, rhs, rtol=1e-10)


@pytest.mark.parametrize("fmt", ["tt", "tucker"])
def test_tolerance_truncation_bound_and_first_rank(fmt):
    """Tolerance truncation (App. A.3.3 / A.2.3): the result lies within tol ||x||, and the first TT bond
    (the mode-0 Tucker rank) is the smallest rank the full tensor's own mode-0 SVD allows with the
    per-bond share tol / sqrt(d-1) (tol / sqrt(d))."""
    rng = np.random.Generator(np.random.PCG64(31))
    shape = (9, 10, 11)
    terms = [[v / np.linalg.norm(v) for v in (rng.standard_normal(n) for n in shape)] for _ in range(7)]
    weights = 10.0 ** -np.arange(7)
    f = lr.FORMATS[fmt]
    x = f.sep(terms, weights)
    X = f.full(x)
    s = np.linalg.svd(X.reshape(shape[0], -1), compute_uv=False)
    for tol in [3e-2, 1e-3, 1e-5]:
        y = f.round(x, rmax=None, tol=tol)
        assert np.linalg.norm(f.full(y) - X) <= tol * np.linalg.norm(X) * (1 + 1e-10)
        loc = tol / np.sqrt(2.0 if fmt == "tt" else 3.0)
        tails = np.sqrt(np.cumsum(s[::-1] ** 2))[::-1]
        k_expected = next(k for k in range(1, len(s) + 1)
                          if (tails[k] if k < len(s) else 0.0) <= loc * np.linalg.norm(s))
        rank = y[0].shape[2] if fmt == "tt" else y[1][0].shape[1]
        assert rank == k_expected, (tol, rank, k_expected)


def test_rank_adaptive_minres_pins():
    """Rank-adapting MinRes (Sec. 4.3's proposal, oracle reading): started at the cap it is the fixed-rank
    iteration; raising the rank beats the fixed starting rank; untruncated at the cap it reaches the
    full-format Fourier-Galerkin solution (an independent solver) to 1e-10."""
    d, N = 2, 31
    A, terms, w = smoothed_cube(d, N, contrast=10.0)
    E = np.eye(d)[0]
    a_tt = lr.tt_from_separable(terms, w)
    op = lr.LowRankGaNi(a_tt, (N,) * d, fmt="tt", rank=8, pinv_eps=0.1)
    fixed8 = lr.minres(op, E, tol=1e-12, maxit=60)
    ad8 = lr.minres_rank_adaptive(op, E, rank_start=8, rank_step=2, tol=1e-12, maxit=60)
    assert ad8["Aeff"] == fixed8["Aeff"] and ad8["iters"] == fixed8["iters"] and ad8["rank"] == 8
    op2 = lr.LowRankGaNi(a_tt, (N,) * d, fmt="tt", rank=2, pinv_eps=0.1)
    fixed2 = lr.minres(op2, E, tol=1e-12, maxit=60)
    ad = lr.minres_rank_adaptive(op, E, rank_start=2, rank_step=2, tol=1e-12, maxit=60)
    assert ad["rank"] > 2 and ad["rel_resid"] < 0.5 * fixed2["rel_resid"]
    # at the cap it stops as the fixed-rank iteration does: on the first rise (True), not on a rise (False)
    ad_on = lr.minres_rank_adaptive(op, E, rank_start=2, rank_step=2, tol=1e-12, maxit=60, stop_on_increase=False)
    assert ad_on["rank"] == ad["rank"] and len(ad_on["history"]) > len(ad["history"])
    assert ad_on["rel_resid"] <= ad["rel_resid"]
    assert op.rank == 8  # restored
    # a tolerance met below the cap raises the rank: the result is the cap's, within the tolerance there
    loose = lr.minres_rank_adaptive(op, E, rank_start=2, rank_step=2, tol=2e-2, maxit=60)
    fixed2_loose = lr.minres(op2, E, tol=2e-2, maxit=60)
    assert fixed2_loose["rel_resid"] <= 2e-2  # the tolerance is reachable at rank 2 alone
    assert loose["rank"] == 8 and loose["rel_resid"] <= 2e-2
    assert lr.tt_ranks(loose["u"])[1] > 2
    # and it stops there only for an iterate of a step at the cap: more iterations than the rises alone take
    assert loose["iters"] > fixed2_loose["iters"]
    Ns = 15
    As, ts, ws = square_inclusion(2, Ns)
    full = fg.solve_gani(As, E, tol=1e-13, maxit=3000)
    opu = lr.LowRankGaNi(lr.tt_from_separable(ts, ws), (Ns, Ns), fmt="tt", rank=Ns, pinv_eps=0.1)
    out = lr.minres_rank_adaptive(opu, E, rank_start=2, rank_step=4, tol=1e-13, maxit=400)
    assert out["rank"] > 2 and out["rel_resid"] <= 1e-13
    assert lr.relative_error(full["Aeff"], out["Aeff"]) <= 1e-10


@pytest.mark.parametrize("fmt,d,N", [("tt", 2, 15), ("tt", 3, 9), ("tucker", 2, 15)])
def test_untruncated_anisotropic_lowrank_equals_full(fmt, d, N):
    """Constant anisotropic part (Sec. 4.4's B): the untruncated low-rank solve equals the full-format
    oracle's tensor-coefficient solve (an independent route: einsum over the full tensor field)."""
    B = np.array([[5.5, -4.5], [-4.5, 5.5]]) if d == 2 else np.array(
        [[4.25, -3.25, -1.25 * np.sqrt(2.0)], [-3.25, 4.25, 1.25 * np.sqrt(2.0)],
         [-1.25 * np.sqrt(2.0), 1.25 * np.sqrt(2.0), 7.5]])
    A, terms, weights = square_inclusion(d, N)
    At = A[None, None] * np.eye(d).reshape((d, d) + (1,) * d) + B.reshape((d, d) + (1,) * d)
    E = np.ones(d)
    full = fg.solve_gani(At, E, tol=1e-13, maxit=3000)
    op = lr.LowRankGaNi(lr.FORMATS[fmt].sep(terms, weights), (N,) * d, fmt=fmt, rank=None, pinv_eps=0.1,
                        rank_tol=1e-15, B=B)
    out = lr.minres(op, E, tol=1e-13, maxit=600, stop_on_increase=False)
    assert lr.relative_error(full["Aeff"], out["Aeff"]) <= 1e-10
