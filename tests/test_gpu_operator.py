"""Rows a1-a9 composed: the preconditioned GaNi operator, right-hand side and A_eff, FULL and TT, CUDA
path vs the oracle (FP64) on the same seeded inputs.

Tolerances: one FULL application is a chain of FP64 FFTs and pointwise products: 1e-11 relative.  One
TT application contains five truncations (Gram-SVD, see test_gpu_tt): 1e-7 relative on the expanded
result.  A_eff after a solve: 1e-6 relative (the FP64-path target), typically ~1e-10 is seen."""
import numpy as np
import pytest
import torch

import paper_1902_07455_gb300 as lrfg
from oracle import fourier_galerkin as fg
from oracle import lowrank as lr
from synthetic import laminate, lognormal_grf, random_tt, smoothed_cube, square_inclusion

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("d,N", [(2, 15), (2, 63), (3, 9), (3, 27), (3, 45)])
def test_full_apply_and_rhs(ctx, d, N):
    A = lognormal_grf(d, N, ell=0.2, seed=13)
    u = np.random.default_rng(1).standard_normal((N,) * d)
    P = ctx.problem(A, lrfg.FULL)
    f = ctx.field_from_full(u)
    assert rel(f.full(), u) <= 1e-13  # forward + inverse round trip
    out = P.apply(f).full()
    Pinv = fg.precond_inv((N,) * d)
    ref = np.real(fg.idft(Pinv * fg.gani_operator(fg.dft(u, d), A), d))
    assert rel(out, ref) <= 1e-11
    E = np.eye(d)[0]
    b = P.rhs(E).full()
    refb = np.real(fg.idft(Pinv * fg.gani_rhs(A, E), d))
    assert rel(b, refb) <= 1e-11


@pytest.mark.parametrize("d,N,kind", [(2, 63, "square"), (3, 15, "grf"), (3, 27, "square"), (2, 45, "grf")])
def test_full_solve(ctx, d, N, kind):
    A = square_inclusion(d, N)[0] if kind == "square" else lognormal_grf(d, N, ell=0.2, seed=3)
    E = np.eye(d)[0]
    ref = fg.solve_gani(A, E, tol=1e-8)
    P = ctx.problem(A, lrfg.FULL, tol=1e-8, maxit=500)
    res, u = P.solve(E)
    assert res.converged and res.status == 0
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"]
    assert abs(res.iters - ref["iters"]) <= 1
    u_ref = np.real(fg.idft(ref["uh"], d))
    assert rel(u.full(), u_ref) <= 1e-6
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-13 * res.Aeff


def _oracle_op(a_terms, a_w, shape, rank, eps):
    return lr.LowRankGaNi(lr.tt_from_separable(a_terms, a_w), shape, fmt="tt", rank=rank, pinv_eps=eps)


@pytest.mark.parametrize("d,N,rank,rx", [(2, 15, 4, [3]), (3, 9, 3, [2, 3]), (3, 27, 5, [4, 4]), (2, 63, 6, [5])])
def test_tt_apply_and_rhs(ctx, d, N, rank, rx):
    shape = (N,) * d
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    op = _oracle_op(terms, w, shape, rank, 0.1)
    x = random_tt(shape, rx, seed=21)
    ref = np.real(lr.tt_full(lr.tt_idft(op.apply(lr.tt_dft(x)))))
    a_tt = lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w))
    P = ctx.problem(a_tt, lrfg.TT, rank=rank, pinv_eps=0.1)
    out = P.apply(ctx.field_from_tt(lrfg.TTensor.from_numpy(x))).full()
    assert rel(out, ref) <= 1e-7
    E = np.eye(d)[0]
    refb = np.real(lr.tt_full(lr.tt_idft(op.rhs(E))))
    assert rel(P.rhs(E).full(), refb) <= 1e-7


@pytest.mark.parametrize("d,N,rank,kind", [(2, 63, 10, "square"), (3, 15, 5, "square"), (3, 27, 6, "cube"),
                                           (2, 45, 8, "cube")])
def test_tt_solve_matches_oracle_minres(ctx, d, N, rank, kind):
    shape = (N,) * d
    if kind == "square":
        _, terms, w = square_inclusion(d, N)
    else:
        _, terms, w = smoothed_cube(d, N, contrast=20.0)
    E = np.eye(d)[0]
    op = _oracle_op(terms, w, shape, rank, 0.1)
    ref = lr.minres(op, E, maxit=60)
    P = ctx.problem(lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w)), lrfg.TT, rank=rank, pinv_eps=0.1,
                    tol=1e-10, maxit=60)
    res, u = P.solve(E)
    # A_eff is the compared quantity; the iteration at which the residual stops decreasing sits on a
    # plateau where rounding-level differences move it by a few steps without changing A_eff
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"]
    assert max(res.ranks) <= rank


def test_tt_laminate_is_harmonic_mean(ctx):
    d, N = 3, 81
    A, terms, w = laminate(d, N, contrast=10.0)
    f = A[:, 0, 0]
    harm = 1.0 / np.mean(1.0 / f)
    P = ctx.problem(lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w)), lrfg.TT, rank=3, tol=1e-12, maxit=200)
    res, _ = P.solve(np.eye(d)[0])
    assert abs(res.Aeff - harm) <= 1e-9 * harm


def test_tt_untruncated_equals_full(ctx):
    d, N = 3, 9
    A, terms, w = square_inclusion(d, N)
    E = np.eye(d)[0]
    full = fg.solve_gani(A, E, tol=1e-13)
    P = ctx.problem(lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w)), lrfg.TT, rank=N, tol=1e-11, maxit=400,
                    stop_on_increase=False)
    res, u = P.solve(E)
    assert abs(res.Aeff - full["Aeff"]) <= 1e-9 * full["Aeff"]
    # the field is unique up to a constant: P~^-1 (unlike P^-1) does not vanish at k = 0, so rounding noise
    # there can leave a tiny mean in the low-rank iterate; compare the zero-mean parts
    g = u.full()
    ref = np.real(fg.idft(full["uh"], d))
    assert rel(g - g.mean(), ref - ref.mean()) <= 1e-7


def test_full_coefficient_compressed_for_tt(ctx):
    d, N, rank = 3, 27, 6
    A = lognormal_grf(d, N, ell=0.25, seed=2)
    E = np.eye(d)[0]
    a_tt = lr.tt_svd(A, rmax=rank)
    op = lr.LowRankGaNi(a_tt, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.1)
    ref = lr.minres(op, E, maxit=40)
    P = ctx.problem(A, lrfg.TT, rank=rank, tol=1e-10, maxit=40)
    assert P.coeff_ranks() == lr.tt_ranks(a_tt)
    res, _ = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"]


def test_energy_bound_lowrank_above_full(ctx):
    d, N = 3, 27
    A, terms, w = smoothed_cube(d, N, contrast=10.0)
    E = np.eye(d)[0]
    Pf = ctx.problem(A, lrfg.FULL, tol=1e-10)
    full, _ = Pf.solve(E)
    prev = None
    for r in [2, 4, 8]:
        P = ctx.problem(lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w)), lrfg.TT, rank=r, maxit=80)
        res, _ = P.solve(E)
        assert res.Aeff >= full.Aeff * (1 - 1e-10)
        prev = res.Aeff
    assert prev - full.Aeff < 1e-2 * full.Aeff


@pytest.mark.parametrize("d,N", [(2, 31), (3, 9)])
def test_aeff_tensor_by_polarisation(ctx, d, N):
    """The homogenised tensor from d (d + 1) / 2 solves in lrfg_problem_aeff_tensor against the oracle's
    solves for the same E: the diagonal from E = e_a, the off-diagonal entries by polarisation."""
    A = lognormal_grf(d, N, ell=0.2, seed=5)
    P = ctx.problem(A, lrfg.FULL, tol=1e-10, maxit=2000)
    T, results = P.aeff_tensor(with_results=True)
    assert len(results) == d * (d + 1) // 2
    eye = np.eye(d)
    q = {(a, a): fg.solve_gani(A, eye[a], tol=1e-10)["Aeff"] for a in range(d)}
    for a in range(d):
        assert abs(T[a, a] - q[a, a]) <= 1e-8 * q[a, a]
        for b in range(a + 1, d):
            s = fg.solve_gani(A, eye[a] + eye[b], tol=1e-10)["Aeff"]
            assert abs(T[a, b] - 0.5 * (s - q[a, a] - q[b, b])) <= 1e-8 * q[a, a]
            assert T[a, b] == T[b, a]
    assert np.all(np.linalg.eigvalsh(T) > 0)
    # the same call straight through ctypes, without results
    from paper_1902_07455_gb300 import _lib as L
    import ctypes
    out = (ctypes.c_double * (d * d))()
    assert ctx.lib.lrfg_problem_aeff_tensor(P.h, out, None) == L.LRFG_OK
    assert np.array_equal(np.array(list(out)).reshape(d, d), T)
    P.free()
