"""Anisotropic coefficients A~(x) = a(x) I + B (the modified materials of Sec. 4.4, B constant symmetric
positive semidefinite) on the GPU against the oracle's tensor-coefficient path (full format) and its
anisotropic low-rank operator, on the same seeded inputs.  Tolerances as for the isotropic path: one full
application 1e-11 (FFT chain), one TT application 1e-7 (five truncations), A_eff after a solve 1e-6 (the
FP64-path target)."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import fourier_galerkin as fg
from oracle import lowrank as lr
from synthetic import lognormal_grf, random_tt, smoothed_cube, square_inclusion

pytestmark = pytest.mark.gpu

# the anisotropic parts printed in Sec. 4.4 (eigenvalues (1, 10) and (1, 5, 10))
B2 = np.array([[5.5, -4.5], [-4.5, 5.5]])
B3 = np.array([[4.25, -3.25, -1.25 * np.sqrt(2.0)], [-3.25, 4.25, 1.25 * np.sqrt(2.0)],
               [-1.25 * np.sqrt(2.0), 1.25 * np.sqrt(2.0), 7.5]])


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def tensor_field(a, B):
    d = a.ndim
    return a[None, None] * np.eye(d).reshape((d, d) + (1,) * d) + B.reshape((d, d) + (1,) * d)


@pytest.mark.parametrize("d,N", [(2, 45), (3, 15)])
def test_full_apply_and_rhs_aniso(ctx, d, N):
    a = lognormal_grf(d, N, ell=0.2, seed=13)
    B = B2 if d == 2 else B3
    At = tensor_field(a, B)
    u = np.random.default_rng(1).standard_normal((N,) * d)
    P = ctx.problem(a, lrfg.FULL, B=B)
    out = P.apply(ctx.field_from_full(u)).full()
    Pinv = fg.precond_inv((N,) * d)
    ref = np.real(fg.idft(Pinv * fg.gani_operator(fg.dft(u, d), At), d))
    assert rel(out, ref) <= 1e-11
    E = np.ones(d)
    b = P.rhs(E).full()
    refb = np.real(fg.idft(Pinv * fg.gani_rhs(At, E), d))
    assert rel(b, refb) <= 1e-11


@pytest.mark.parametrize("d,N,prec", [(2, 63, lrfg.FP64), (3, 27, lrfg.FP64), (3, 27, lrfg.MIXED)])
def test_full_solve_aniso(ctx, d, N, prec):
    a = square_inclusion(d, N)[0]
    B = B2 if d == 2 else B3
    E = np.ones(d)
    ref = fg.solve_gani(tensor_field(a, B), E, tol=1e-10, maxit=3000)
    tol = 1e-8 if prec == lrfg.FP64 else 1e-5
    P = ctx.problem(a, lrfg.FULL, tol=tol, maxit=3000, prec=prec, B=B)
    res, u = P.solve(E)
    assert res.converged
    assert abs(res.Aeff - ref["Aeff"]) <= (1e-6 if prec == lrfg.FP64 else 1e-4) * ref["Aeff"]
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-13 * res.Aeff


@pytest.mark.parametrize("d,N,rank,rx", [(2, 15, 4, [3]), (3, 9, 3, [2, 3]), (3, 27, 5, [4, 4])])
def test_tt_apply_aniso(ctx, d, N, rank, rx):
    shape = (N,) * d
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    B = B2 if d == 2 else B3
    op = lr.LowRankGaNi(lr.tt_from_separable(terms, w), shape, fmt="tt", rank=rank, pinv_eps=0.1, B=B)
    x = random_tt(shape, rx, seed=21)
    ref = np.real(lr.tt_full(lr.tt_idft(op.apply(lr.tt_dft(x)))))
    P = ctx.problem(lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w)), lrfg.TT, rank=rank, B=B)
    out = P.apply(ctx.field_from_tt(lrfg.TTensor.from_numpy(x))).full()
    assert rel(out, ref) <= 1e-7


@pytest.mark.parametrize("d,N,rank", [(2, 31, 8), (3, 15, 6)])
def test_tt_solve_aniso(ctx, d, N, rank):
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    B = B2 if d == 2 else B3
    E = np.ones(d)
    a_tt = lr.tt_from_separable(terms, w)
    op = lr.LowRankGaNi(a_tt, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.1, B=B)
    ref = lr.minres(op, E, tol=1e-10, maxit=60)
    P = ctx.problem(lrfg.TTensor.from_numpy(a_tt), lrfg.TT, rank=rank, tol=1e-10, maxit=60, B=B)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    assert abs(res.iters - ref["iters"]) <= 2
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-12 * res.Aeff


def test_untruncated_tt_aniso_equals_full(ctx):
    d, N = 2, 15
    A, terms, w = square_inclusion(d, N)
    E = np.ones(d)
    full = fg.solve_gani(tensor_field(A, B2), E, tol=1e-12, maxit=3000)
    P = ctx.problem(lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w)), lrfg.TT, rank=N, tol=1e-12, maxit=400,
                    stop_on_increase=False, B=B2)
    res, _ = P.solve(E)
    assert abs(res.Aeff - full["Aeff"]) <= 1e-9 * full["Aeff"]


def test_zero_b_is_isotropic_bitwise(ctx):
    a = square_inclusion(2, 31)[0]
    r0, _ = ctx.problem(a, lrfg.FULL, tol=1e-8).solve([1.0, 0.0], want_field=False)
    r1, _ = ctx.problem(a, lrfg.FULL, tol=1e-8, B=np.zeros((2, 2))).solve([1.0, 0.0], want_field=False)
    assert r0.Aeff == r1.Aeff and r0.iters == r1.iters


def test_b_validation(ctx):
    a = square_inclusion(2, 15)[0]
    with pytest.raises(lrfg.LrfgError) as e:
        ctx.problem(a, lrfg.FULL, B=np.array([[1.0, 0.5], [0.0, 1.0]]))  # not symmetric
    assert e.value.status == 1 and "symmetric" in str(e.value)
    with pytest.raises(lrfg.LrfgError) as e:
        ctx.problem(a, lrfg.FULL, B=np.array([[1.0, 2.0], [2.0, 1.0]]))  # eigenvalue -1
    assert e.value.status == 1 and "semidefinite" in str(e.value)


@pytest.mark.parametrize("fmt,d,N,rank", [("tucker", 2, 31, 6), ("tucker", 3, 15, 4), ("cp", 2, 31, 6)])
def test_tucker_cp_aniso(ctx, fmt, d, N, rank):
    """Tucker and CP (d = 2, the Tucker path) with the anisotropic part: one application and a solve
    against the oracle's anisotropic operator in that format."""
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    B = B2 if d == 2 else B3
    shape = (N,) * d
    a_tk = lr.tucker_from_separable(terms, w)
    okfmt = "tucker" if fmt == "tucker" else "cp"
    a_or = lr.FORMATS[okfmt].sep(terms, w)
    op = lr.LowRankGaNi(a_or, shape, fmt=okfmt, rank=rank, pinv_eps=0.1, B=B)
    E = np.ones(d)
    ref = lr.minres(op, E, tol=1e-10, maxit=40)
    P = ctx.problem(lrfg.TuckerTensor.from_numpy(*a_tk), lrfg.TUCKER if fmt == "tucker" else lrfg.CP, rank=rank,
                    tol=1e-10, maxit=40, B=B)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-12 * res.Aeff
    if fmt == "tucker":
        rng = np.random.default_rng(4)
        core = rng.standard_normal((3,) * d)
        facs = [rng.standard_normal((N, 3)) / np.sqrt(N) for _ in range(d)]
        x = (core, facs)
        refx = np.real(lr.tucker_full(*lr.tucker_idft(op.apply(lr.tucker_dft(x)))))
        out = P.apply(ctx.field_from_tucker(lrfg.TuckerTensor.from_numpy(core, facs))).full()
        assert rel(out, refx) <= 1e-7
