"""Fourier-Galerkin with exact integration (Ga, Sec. 2.2.3) in full format on the GPU against the Ga oracle
(``oracle.galerkin_exact``, pinned by a dense Galerkin solve and quadrature) on the same seeded pixel
materials.  Tolerances: one preconditioned application and the right-hand side 1e-11 (FFT chains on the grid
and the double grid), A_eff after a solve to residual 1e-10: 1e-9; closed forms 1e-12."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import fourier_galerkin as fg
from oracle import galerkin_exact as ga
from synthetic import lognormal_grf, random_field, square_inclusion

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("d,N", [(2, 13), (2, 25), (3, 13)])
def test_ga_apply_and_rhs(ctx, d, N):
    a = random_field((N,) * d, seed=N)
    At = ga.ga_coefficient(a)
    u = np.random.default_rng(2).standard_normal((N,) * d)
    P = ctx.problem(a, lrfg.FULL, disc=lrfg.GA)
    out = P.apply(ctx.field_from_full(u)).full()
    Pinv = fg.precond_inv((N,) * d)
    ref = np.real(fg.idft(Pinv * ga.ga_operator(fg.dft(u, d), At), d))
    assert rel(out, ref) <= 1e-11
    E = np.arange(1.0, d + 1.0)
    b = P.rhs(E).full()
    refb = np.real(fg.idft(Pinv * ga.ga_rhs(At, E, N), d))
    assert rel(b, refb) <= 1e-11


@pytest.mark.parametrize("d,N,kind", [(2, 63, "square"), (2, 81, "grf"), (3, 13, "square"), (3, 25, "grf")])
def test_ga_solve(ctx, d, N, kind):
    a = square_inclusion(d, N)[0] if kind == "square" else lognormal_grf(d, N, ell=0.2, seed=7)
    E = np.eye(d)[0]
    ref = ga.solve_ga(a, E, tol=1e-11, maxit=3000)
    res, u = ctx.problem(a, lrfg.FULL, disc=lrfg.GA, tol=1e-10, maxit=3000).solve(E)
    assert res.converged
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-9 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    assert rel(u.full(), np.real(fg.idft(ref["uh"], d))) <= 1e-7
    # exact integration is a Galerkin method: its A_eff lies above GaNi's limit behaviour only through the
    # discretisation; both must lie within the Voigt-Reuss bounds of the pixel material
    assert 1.0 / np.mean(1.0 / a) <= res.Aeff <= np.mean(a)


def test_ga_closed_forms(ctx):
    N = 25
    f = 1.0 + 9.0 * (np.abs(fg.grid_points(N)) < 0.25)
    lam = np.outer(f, np.ones(N))
    r, _ = ctx.problem(lam, lrfg.FULL, disc=lrfg.GA, tol=1e-12).solve([0.0, 1.0], want_field=False)
    assert abs(r.Aeff - lam.mean()) <= 1e-12 * lam.mean()  # along the layers: the mean
    B = np.array([[5.5, -4.5], [-4.5, 5.5]])
    E = np.array([1.0, 2.0])
    c = np.full((N, N), 2.0)
    r, _ = ctx.problem(c, lrfg.FULL, disc=lrfg.GA, B=B, tol=1e-12).solve(E, want_field=False)
    ref = float(E @ (2.0 * np.eye(2) + B) @ E)
    assert abs(r.Aeff - ref) <= 1e-12 * ref  # constant A = 2 I + B: A_eff = E.A E


def test_ga_not_supported(ctx):
    a = random_field((45, 45), seed=1)  # double grid 89: prime
    with pytest.raises(lrfg.LrfgError) as e:
        ctx.problem(a, lrfg.FULL, disc=lrfg.GA)
    assert e.value.status == 6
    a = random_field((13, 13), seed=1)
    for kw in (dict(fmt=lrfg.FULL, prec=lrfg.MIXED), dict(fmt=lrfg.TT, rank=3, prec=lrfg.MIXED)):
        fmt = kw.pop("fmt")
        with pytest.raises(lrfg.LrfgError) as e:
            ctx.problem(a, fmt, disc=lrfg.GA, **kw)
        assert e.value.status == 6


# ---- Ga in TT format (the low-rank Ga of the paper's timing study) ------------------------------------
from oracle import lowrank as lr  # noqa: E402
from synthetic import random_tt, smoothed_cube  # noqa: E402


@pytest.mark.parametrize("d,N,rank,rx", [(2, 13, 4, [3]), (3, 13, 3, [2, 3]), (2, 25, 6, [4])])
def test_tt_ga_apply_and_rhs(ctx, d, N, rank, rx):
    shape = (N,) * d
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    a_tt = lr.tt_from_separable(terms, w)
    op = lr.LowRankGaTT(a_tt, shape, rank=rank, pinv_eps=0.1)
    x = random_tt(shape, rx, seed=21)
    ref = np.real(lr.tt_full(lr.tt_idft(op.apply(lr.tt_dft(x)))))
    P = ctx.problem(lrfg.TTensor.from_numpy(a_tt), lrfg.TT, rank=rank, pinv_eps=0.1, disc=lrfg.GA)
    out = P.apply(ctx.field_from_tt(lrfg.TTensor.from_numpy(x))).full()
    assert rel(out, ref) <= 1e-7
    E = np.eye(d)[0]
    refb = np.real(lr.tt_full(lr.tt_idft(op.rhs(E))))
    assert rel(P.rhs(E).full(), refb) <= 1e-7


@pytest.mark.parametrize("d,N,rank", [(2, 25, 8), (3, 13, 5)])
def test_tt_ga_solve(ctx, d, N, rank):
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    a_tt = lr.tt_from_separable(terms, w)
    E = np.eye(d)[0]
    ref = lr.minres(lr.LowRankGaTT(a_tt, (N,) * d, rank=rank, pinv_eps=0.1), E, tol=1e-10, maxit=40)
    P = ctx.problem(lrfg.TTensor.from_numpy(a_tt), lrfg.TT, rank=rank, tol=1e-10, maxit=40, disc=lrfg.GA)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-12 * res.Aeff


def test_untruncated_tt_ga_equals_full_ga(ctx):
    d, N = 2, 13
    a, terms, w = square_inclusion(d, N)
    E = np.eye(d)[0]
    full, _ = ctx.problem(a, lrfg.FULL, disc=lrfg.GA, tol=1e-12, maxit=3000).solve(E, want_field=False)
    tt, _ = ctx.problem(lrfg.TTensor.from_numpy(lr.tt_from_separable(terms, w)), lrfg.TT, rank=N, tol=1e-12,
                        maxit=400, stop_on_increase=False, disc=lrfg.GA).solve(E, want_field=False)
    assert abs(tt.Aeff - full.Aeff) <= 1e-9 * full.Aeff


# ---- Ga in Tucker and CP format -------------------------------------------------------------------------
def _random_tucker(shape, ranks, seed):
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(ranks))
    factors = [rng.standard_normal((n, r)) / np.sqrt(n) for n, r in zip(shape, ranks)]
    return core, factors


def _tucker_coeff(fmt, terms, w):
    """The coefficient's exact Tucker form, and the oracle's form of the same format."""
    tk = lr.tucker_from_separable(terms, w)
    return tk, (tk if fmt == "tucker" else lr.cp_from_separable(terms, w))


@pytest.mark.parametrize("fmt,d,N,rank,rx", [("tucker", 2, 13, 4, (3, 3)), ("tucker", 3, 13, 3, (3, 2, 3)),
                                             ("cp", 2, 25, 5, (4, 4))])
def test_tucker_cp_ga_apply_and_rhs(ctx, fmt, d, N, rank, rx):
    shape = (N,) * d
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    tk, a_lr = _tucker_coeff(fmt, terms, w)
    op = lr.LowRankGa(a_lr, shape, rank=rank, pinv_eps=0.1, fmt=fmt)
    core, factors = _random_tucker(shape, rx, seed=23)
    if fmt == "tucker":
        ref = np.real(lr.tucker_full(*lr.tucker_idft(op.apply(lr.tucker_dft((core, factors))))))
        refb = np.real(lr.tucker_full(*lr.tucker_idft(op.rhs(np.eye(d)[0]))))
    else:  # a rank-r CP operand: the Tucker input with a diagonal core
        core = np.diag(np.diag(core))
        cp = (np.diag(core).copy(), factors[0], factors[1])
        ref = np.real(lr.cp_full(lr.cp_idft(op.apply(lr.cp_dft(cp)))))
        refb = np.real(lr.cp_full(lr.cp_idft(op.rhs(np.eye(d)[0]))))
    P = ctx.problem(lrfg.TuckerTensor.from_numpy(*tk), lrfg.TUCKER if fmt == "tucker" else lrfg.CP, rank=rank,
                    pinv_eps=0.1, disc=lrfg.GA)
    out = P.apply(ctx.field_from_tucker(lrfg.TuckerTensor.from_numpy(core, factors))).full()
    # the Tucker operator's bound (its P~^-1 product's collinear factors; see test_gpu_tucker)
    assert rel(out, ref) <= 1e-6
    assert rel(P.rhs(np.eye(d)[0]).full(), refb) <= 1e-7


@pytest.mark.parametrize("fmt,d,N,rank", [("tucker", 2, 25, 6), ("tucker", 3, 13, 4), ("cp", 2, 25, 6)])
def test_tucker_cp_ga_solve(ctx, fmt, d, N, rank):
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    tk, a_lr = _tucker_coeff(fmt, terms, w)
    E = np.eye(d)[0]
    ref = lr.minres(lr.LowRankGa(a_lr, (N,) * d, rank=rank, pinv_eps=0.1, fmt=fmt), E, tol=1e-10, maxit=40)
    P = ctx.problem(lrfg.TuckerTensor.from_numpy(*tk), lrfg.TUCKER if fmt == "tucker" else lrfg.CP, rank=rank,
                    tol=1e-10, maxit=40, disc=lrfg.GA)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-12 * res.Aeff


@pytest.mark.parametrize("fmt", ["tucker", "cp"])
def test_untruncated_tucker_cp_ga_equals_full_ga(ctx, fmt):
    d, N = 2, 13
    a, terms, w = square_inclusion(d, N)
    E = np.eye(d)[0]
    full, _ = ctx.problem(a, lrfg.FULL, disc=lrfg.GA, tol=1e-12, maxit=3000).solve(E, want_field=False)
    tk = lr.tucker_from_separable(terms, w)
    lo, _ = ctx.problem(lrfg.TuckerTensor.from_numpy(*tk), lrfg.TUCKER if fmt == "tucker" else lrfg.CP, rank=N,
                        tol=1e-12, maxit=400, stop_on_increase=False, disc=lrfg.GA).solve(E, want_field=False)
    assert abs(lo.Aeff - full.Aeff) <= 1e-9 * full.Aeff


# ---- low-rank Ga with a constant anisotropic part (A~ = a~ I + B 1~) ---------------------------------------
B2 = np.array([[0.7, 0.25], [0.25, 0.4]])
B3 = np.array([[0.6, 0.2, 0.0], [0.2, 0.5, 0.1], [0.0, 0.1, 0.3]])


def _lowrank_coeff(fmt, terms, w):
    if fmt == "tt":
        t = lr.tt_from_separable(terms, w)
        return t, t, lrfg.TTensor.from_numpy(t), lrfg.TT
    tk, a_lr = _tucker_coeff(fmt, terms, w)
    return tk, a_lr, lrfg.TuckerTensor.from_numpy(*tk), (lrfg.TUCKER if fmt == "tucker" else lrfg.CP)


@pytest.mark.parametrize("fmt,d,N,rank", [("tt", 2, 13, 4), ("tt", 3, 13, 3), ("tucker", 3, 13, 3), ("cp", 2, 13, 4)])
def test_lowrank_ga_anisotropic_apply_and_rhs(ctx, fmt, d, N, rank):
    shape = (N,) * d
    B = B2 if d == 2 else B3
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    _, a_lr, coeff, code = _lowrank_coeff(fmt, terms, w)
    op = lr.LowRankGa(a_lr, shape, rank=rank, pinv_eps=0.1, fmt=fmt, B=B)
    P = ctx.problem(coeff, code, rank=rank, pinv_eps=0.1, disc=lrfg.GA, B=B)
    E = np.eye(d)[0]
    if fmt == "tt":
        x = random_tt(shape, [3] * (d - 1), seed=25)
        ref = np.real(lr.tt_full(lr.tt_idft(op.apply(lr.tt_dft(x)))))
        out = P.apply(ctx.field_from_tt(lrfg.TTensor.from_numpy(x))).full()
        refb = np.real(lr.tt_full(lr.tt_idft(op.rhs(E))))
        tol = 1e-7
    else:
        core, factors = _random_tucker(shape, (3,) * d, seed=25)
        if fmt == "cp":
            core = np.diag(np.diag(core))
            cp = (np.diag(core).copy(), factors[0], factors[1])
            ref = np.real(lr.cp_full(lr.cp_idft(op.apply(lr.cp_dft(cp)))))
            refb = np.real(lr.cp_full(lr.cp_idft(op.rhs(E))))
        else:
            ref = np.real(lr.tucker_full(*lr.tucker_idft(op.apply(lr.tucker_dft((core, factors))))))
            refb = np.real(lr.tucker_full(*lr.tucker_idft(op.rhs(E))))
        out = P.apply(ctx.field_from_tucker(lrfg.TuckerTensor.from_numpy(core, factors))).full()
        tol = 1e-6  # the Tucker operator's bound (collinear P~^-1 factors)
    assert rel(out, ref) <= tol
    assert rel(P.rhs(E).full(), refb) <= 1e-7


@pytest.mark.parametrize("fmt,d,N,rank", [("tt", 2, 25, 6), ("tt", 3, 13, 4), ("tucker", 3, 13, 4), ("cp", 2, 25, 6)])
def test_lowrank_ga_anisotropic_solve(ctx, fmt, d, N, rank):
    B = B2 if d == 2 else B3
    _, terms, w = smoothed_cube(d, N, contrast=10.0)
    _, a_lr, coeff, code = _lowrank_coeff(fmt, terms, w)
    E = np.eye(d)[0]
    ref = lr.minres(lr.LowRankGa(a_lr, (N,) * d, rank=rank, pinv_eps=0.1, fmt=fmt, B=B), E, tol=1e-10, maxit=40)
    P = ctx.problem(coeff, code, rank=rank, tol=1e-10, maxit=40, disc=lrfg.GA, B=B)
    res, u = P.solve(E)
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-6 * ref["Aeff"], (res.Aeff, ref["Aeff"])
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-12 * res.Aeff


@pytest.mark.parametrize("fmt", ["tt", "tucker"])
def test_untruncated_lowrank_ga_anisotropic_equals_full_ga(ctx, fmt):
    d, N = 2, 13
    a, terms, w = square_inclusion(d, N)
    E = np.array([1.0, 0.5])
    full, _ = ctx.problem(a, lrfg.FULL, disc=lrfg.GA, tol=1e-12, maxit=3000, B=B2).solve(E, want_field=False)
    _, _, coeff, code = _lowrank_coeff(fmt, terms, w)
    # rank 2N - 1: no truncation on the double grid either
    lo, _ = ctx.problem(coeff, code, rank=2 * N - 1, tol=1e-12, maxit=400, stop_on_increase=False, disc=lrfg.GA,
                        B=B2).solve(E, want_field=False)
    assert abs(lo.Aeff - full.Aeff) <= 1e-9 * full.Aeff


def test_full_ga_anisotropic_matches_dense_galerkin(ctx):
    """Full-format Ga with a constant anisotropic part against the dense Galerkin solve of the anisotropic
    material assembled from quadrature (the closed form of a constant material above cannot see how B is
    weighted against the double-grid product: there the fluctuation vanishes)."""
    import tests.test_oracle_ga as tg
    d, N = 2, 13
    a, _, _ = square_inclusion(d, N)
    for E in (np.array([1.0, 0.5]), np.array([0.0, 1.0])):
        ref = tg.dense_galerkin(a, E, B2)
        r, _ = ctx.problem(a, lrfg.FULL, disc=lrfg.GA, tol=1e-12, maxit=3000, B=B2).solve(E, want_field=False)
        assert abs(r.Aeff - ref) <= 1e-9 * ref, (r.Aeff, ref)
