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
    for kw in (dict(fmt=lrfg.TT, rank=3), dict(fmt=lrfg.FULL, prec=lrfg.MIXED)):
        fmt = kw.pop("fmt")
        with pytest.raises(lrfg.LrfgError) as e:
            ctx.problem(a, fmt, disc=lrfg.GA, **kw)
        assert e.value.status == 6
