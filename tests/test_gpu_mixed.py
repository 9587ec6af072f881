"""LRFG_MIXED on the FULL path (FP32 vectors, coefficient and FFTs; FP64 inner products, step lengths,
residual test and A_eff) against the FP64 oracle on the same seeded inputs.

Tolerances, from FP32 unit roundoff u = 2^-24 = 6e-8:
- one operator application is a chain of 2d FFT passes of O(log N) depth, pointwise products with the
  coefficient and the Fourier multipliers: its error is a few u log2(N) times the operator's norm, so
  1e-5 relative (2-norm) bounds it at every size here with a margin of ~10;
- a solve run to a relative preconditioned residual of 1e-5: the field is within kappa * 1e-5 of the
  discrete solution, kappa <= the phase contrast (10), so 2e-4 relative; A_eff is stationary at the
  solution (its error is quadratic in the field error, Sec. 2.4) and is evaluated in FP64 from the
  FP64-converted field, so 1e-5 relative."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from oracle import fourier_galerkin as fg
from synthetic import lognormal_grf, square_inclusion

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("d,N", [(2, 15), (2, 63), (2, 81), (2, 243), (3, 9), (3, 27), (3, 45), (3, 81)])
def test_mixed_apply_and_rhs(ctx, d, N):
    A = lognormal_grf(d, N, ell=0.2, seed=13)
    u = np.random.default_rng(1).standard_normal((N,) * d)
    P = ctx.problem(A, lrfg.FULL, prec=lrfg.MIXED)
    out = P.apply(ctx.field_from_full(u)).full()
    Pinv = fg.precond_inv((N,) * d)
    ref = np.real(fg.idft(Pinv * fg.gani_operator(fg.dft(u, d), A), d))
    assert rel(out, ref) <= 1e-5
    assert rel(out, ref) >= 1e-12  # it really ran in FP32
    E = np.eye(d)[1]
    refb = np.real(fg.idft(Pinv * fg.gani_rhs(A, E), d))
    assert rel(P.rhs(E).full(), refb) <= 1e-5


@pytest.mark.parametrize("d,N,kind", [(2, 63, "square"), (3, 27, "square"), (3, 45, "grf"), (2, 125, "grf")])
def test_mixed_solve(ctx, d, N, kind):
    A = square_inclusion(d, N)[0] if kind == "square" else lognormal_grf(d, N, ell=0.2, seed=3)
    E = np.eye(d)[0]
    ref = fg.solve_gani(A, E, tol=1e-10)
    P = ctx.problem(A, lrfg.FULL, tol=1e-5, maxit=500, prec=lrfg.MIXED)
    res, u = P.solve(E)
    assert res.converged and res.rel_resid <= 1e-5
    assert abs(res.Aeff - ref["Aeff"]) <= 1e-5 * ref["Aeff"]
    u_ref = np.real(fg.idft(ref["uh"], d))
    assert rel(u.full(), u_ref) <= 2e-4
    # the field handed out is FP64: A_eff of it through the FP64 evaluation agrees to rounding
    assert abs(P.aeff(E, u) - res.Aeff) <= 1e-13 * res.Aeff


def test_mixed_and_fp64_same_iterate_count(ctx):
    A = lognormal_grf(3, 27, ell=0.2, seed=5)
    E = [0.0, 0.0, 1.0]
    r64, _ = ctx.problem(A, lrfg.FULL, tol=1e-5, maxit=500).solve(E, want_field=False)
    r32, _ = ctx.problem(A, lrfg.FULL, tol=1e-5, maxit=500, prec=lrfg.MIXED).solve(E, want_field=False)
    assert abs(r32.iters - r64.iters) <= 1
    assert abs(r32.Aeff - r64.Aeff) <= 1e-5 * r64.Aeff
