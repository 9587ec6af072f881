"""The TT path at N = 1215 per axis (1.8e9 grid points, which the oracle cannot hold): pins that hold at
any size.

- Laminate a = a(x_1): for odd N the GaNi solution is exact for E along the layering normal and
  tangent, A_eff,11 = harmonic mean and A_eff,22 = arithmetic mean of the samples a(x_k1) (closed forms;
  the field is of TT rank 1, so truncation is exact).  Tolerance 1e-9 relative (FP64 MinRes to 1e-12).
- tanh-smoothed cube of contrast 100 (coefficient rank 2), TT rank 10: A_eff lies between the Reuss and
  Voigt bounds of the grid samples (harmonic and arithmetic means), and the low-rank A_eff is an upper
  bound of the full one, so it must not fall below the Reuss bound."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg
from synthetic import laminate, smoothed_cube

pytestmark = pytest.mark.gpu
N = 1215


def _tt_from_terms(terms):
    return [lrfg.TTensor.from_numpy([np.asarray(f, dtype=np.float64).reshape(1, N, 1) for f in t]) for t in terms]


def test_laminate_1215_closed_forms(ctx):
    _, terms, _ = laminate(3, N, contrast=10.0, full=False)
    f = terms[0][0]
    harm, arith = 1.0 / np.mean(1.0 / f), np.mean(f)
    a_tt = _tt_from_terms(terms)[0]
    P = ctx.problem(a_tt, lrfg.TT, rank=3, tol=1e-12, maxit=200)
    r1, _ = P.solve([1.0, 0.0, 0.0], want_field=False)
    assert abs(r1.Aeff - harm) <= 1e-9 * harm
    r2, _ = P.solve([0.0, 1.0, 0.0], want_field=False)
    assert abs(r2.Aeff - arith) <= 1e-9 * arith


def test_smoothed_cube_1215_within_bounds(ctx):
    contrast = 100.0
    _, terms, w = smoothed_cube(3, N, contrast=contrast, full=False)
    t1, t2 = _tt_from_terms(terms)
    a_tt = ctx.tt_add(w[0], t1, w[1], t2)
    assert a_tt.ranks == [1, 2, 2, 1]
    h = terms[1][0]
    voigt = 1.0 + (contrast - 1.0) * float(np.mean(h)) ** 3
    hh = np.outer(h, h)
    reuss = 1.0 / (sum(float(np.sum(1.0 / (1.0 + (contrast - 1.0) * h[i] * hh))) for i in range(N)) / float(N) ** 3)
    P = ctx.problem(a_tt, lrfg.TT, rank=10, tol=1e-12, maxit=60)
    res, _ = P.solve([1.0, 0.0, 0.0], want_field=False)
    assert reuss <= res.Aeff <= voigt
