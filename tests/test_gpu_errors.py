"""Error behaviour of the C ABI on a GPU (host-side validation; nothing here faults a device)."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1902_07455_gb300 as lrfg
from paper_1902_07455_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def _status(fn):
    with pytest.raises(lrfg.LrfgError) as e:
        fn()
    return e.value.status


def test_even_grid_rejected(ctx):
    assert _status(lambda: ctx.problem(np.ones((8, 8)), lrfg.FULL)) == L.LRFG_EINVAL
    assert _status(lambda: ctx.field_from_full(np.ones((9, 10)))) == L.LRFG_EINVAL


def test_bad_rank_and_coefficients(ctx):
    assert _status(lambda: ctx.problem(np.ones((9, 9)), lrfg.TT, rank=0)) == L.LRFG_EINVAL
    a = np.ones((9, 9))
    a[3, 4] = np.nan
    assert _status(lambda: ctx.problem(a, lrfg.FULL)) == L.LRFG_EINVAL
    a[3, 4] = -1.0
    assert _status(lambda: ctx.problem(a, lrfg.FULL)) == L.LRFG_EINVAL
    assert _status(lambda: ctx.problem(np.ones((9, 9, 9, 9)), lrfg.FULL)) == L.LRFG_EINVAL


def test_mixed_precision_only_for_full_and_tt(ctx):
    lib = ctx.lib
    c = L.lrfg_coeff()
    arr = np.ones((9, 9))
    c.d, c.fmt, c.values, c.on_device = 2, L.LRFG_FULL, arr.ctypes.data, 0
    c.N[0] = c.N[1] = 9
    o = L.lrfg_opts()
    o.fmt, o.prec, o.rank, o.tol, o.maxit = L.LRFG_TUCKER, L.LRFG_MIXED, 1, 1e-8, 10
    h = C.c_void_p()
    assert lib.lrfg_problem_create(ctx.h, C.byref(c), C.byref(o), C.byref(h)) == L.LRFG_ENOTSUP
    assert b"LRFG_FULL" in lib.lrfg_last_error(ctx.h)
    o.prec = 7
    assert lib.lrfg_problem_create(ctx.h, C.byref(c), C.byref(o), C.byref(h)) == L.LRFG_EINVAL


def test_budget_exhaustion_is_enomem():
    small = lrfg.Context(0, budget=1 << 20)
    try:
        assert _status(lambda: small.problem(np.ones((63, 63, 63)), lrfg.FULL)) == L.LRFG_ENOMEM
    finally:
        small.close()


def test_iteration_cap_reports_noconv(ctx):
    from synthetic import square_inclusion
    A = square_inclusion(2, 63)[0]
    P = ctx.problem(A, lrfg.FULL, tol=1e-14, maxit=3)
    res, _ = P.solve([1.0, 0.0])
    assert res.status == L.LRFG_ENOCONV and not res.converged and res.iters == 3


def test_zero_macroscopic_field(ctx):
    from synthetic import square_inclusion
    A = square_inclusion(2, 15)[0]
    for fmt in (lrfg.FULL, lrfg.TT):
        P = ctx.problem(A, fmt, rank=3)
        res, _ = P.solve([0.0, 0.0])
        assert res.Aeff == 0.0
