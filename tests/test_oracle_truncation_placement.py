"""Pins of the parts of the low-rank oracle that the untruncated pins cannot see (CPU only).

1. Where the truncations sit.  Eq. (Pls_lowrank) truncates three times inside one application of the
   operator: the material product A~ e_a of every component, the divergence sum, and the product with
   P~^-1; the right-hand side truncates once, after P~^-1.  With every T the identity (the untruncated and
   laminate pins) a misplaced T changes nothing, so here the operator is recomputed by an independent
   route at ranks where every T cuts: every intermediate is a full grid, built with the full-format
   oracle's grad^, grad^*, F and F^-1 (Sec. 2.2.1) and, for Ga, its own injection, projection and modified
   coefficient (Sec. 2.2.3); P~^-1 is the exponential sum evaluated on k.k; and T is the TT-SVD of the
   expanded tensor (App. A.3.3) at the rank of the solution.  The TT rounding of any exact TT
   representation of a tensor is the TT-SVD of that tensor (both are the sequential truncated SVDs of the
   same unfoldings), so the two routes agree to rounding when the kept singular values are separated from
   the dropped ones, which random operands give.
2. The stopping rule of the minimal-residual iteration (Sec. 4.3): when the residual fails to decrease the
   iteration stops and returns the iterate with the smallest residual, not the last one.  A scripted
   operator makes the residual rise at the third step.
"""
import numpy as np
import pytest

from oracle import expsum
from oracle import fourier_galerkin as fg
from oracle import galerkin_exact as ge
from oracle import lowrank as lr
from synthetic import random_tt


def T_full(X, r):
    """T of a full tensor: its TT-SVD at rank r, expanded."""
    return lr.tt_full(lr.tt_svd(X, rmax=r))


def pinv_grid(shape, pinv_eps):
    """The exponential sum sum_m w_m exp(-t_m k.k) on the frequency grid."""
    xmax = float(sum(((n - 1) // 2) ** 2 for n in shape))
    t, w = expsum.expsum_inverse(xmax, pinv_eps)
    kk = np.sum(fg._kgrid(shape).astype(np.float64) ** 2, axis=0)
    return expsum.expsum_eval(kk, t, w)


def component(d, a, x):
    """A d-component field that is x in component a and zero elsewhere."""
    out = np.zeros((d,) + x.shape, dtype=np.complex128)
    out[a] = x
    return out


def gani_apply_full(a_full, vh, r, pinv_eps):
    """T P~^-1 T grad^* F T A~ F^-1 grad^ v with every intermediate on the full grid."""
    d = vh.ndim
    g = fg.grad_hat(vh)
    acc = np.zeros(vh.shape, dtype=np.complex128)
    for a in range(d):
        w = T_full(a_full * fg.idft(g[a], d), r)                 # T A~ e_a   (values)
        acc = acc + fg.div_hat(component(d, a, fg.dft(w, d)))   # grad^* F, summed over a
    s = T_full(acc, r)                                          # T after the sum
    return T_full(pinv_grid(vh.shape, pinv_eps) * s, r)          # T P~^-1


def gani_rhs_full(a_full, E, r, pinv_eps):
    """-T P~^-1 grad^* F A~ E on the full grid."""
    d = a_full.ndim
    ah = fg.dft(a_full.astype(np.complex128), d)
    acc = np.zeros(a_full.shape, dtype=np.complex128)
    for a in range(d):
        acc = acc + fg.div_hat(component(d, a, float(E[a]) * ah))
    return -T_full(pinv_grid(a_full.shape, pinv_eps) * acc, r)


def ga_apply_full(At, vh, r, pinv_eps, T=None):
    """T P~^-1 T grad^* I* F_M T A~ F_M^-1 I grad^ v on full grids (Ga, double grid M = 2N - 1); T: the
    truncation of a full tensor (default T_full)."""
    T = T or T_full
    d = vh.ndim
    N, M = vh.shape[0], At.shape[0]
    g = fg.grad_hat(vh)
    acc = np.zeros(vh.shape, dtype=np.complex128)
    for a in range(d):
        e = fg.idft(ge.inject(g[a], M, d), d)                   # gradient component on the double grid
        w = T(At * e, r)                                        # T A~ e_a there
        acc = acc + fg.div_hat(component(d, a, ge.project(fg.dft(w, d), N, d)))
    s = T(acc, r)
    return T(pinv_grid(vh.shape, pinv_eps) * s, r)


def ga_rhs_full(At, E, N, r, pinv_eps, T=None):
    T = T or T_full
    d = At.ndim
    ah = ge.project(fg.dft(At.astype(np.complex128), d), N, d)
    acc = np.zeros((N,) * d, dtype=np.complex128)
    for a in range(d):
        acc = acc + fg.div_hat(component(d, a, float(E[a]) * ah))
    return -T(pinv_grid((N,) * d, pinv_eps) * acc, r)


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


CASES = [(2, 9, 3, 2), (2, 15, 3, 3), (3, 7, 2, 2)]  # d, N, coefficient rank, solution rank


def _operands(d, N, ra, seed):
    a_tt = random_tt((N,) * d, [ra] * (d - 1), seed=seed)
    a_tt[0] = a_tt[0] + 3.0  # keep the coefficient away from zero (not needed by the algebra, just tidy)
    v = random_tt((N,) * d, [3] * (d - 1), seed=seed + 1)
    vh = [np.asarray(G, dtype=np.complex128) for G in v]
    return a_tt, vh


@pytest.mark.parametrize("d,N,ra,r", CASES)
def test_gani_apply_truncations_where_eq_pls_lowrank_puts_them(d, N, ra, r):
    a_tt, vh = _operands(d, N, ra, 11 + d + N)
    op = lr.LowRankGaNi(a_tt, (N,) * d, fmt="tt", rank=r, pinv_eps=0.1)
    got = lr.tt_full(op.apply(vh))
    ref = gani_apply_full(lr.tt_full(a_tt), lr.tt_full(vh), r, 0.1)
    assert rel(got, ref) <= 1e-11, rel(got, ref)
    # every T cuts: the untruncated operator is far from the truncated one
    untr = gani_apply_full(lr.tt_full(a_tt), lr.tt_full(vh), None, 0.1)
    assert rel(untr, ref) > 1e-3


@pytest.mark.parametrize("d,N,ra,r", CASES)
def test_gani_rhs_truncation_after_the_preconditioner(d, N, ra, r):
    a_tt, _ = _operands(d, N, ra, 31 + d + N)
    E = np.array([1.0, -0.5, 0.25][:d])
    op = lr.LowRankGaNi(a_tt, (N,) * d, fmt="tt", rank=r, pinv_eps=0.1)
    got = lr.tt_full(op.rhs(E))
    ref = gani_rhs_full(lr.tt_full(a_tt), E, r, 0.1)
    assert rel(got, ref) <= 1e-11, rel(got, ref)
    assert rel(gani_rhs_full(lr.tt_full(a_tt), E, None, 0.1), ref) > 1e-3


@pytest.mark.parametrize("d,N,ra,r", [(2, 9, 2, 2), (2, 13, 3, 3), (3, 7, 2, 2)])
def test_ga_tt_apply_and_rhs_by_full_grids(d, N, ra, r):
    a_tt, vh = _operands(d, N, ra, 51 + d + N)
    a_pix = np.real(lr.tt_full(a_tt))
    At = ge.ga_coefficient(a_pix)
    op = lr.LowRankGaTT(a_tt, (N,) * d, rank=r, pinv_eps=0.1)
    got = lr.tt_full(op.apply(vh))
    ref = ga_apply_full(At, lr.tt_full(vh), r, 0.1)
    assert rel(got, ref) <= 1e-11, rel(got, ref)
    E = np.array([1.0, 0.5, -0.25][:d])
    got_b = lr.tt_full(op.rhs(E))
    ref_b = ga_rhs_full(At, E, N, r, 0.1)
    assert rel(got_b, ref_b) <= 1e-11, rel(got_b, ref_b)


# ---- the stopping rule ----------------------------------------------------------------------------
class ScriptedOperator:
    """A small SPD operator on full-rank TTs (d = 2, N = 3, so no truncation loses anything) whose T is the
    identity except on one scripted call, where it scales its argument up; A_eff is replaced by a marker
    that identifies the iterate it is evaluated on."""

    def __init__(self, bump_call, factor=100.0):
        rng = np.random.Generator(np.random.PCG64(7))
        Q, _ = np.linalg.qr(rng.standard_normal((9, 9)))
        self.C = Q @ np.diag(np.linspace(1.0, 4.0, 9)) @ Q.T
        self.b = rng.standard_normal(9)
        self.f = lr.FORMATS["tt"]
        self.shape = (3, 3)
        self.calls = 0
        self.bump_call = bump_call
        self.factor = factor

    def _tt(self, x):
        return [np.asarray(G, dtype=np.complex128) for G in lr.tt_svd(np.asarray(x).reshape(3, 3))]

    def _vec(self, x):
        return lr.tt_full(x).reshape(9)

    def rhs(self, E):
        return self._tt(self.b)

    def apply(self, x):
        return self._tt(self.C @ self._vec(x))

    def T(self, x):
        self.calls += 1
        y = self._vec(x)
        return self._tt(self.factor * y if self.calls == self.bump_call else y)

    def homogenised_coefficient(self, uh, E):
        return float(np.real(np.sum(self._vec(uh) * np.arange(1, 10))))


def minres_stop_pin(minres=None):
    """Residuals 1 > r_1 > r_2 < r_3: the iteration must stop there and return u_2 (and its A_eff)."""
    minres = minres or lr.minres
    # T calls: u_1, r_1, u_2, r_2, u_3, r_3 -> the sixth truncation (the residual of u_3) is scaled up
    op = ScriptedOperator(bump_call=6)
    seen = {}
    out = minres(op, np.zeros(2), tol=1e-14, maxit=20, callback=lambda it, u, nr: seen.setdefault(it, (u, nr)))
    h = out["history"]
    assert len(h) == 4 and h[1] < h[0] and h[2] < h[1] and h[3] > h[2], h
    assert out["iters"] == 2
    assert out["rel_resid"] == h[2]
    u2 = seen[2][0]
    assert np.array_equal(lr.tt_full(out["u"]), lr.tt_full(u2))
    assert out["Aeff"] == op.homogenised_coefficient(u2, None)


def test_minres_returns_the_best_iterate_when_the_residual_rises():
    minres_stop_pin()


def test_minres_without_the_rise_runs_on():
    # the same operator without the scripted bump decreases monotonically and stops only at maxit
    op = ScriptedOperator(bump_call=-1)
    out = lr.minres(op, np.zeros(2), tol=1e-14, maxit=5)
    assert out["iters"] == 5 and all(b < a for a, b in zip(out["history"], out["history"][1:]))


def test_minres_patience_continues_past_one_rise():
    """stop_on_increase = k > 1: the iteration survives fewer than k consecutive failures to decrease and returns the
    best iterate seen; after the scripted rise at step 3 the next steps improve on step 2 again."""
    # a residual scaled by 3 at step 3: a rise, then the next steps (an overshot step, then recovery) pass below
    # step 2's residual within the patience
    op = ScriptedOperator(bump_call=6, factor=3.0)
    out = lr.minres(op, np.zeros(2), tol=1e-14, maxit=8, stop_on_increase=3)
    h = out["history"]
    assert h[3] > h[2]
    assert out["iters"] > 3 and out["rel_resid"] < h[2]
    assert out["rel_resid"] == min(h)
    # patience 1 is the paper's rule: stop at the first rise
    one = lr.minres(ScriptedOperator(bump_call=6, factor=3.0), np.zeros(2), tol=1e-14, maxit=8, stop_on_increase=1)
    assert one["iters"] == 2


def T_hosvd(X, r):
    """T of a full tensor in Tucker format: its truncated HOSVD at multilinear rank r (App. A.2.3), expanded."""
    return lr.tucker_full(*lr.tucker_hosvd(X, rmax=r))


@pytest.mark.parametrize("d,N,ra,r", [(2, 9, 2, 2), (3, 7, 2, 2)])
def test_ga_tucker_apply_and_rhs_by_full_grids(d, N, ra, r):
    """Ga in Tucker format against the full-grid route with T the truncated HOSVD of the expanded tensor:
    the Tucker truncation (QR of the factors, HOSVD of the core) of any exact Tucker form of a tensor is the
    truncated HOSVD of that tensor."""
    a_tt, vh = _operands(d, N, ra, 71 + d + N)
    a_pix = np.real(lr.tt_full(a_tt))
    a_tk = lr.tucker_hosvd(a_pix)  # exact Tucker form of the pixel values
    v_tk = lr.tucker_hosvd(lr.tt_full(vh))
    At = ge.ga_coefficient(a_pix)
    op = lr.LowRankGa(a_tk, (N,) * d, rank=r, pinv_eps=0.1, fmt="tucker")
    got = lr.tucker_full(*op.apply(v_tk))
    ref = ga_apply_full(At, lr.tt_full(vh), r, 0.1, T=T_hosvd)
    assert rel(got, ref) <= 1e-11, rel(got, ref)
    E = np.array([1.0, 0.5, -0.25][:d])
    got_b = lr.tucker_full(*op.rhs(E))
    ref_b = ga_rhs_full(At, E, N, r, 0.1, T=T_hosvd)
    assert rel(got_b, ref_b) <= 1e-11, rel(got_b, ref_b)
    assert rel(ga_apply_full(At, lr.tt_full(vh), None, 0.1, T=T_hosvd), ref) > 1e-3  # every T cuts
