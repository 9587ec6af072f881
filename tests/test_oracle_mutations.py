"""Planted mistakes in the oracle (on the CPU only): each plausible error must fail at least one pin.

Each case monkeypatches one oracle function with a typical slip (a sign, a dropped term or weight, a
transposed index, a wrong frequency order) and checks that the named pin from the other oracle tests
now fails.  This shows that the pins constrain the oracle rather than echo it.
"""
import numpy as np
import pytest

from oracle import fourier_galerkin as fg
from oracle import lowrank as lr

import tests.test_oracle_full as tf
import tests.test_oracle_lowrank as tl


def _must_fail(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_sign_of_gradient(monkeypatch):
    orig = fg.grad_hat
    monkeypatch.setattr(fg, "grad_hat", lambda uh: -orig(uh))
    _must_fail(tf.test_gradient_matches_closed_form_differentiation, 9)


def test_sign_of_right_hand_side(monkeypatch):
    # (a sign flip inside div_hat alone is harmless: it negates both sides of the system)
    orig = fg.gani_rhs
    monkeypatch.setattr(fg, "gani_rhs", lambda A, E: -orig(A, E))
    _must_fail(tf.test_pcg_matches_dense_direct_solve, 2, 9, "sq")


def test_missing_cell_average_weight(monkeypatch):
    def bad(uh, A, E):
        E = np.asarray(E, dtype=np.float64)
        d = E.shape[0]
        e = np.real(fg.idft(fg.grad_hat(uh), d))
        f = e + E.reshape((d,) + (1,) * d)
        return float(np.sum(A * np.sum(f * f, axis=0)))  # sum instead of the cell average
    monkeypatch.setattr(fg, "homogenised_coefficient", bad)
    _must_fail(tf.test_constant_coefficient_exact, 2, 15)


def test_unwrapped_frequencies(monkeypatch):
    monkeypatch.setattr(fg, "frequencies", lambda N: np.arange(N, dtype=np.int64))
    _must_fail(tf.test_gradient_matches_closed_form_differentiation, 9)


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_dropped_preconditioner_zero_mode(monkeypatch):
    """Keeping k = 0 in P^-1 (1/(k.k) with k.k := 1 there) lets a mean into u, which the dense solve
    (zero-mean minimiser) rejects through the field pin."""
    def bad(shape):
        K = fg._kgrid(shape)
        kk = np.sum(K.astype(np.float64) ** 2, axis=0)
        kk[(0,) * len(shape)] = 1.0
        return 1.0 / kk
    monkeypatch.setattr(fg, "precond_inv", bad)
    orig_rhs = fg.gani_rhs

    def rhs_with_mean(A, E):  # a k = 0 component, which the exact pseudo-inverse annihilates
        b = orig_rhs(A, E)
        b[(0,) * b.ndim] += 1e-3
        return b
    monkeypatch.setattr(fg, "gani_rhs", rhs_with_mean)
    _must_fail(tf.test_pcg_matches_dense_direct_solve, 2, 9, "sq")


def test_transposed_khatri_rao(monkeypatch):
    def bad(x, y):
        out = []
        for G, H in zip(x, y):
            a, n, b = G.shape
            c, _, e = H.shape
            out.append(np.einsum("inj,knl->iknlj", G, H).reshape(a * c, n, b * e))  # rank pair swapped
        return out
    monkeypatch.setattr(lr.FORMATS["tt"], "had", bad)
    _must_fail(tl.test_format_ops_match_full, "tt", (5, 7, 9))


def test_dropped_cross_term_in_lowrank_aeff(monkeypatch):
    def bad(self, uh, E):
        f = self.f
        size = float(np.prod(self.shape))
        ones = f.sep([[np.ones(n) for n in self.shape]])
        val = float(np.dot(E, E)) * np.real(f.dot(ones, self.a)) / size
        for a in range(self.d):
            e = f.idft(f.mmul(uh, a, 2j * np.pi * self.K[a]))
            val += np.real(f.dot(e, f.had(self.a, e))) / size  # 2 E.<a, e> term dropped
        return float(val)
    monkeypatch.setattr(lr.LowRankGaNi, "homogenised_coefficient", bad)
    _must_fail(tl.test_untruncated_lowrank_equals_full, "tt", 2, 15)


def test_wrong_minres_step(monkeypatch):
    """omega = ||r||^2 / ||C r||^2 instead of (C r, r) / ||C r||^2: a classic slip."""
    def bad_minres(op, E, tol=1e-10, maxit=200, stop_on_increase=True, callback=None):
        f = op.f
        b = op.rhs(np.asarray(E, dtype=np.float64))
        u = f.zeros(op.shape)
        for _ in range(maxit):
            r = op.T(f.add(b, f.scale(op.apply(u), -1.0)))
            q = op.apply(r)
            omega = np.real(f.dot(r, r)) / np.real(f.dot(q, q))
            u = op.T(f.add(u, f.scale(r, omega)))
        return dict(u=u, iters=maxit, rel_resid=0.0, history=[], Aeff=op.homogenised_coefficient(u, E))
    monkeypatch.setattr(lr, "minres", bad_minres)
    _must_fail(tl.test_untruncated_lowrank_equals_full, "tt", 2, 15)


# ---- planted mistakes in the oracle's extensions (Ga, anisotropy, tolerance truncation, rank adaptation)
import tests.test_oracle_ga as tg  # noqa: E402
from oracle import galerkin_exact as ga  # noqa: E402


def test_ga_cell_sinc_with_the_wrong_width(monkeypatch):
    """s(m) of a cell of width 2/N instead of 1/N: the quadrature pin of the modified coefficient fails."""
    def bad(m, N):
        m = np.asarray(m, dtype=np.float64)
        out = np.full(m.shape, 2.0 / N)
        nz = m != 0
        out[nz] = np.sin(2.0 * np.pi * m[nz] / N) / (np.pi * m[nz])
        return out
    monkeypatch.setattr(ga, "_sinc_cell", bad)
    _must_fail(tg.test_coefficient_matches_quadrature_of_the_dirichlet_kernel)


def test_ga_injection_without_wrapping(monkeypatch):
    """Negative frequencies placed at their N-grid storage index on the double grid: the dense Galerkin pin
    fails."""
    def bad(vh, M, d):
        N = vh.shape[-1]
        out = np.zeros(vh.shape[:-d] + (M,) * d, dtype=np.complex128)
        idx = np.ix_(*([np.arange(N)] * d))
        out[(Ellipsis,) + idx] = vh
        return out
    monkeypatch.setattr(ga, "inject", bad)
    with pytest.raises((AssertionError, ZeroDivisionError)):  # a wrong (here singular) operator
        tg.test_ga_solve_matches_dense_galerkin(5, 1)


def test_ga_aeff_on_the_grid_instead_of_the_double_grid(monkeypatch):
    """A_eff by the rectangle rule of the grid (the GaNi formula) instead of the exact double-grid sum."""
    monkeypatch.setattr(ga, "homogenised_coefficient_ga",
                        lambda uh, At, E: fg.homogenised_coefficient(uh, np.full(uh.shape, At.sum()), E))
    _must_fail(tg.test_ga_solve_matches_dense_galerkin, 5, 1)


def test_anisotropic_part_with_the_wrong_sign(monkeypatch):
    """a e_a - sum_b B_ab e_b in the low-rank material product: untruncated low rank no longer equals the
    full-format tensor solve."""
    orig = lr.LowRankGaNi.apply

    def bad(self, vh):
        self.B = -self.B
        try:
            return orig(self, vh)
        finally:
            self.B = -self.B
    monkeypatch.setattr(lr.LowRankGaNi, "apply", bad)
    _must_fail(tl.test_untruncated_anisotropic_lowrank_equals_full, "tt", 2, 15)


def test_tolerance_not_split_over_the_bonds(monkeypatch):
    """tol per TT bond instead of tol / sqrt(d - 1): the first-bond rank pin fails."""
    orig = lr.tt_round
    monkeypatch.setattr(lr, "tt_round", lambda x, rmax=None, tol=None: orig(
        x, rmax=rmax, tol=None if tol is None else tol * np.sqrt(max(len(x) - 1, 1))))
    monkeypatch.setitem(lr.FORMATS["tt"].__dict__, "round", lr.tt_round)
    _must_fail(tl.test_tolerance_truncation_bound_and_first_rank, "tt")


def test_rank_adaptation_without_rebuilding_the_rhs(monkeypatch):
    """The right-hand side kept at the starting rank after a raise: the untruncated pin (A_eff of the full
    solve) fails."""
    orig_rhs = lr.LowRankGaNi.rhs
    cache = {}

    def frozen(self, E):
        key = id(self)
        if key not in cache:
            cache[key] = orig_rhs(self, E)
        return cache[key]
    monkeypatch.setattr(lr.LowRankGaNi, "rhs", frozen)
    _must_fail(tl.test_rank_adaptive_minres_pins)


# ---- planted mistakes in the placement of the truncations and in the stopping rule ------------------
import tests.test_oracle_truncation_placement as tp  # noqa: E402


def _gani_apply_variant(drop_sum_T=False, T_before_material=False, T_before_pinv=False):
    def apply(self, vh):
        f = self.f
        acc = None
        for a in range(self.d):
            e = f.idft(f.mmul(vh, a, 2j * np.pi * self.K[a]))
            w = f.had(self.a, self.T(e)) if T_before_material else self.T(f.had(self.a, e))
            term = f.mmul(f.dft(w), a, -2j * np.pi * self.K[a])
            acc = term if acc is None else f.add(acc, term)
        s = acc if drop_sum_T else self.T(acc)
        return f.had(self.Pinv, self.T(s)) if T_before_pinv else self.T(f.had(self.Pinv, s))
    return apply


@pytest.mark.parametrize("variant", [dict(drop_sum_T=True), dict(T_before_material=True),
                                     dict(T_before_pinv=True)])
def test_misplaced_truncation_in_the_operator(monkeypatch, variant):
    monkeypatch.setattr(lr.LowRankGaNi, "apply", _gani_apply_variant(**variant))
    _must_fail(tp.test_gani_apply_truncations_where_eq_pls_lowrank_puts_them, 3, 7, 2, 2)


def test_right_hand_side_truncated_before_the_preconditioner(monkeypatch):
    def bad(self, E):
        f = self.f
        ah = f.dft(self.a)
        acc = None
        for a in range(self.d):
            term = f.mmul(f.scale(ah, float(E[a])), a, -2j * np.pi * self.K[a])
            acc = term if acc is None else f.add(acc, term)
        return f.scale(f.had(self.Pinv, self.T(acc)), -1.0)
    monkeypatch.setattr(lr.LowRankGaNi, "rhs", bad)
    _must_fail(tp.test_gani_rhs_truncation_after_the_preconditioner, 2, 15, 3, 3)


def test_ga_tt_without_the_truncation_on_the_double_grid(monkeypatch):
    def bad(self, vh):
        f = self.f
        acc = None
        for a in range(self.d):
            w = f.had(self.At, self._grad_double(vh, a))      # T dropped
            term = f.mmul(self._project(f.dft(w)), a, -2j * np.pi * self.K[a])
            acc = term if acc is None else f.add(acc, term)
        return self.T(f.had(self.Pinv, self.T(acc)))
    monkeypatch.setattr(lr.LowRankGaTT, "apply", bad)
    _must_fail(tp.test_ga_tt_apply_and_rhs_by_full_grids, 2, 9, 2, 2)


def test_minres_returning_the_last_iterate():
    """The iteration stops when the residual rises but hands back the last iterate, not the best."""
    def bad_minres(op, E, tol=1e-10, maxit=200, stop_on_increase=True, callback=None):
        f = op.f
        b = op.rhs(E)
        nb = f.norm(b)
        u, hist, it, best = f.zeros(op.shape), [], 0, np.inf
        while True:
            r = op.T(f.add(b, f.scale(op.apply(u), -1.0))) if it > 0 else b
            nr = f.norm(r) / nb
            hist.append(nr)
            if callback is not None:
                callback(it, u, nr)
            if nr >= best or nr <= tol or it >= maxit:
                break
            best = nr
            q = op.apply(r)
            omega = np.real(f.dot(q, r)) / np.real(f.dot(q, q))
            u = op.T(f.add(u, f.scale(r, omega))) if it > 0 else op.T(f.scale(r, omega))
            it += 1
        return dict(u=u, iters=it, rel_resid=nr, history=hist, Aeff=op.homogenised_coefficient(u, E))
    _must_fail(tp.minres_stop_pin, bad_minres)


# ---- planted mistakes in the randomised rounding ------------------------------------------------------
import tests.test_oracle_sketch as tsk  # noqa: E402
from oracle import sketch as sk_mod  # noqa: E402


def _bad_round_sketch(carry=True, final=True, right_sweep_from_left=False):
    def bad(y, omega, rmax=None, tol=None):
        d = len(y)
        W = [None] * d
        W[d - 1] = np.ones((1, 1))
        for j in range(d - 1, 0, -1):
            src = y[d - j] if right_sweep_from_left and y[d - j].shape == y[j].shape else y[j]
            W[j - 1] = np.einsum("anb,bm,lnm->al", src, W[j], omega[j], optimize=True)
        x = [np.array(G, copy=True) for G in y]
        for j in range(d - 1):
            a, n, b = x[j].shape
            X = x[j].reshape(a * n, b)
            Q, _ = np.linalg.qr(X @ W[j])
            M = Q.conj().T @ X
            x[j] = Q.reshape(a, n, Q.shape[1])
            if carry:
                x[j + 1] = np.tensordot(M, x[j + 1], axes=([1], [0]))
            else:
                x[j + 1] = np.tensordot(np.eye(Q.shape[1], b), x[j + 1], axes=([1], [0]))
        return lr.tt_truncate_left_orth(x, rmax=rmax, tol=tol) if final else x
    return bad


@pytest.mark.parametrize("variant", [dict(carry=False), dict(final=False)])
def test_randomised_rounding_slips(monkeypatch, variant):
    monkeypatch.setattr(sk_mod, "tt_round_sketch", _bad_round_sketch(**variant))
    _must_fail(tsk.test_exact_when_the_sketch_covers_the_ranks, (7, 9, 11), [4, 5], 6, 3)


@pytest.mark.parametrize("variant", ["plain_ones", "no_b_in_aeff"])
def test_ga_anisotropy_slips(monkeypatch, variant):
    """Low-rank Ga with B: the anisotropic part multiplied by the grid's plain ones instead of the modified
    coefficient of 1, or left out of A_eff."""
    import tests.test_oracle_ga as tg
    orig_init = lr.LowRankGa.__init__
    if variant == "plain_ones":
        def init(self, *args, **kw):
            orig_init(self, *args, **kw)
            self.Ones = self.f.sep([[np.ones(2 * n - 1) for n in self.shape]])
        monkeypatch.setattr(lr.LowRankGa, "__init__", init)
    else:
        orig_aeff = lr.LowRankGa.homogenised_coefficient

        def aeff(self, uh, E):
            B, self.B = self.B, None
            try:
                return orig_aeff(self, uh, E)
            finally:
                self.B = B
        monkeypatch.setattr(lr.LowRankGa, "homogenised_coefficient", aeff)
    _must_fail(tg.test_untruncated_lowrank_ga_with_anisotropy_matches_dense_galerkin, "tt", 5)


def _bad_truncate_left_orth(variant):
    def bad(x, rmax=None, tol=None):
        d = len(x)
        if variant == "from_the_left":
            return lr.tt_round(x, rmax=rmax, tol=tol)
        G = [g.copy() for g in x]
        loc_tol = None if tol is None else (tol if variant == "tol_not_split" else tol / np.sqrt(max(d - 1, 1)))
        for j in range(d - 1, 0, -1):
            a, n, b = G[j].shape
            U, s, Vt = np.linalg.svd(G[j].reshape(a, n * b), full_matrices=False)
            k = lr._keep(s, rmax, loc_tol)
            G[j] = Vt[:k].reshape(k, n, b)
            carry = U[:, :k] if variant == "no_singular_values" else U[:, :k] * s[:k]
            G[j - 1] = np.tensordot(G[j - 1], carry, axes=([2], [0]))
        return G
    return bad


@pytest.mark.parametrize("variant", ["from_the_left", "no_singular_values"])
def test_truncation_from_the_right_slips(monkeypatch, variant):
    """The truncation that ends the randomised rounding: swept from the left instead, or carrying U without the
    singular values into the carriage on the left."""
    monkeypatch.setattr(lr, "tt_truncate_left_orth", _bad_truncate_left_orth(variant))
    _must_fail(tsk.test_right_to_left_rounding_is_the_mirrored_rounding, (7, 9, 11), [4, 5], 3, None)
    if variant == "no_singular_values":
        _must_fail(tsk.test_right_to_left_rounding_at_one_bond_is_eckart_young)


# ---- planted mistakes in the exponential sum and the Tucker / CP truncations ------------------------------------
import oracle.expsum as es_mod  # noqa: E402


def test_expsum_weights_off_by_a_factor(monkeypatch):
    """The sinc-quadrature weights h e^tau with h taken from the wrong step (a 5% larger h in the weights)."""
    orig = es_mod.expsum_inverse

    def bad(xmax, eps):
        t, w = orig(xmax, eps)
        return t, 1.05 * w
    monkeypatch.setattr(es_mod, "expsum_inverse", bad)
    _must_fail(tl.test_expsum_inverse_accuracy, 63, 2, 1e-2)


def test_cp_truncation_without_its_weights(monkeypatch):
    """App. A.1.3 with the weights c left out of the SVD of R1 diag(c) R2^T (reading 10)."""
    def bad(x, rmax=None, tol=None):
        c, B1, B2 = x
        Q1, R1 = np.linalg.qr(B1)
        Q2, R2 = np.linalg.qr(B2)
        U, s, Vt = np.linalg.svd(R1 @ R2.T, full_matrices=False)
        k = lr._keep(s, rmax, tol)
        return s[:k], Q1 @ U[:, :k], Q2 @ Vt[:k].T
    monkeypatch.setattr(lr, "cp_round", bad)
    _must_fail(tl.test_cp_truncation_is_eckart_young)


def test_hosvd_with_the_wrong_unfolding(monkeypatch):
    """HOSVD factors from the tensor reshaped row-major to N_j x (rest) instead of unfolded along mode j."""
    def bad(A, rmax=None, tol=None):
        d = A.ndim
        factors = []
        loc_tol = None if tol is None else tol / np.sqrt(d)
        for j in range(d):
            M = A.reshape(A.shape[j], -1)
            U, s, _ = np.linalg.svd(M, full_matrices=False)
            factors.append(U[:, :lr._keep(s, rmax, loc_tol)])
        core = A
        for j, B in enumerate(factors):
            core = np.moveaxis(np.tensordot(B.conj().T, core, axes=([1], [j])), 0, j)
        return core, factors
    monkeypatch.setattr(lr, "tucker_hosvd", bad)
    _must_fail(tl.test_tt_svd_and_hosvd_error_bounds)


def test_truncation_from_the_right_with_the_tolerance_not_split(monkeypatch):
    """The truncation from the right with the whole tolerance at every bond instead of tol / sqrt(d - 1)."""
    monkeypatch.setattr(lr, "tt_truncate_left_orth", _bad_truncate_left_orth("tol_not_split"))
    _must_fail(tsk.test_truncation_from_the_right_keeps_the_tolerance_bound)
