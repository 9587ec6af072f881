"""Pins of the oracle's randomised TT rounding (oracle/sketch.py) and of its use in the operator (CPU only).

* SplitMix64 reproduces the published first outputs of stream 0.
* When the input's TT ranks do not exceed the sketch ranks, the sketch spans every unfolding exactly and the
  randomised rounding equals the deterministic TT rounding of App. A.3.3 (expanded, to rounding).
* Above that, it is near-optimal: its error stays within a small factor of the deterministic rounding's
  (the probabilistic bound of the randomised range finder with oversampling), and its output is
  left-orthonormal with the requested ranks.
* In the operator of Eq. (Pls_lowrank): with product ranks below the sketch ranks the sketched operator and
  right-hand side equal the deterministic ones, and a minimal-residual solve with the sketched rounding
  reaches the deterministic solve's A_eff.
"""
import numpy as np
import pytest

from oracle import lowrank as lr
from oracle import sketch as sk
from synthetic import random_tt, smoothed_cube


def test_splitmix64_published_outputs():
    # first three outputs of SplitMix64 seeded with 0 (the reference implementation's test values)
    v = sk.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sketch_entries_are_rademacher_and_reproducible():
    om = sk.sketch_tt((9, 11, 13), 7, seed=5)
    assert [G.shape for G in om] == [(1, 9, 7), (7, 11, 7), (7, 13, 1)]
    allv = np.concatenate([G.ravel() for G in om])
    assert set(np.unique(allv)) == {-1.0, 1.0}
    assert abs(allv.mean()) < 0.1
    again = sk.sketch_tt((9, 11, 13), 7, seed=5)
    assert all(np.array_equal(a, b) for a, b in zip(om, again))
    other = sk.sketch_tt((9, 11, 13), 7, seed=6)
    assert not np.array_equal(om[1], other[1])


def _rel(x, y):
    return np.linalg.norm(lr.tt_full(x) - lr.tt_full(y)) / np.linalg.norm(lr.tt_full(y))


@pytest.mark.parametrize("shape,ranks,ell,rmax", [((9, 11), [5], 7, 3), ((7, 9, 11), [4, 5], 6, 3),
                                                  ((7, 9, 11), [4, 5], 5, 5)])
def test_exact_when_the_sketch_covers_the_ranks(shape, ranks, ell, rmax):
    y = random_tt(shape, ranks, seed=3)
    om = sk.sketch_tt(shape, ell, seed=19)
    got = sk.tt_round_sketch(y, om, rmax=rmax)
    ref = lr.tt_round_rl(y, rmax=rmax)
    # (a bond where the tensor's rank is below rmax may carry zero singular values on either side)
    assert all(r <= rmax for r in lr.tt_ranks(got))
    assert _rel(got, ref) <= 1e-11


def test_near_optimal_above_the_sketch_ranks():
    # a Khatri-Rao product of rank 6 x 6 = 36 (the kind of tensor the solver rounds) truncated to rank 6
    shape = (15, 17, 19)
    x = random_tt(shape, [6, 6], seed=1)
    y = random_tt(shape, [6, 6], seed=2)
    z = lr.tt_hadamard(x, y)
    ref = lr.tt_round(z, rmax=6)
    e_det = _rel(ref, z)
    for seed in range(4):
        got = sk.tt_round_sketch(z, sk.sketch_tt(shape, 6 + 8, seed=seed), rmax=6)
        assert lr.tt_ranks(got) == [1, 6, 6, 1]
        e = _rel(got, z)
        assert e <= 1.5 * e_det, (e, e_det)
        for G in got[1:]:  # right-orthonormal carriages after the truncation from the right
            a, n, b = G.shape
            M = G.reshape(a, n * b)
            assert np.allclose(M @ M.T, np.eye(a), atol=1e-12)


def test_sketch_with_tolerance_keeps_the_bound():
    shape = (13, 15, 17)
    z = lr.tt_hadamard(random_tt(shape, [5, 5], seed=7), random_tt(shape, [5, 5], seed=8))
    tol = 0.05
    got = sk.tt_round_sketch(z, sk.sketch_tt(shape, 30, seed=1), rmax=20, tol=tol)
    assert _rel(got, z) <= tol * 1.0001
    assert max(lr.tt_ranks(got)) <= 20


def _ops(d, N, rank, over):
    _, terms, w = smoothed_cube(d, N, contrast=10.0, full=False)
    a = lr.tt_from_separable(terms, w)
    det = lr.LowRankGaNi(a, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.3)
    skt = lr.LowRankGaNi(a, (N,) * d, fmt="tt", rank=rank, pinv_eps=0.3, sketch=(over, 11))
    return det, skt


def test_sketched_operator_equals_deterministic_when_the_sketch_covers_the_products():
    # coefficient rank 2, operand rank 2: material products of rank 4, P~^-1 products of rank R * 2, all
    # below the sketch ranks rank + p, so every sketched T is the deterministic one
    det, skt = _ops(2, 15, rank=2, over=40)
    v = [np.asarray(G, dtype=np.complex128) for G in random_tt((15, 15), [2], seed=4)]
    assert _rel(skt.apply(v), det.apply(v)) <= 1e-10
    E = np.array([1.0, 0.0])
    assert _rel(skt.rhs(E), det.rhs(E)) <= 1e-10


def test_sketched_minres_reaches_the_deterministic_aeff():
    det, skt = _ops(2, 31, rank=6, over=8)
    E = np.array([1.0, 0.0])
    a = lr.minres(det, E, maxit=40)
    b = lr.minres(skt, E, maxit=40)
    assert abs(a["Aeff"] - b["Aeff"]) <= 1e-5 * a["Aeff"], (a["Aeff"], b["Aeff"])


def test_kept_sketch_rank_is_the_sketch_projection():
    # final=False returns the rank-l left-orthonormal projection of the sketch: its deterministic rounding to r is
    # the full randomised rounding, and with ranks covered it reproduces the input
    shape = (9, 11, 13)
    y = random_tt(shape, [4, 5], seed=3)
    om = sk.sketch_tt(shape, 7, seed=2)
    kept = sk.tt_round_sketch(y, om, rmax=3, final=False)
    assert lr.tt_ranks(kept)[1:-1] == [7, 7] or max(lr.tt_ranks(kept)) <= 7
    assert _rel(kept, y) <= 1e-12
    assert _rel(lr.tt_truncate_left_orth(kept, rmax=3), sk.tt_round_sketch(y, om, rmax=3)) <= 1e-12
    for G in kept[:-1]:
        a, n, b = G.shape
        M = G.reshape(a * n, b)
        assert np.allclose(M.T @ M, np.eye(b), atol=1e-12)


# ---- the truncation from the right that ends the randomised rounding -------------------------------------------
def _mirror(x):
    """The same tensor with its modes in reverse order: carriage j of the mirror is carriage d-1-j transposed."""
    return [G.transpose(2, 1, 0).copy() for G in reversed(x)]


@pytest.mark.parametrize("shape,ranks,rmax,tol", [((7, 9, 11), [4, 5], 3, None), ((9, 8, 10), [6, 7], 4, None),
                                                  ((11, 13), [6], 3, None), ((8, 9, 10), [6, 6], 6, 0.2)])
def test_right_to_left_rounding_is_the_mirrored_rounding(shape, ranks, rmax, tol):
    # rounding from the left of the mirrored tensor, mirrored back, is rounding from the right: every SVD sees
    # the same unfolding in the same order (App. A.3.3 with the modes read backwards)
    y = random_tt(shape, ranks, seed=11)
    got = lr.tt_round_rl(y, rmax=rmax, tol=tol)
    ref = _mirror(lr.tt_round(_mirror(y), rmax=rmax, tol=tol))
    assert lr.tt_ranks(got) == lr.tt_ranks(ref)
    assert _rel(got, ref) <= 1e-11


def test_right_to_left_rounding_at_one_bond_is_eckart_young():
    # ranks [4, 5] rounded to 4: only the last bond loses rank, and the first SVD from the right sees the exact
    # unfolding (N0 N1) x N2, so the result is its best rank-4 approximation (Eckart-Young), from the SVD of the
    # full matrix; the first bond then has rank <= 4 already and is left as it is
    shape = (7, 9, 11)
    y = random_tt(shape, [4, 5], seed=12)
    A = lr.tt_full(y)
    U, s, Vt = np.linalg.svd(A.reshape(-1, shape[2]), full_matrices=False)
    best = ((U[:, :4] * s[:4]) @ Vt[:4]).reshape(shape)
    got = lr.tt_round_rl(y, rmax=4)
    assert lr.tt_ranks(got) == [1, 4, 4, 1]
    assert np.linalg.norm(lr.tt_full(got) - best) / np.linalg.norm(best) <= 1e-12


def test_truncation_from_the_right_keeps_the_tolerance_bound():
    shape = (12, 13, 14)
    z = lr.tt_hadamard(random_tt(shape, [4, 4], seed=21), random_tt(shape, [4, 4], seed=22))
    for tol in (0.3, 0.1, 0.01):
        got = lr.tt_round_rl(z, tol=tol)
        assert _rel(got, z) <= tol * (1 + 1e-12)
    # and it is quasi-optimal at a fixed rank: within sqrt(d-1) of the best error of each unfolding combined
    got = lr.tt_round_rl(z, rmax=5)
    A = lr.tt_full(z)
    tails = []
    for j in range(1, 3):
        s = np.linalg.svd(A.reshape(int(np.prod(shape[:j])), -1), compute_uv=False)
        tails.append(np.sum(s[5:] ** 2))
    assert np.linalg.norm(lr.tt_full(got) - A) ** 2 <= sum(tails) * (1 + 1e-9)


def test_right_to_left_rounding_leaves_right_orthonormal_carriages():
    # after the truncations from the right, carriages 1..d-1 have orthonormal rows (their SVD factors V^*) and the
    # first carriage carries the norm
    z = lr.tt_hadamard(random_tt((9, 10, 11), [4, 4], seed=31), random_tt((9, 10, 11), [3, 4], seed=32))
    got = lr.tt_round_rl(z, rmax=6)
    for G in got[1:]:
        a, n, b = G.shape
        M = G.reshape(a, n * b)
        assert np.abs(M @ M.T - np.eye(a)).max() <= 1e-13
    assert abs(np.linalg.norm(got[0]) - np.linalg.norm(lr.tt_full(got))) <= 1e-12 * np.linalg.norm(got[0])
