"""Rows a3-a7 (Khatri–Rao Hadamard, sum, truncation, preconditioner, inner product) and the TT-SVD
compression: CUDA path vs the oracle on the same seeded inputs, compared as expanded full tensors
(carriages are gauge-dependent).

Tolerances (FP64): exact-arithmetic operations (Hadamard, sum, expand, dot) 1e-13 relative.  Truncation
computes the same TT-SVD truncation from (balanced) Gram matrices, whose singular vectors carry an error of
about eps * (sigma_1 / sigma_k)^2 / relgap; the test tensors keep sigma_1/sigma_k <= 1e2 and a relative gap
>= 0.3 at the cut, so we allow 1e-8 relative (Frobenius) on a truncated random tensor.  The exponential-sum
preconditioner output has a wider scale range (weights from 1e-6 to 10); an FP64 emulation of the same
Gram-SVD on these inputs deviates from QR+SVD rounding by up to 4e-9, so we allow 1e-7 there."""
import numpy as np
import pytest
import torch

import paper_1902_07455_gb300 as lrfg
from oracle import lowrank as lr
from synthetic import lognormal_grf, random_tt

pytestmark = pytest.mark.gpu


def T(cores):
    return lrfg.TTensor.from_numpy(cores)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("shape,rx,ry", [((5, 7, 9), [2, 3], [3, 2]), ((15, 13), [4], [3]), ((45, 27, 81), [5, 4], [3, 6])])
def test_hadamard_add_expand_dot(ctx, shape, rx, ry):
    x = random_tt(shape, rx, seed=1)
    y = random_tt(shape, ry, seed=2)
    X, Y = lr.tt_full(x), lr.tt_full(y)
    gx, gy = T(x), T(y)
    assert rel(ctx.tt_expand(gx).cpu().numpy(), X) <= 1e-13
    h = ctx.tt_hadamard(gx, gy)
    assert h.ranks == [1] + [a * b for a, b in zip(rx, ry)] + [1]
    assert rel(ctx.tt_expand(h).cpu().numpy(), lr.tt_full(lr.tt_hadamard(x, y))) <= 1e-13
    s = ctx.tt_add(0.7, gx, -1.3, gy)
    assert rel(ctx.tt_expand(s).cpu().numpy(), 0.7 * X - 1.3 * Y) <= 1e-13
    assert abs(ctx.tt_dot(gx, gy) - np.real(lr.tt_dot(x, y))) <= 1e-12 * np.linalg.norm(X) * np.linalg.norm(Y)


def _gapped(shape, big, small, seed, eps=1e-3):
    a = random_tt(shape, big, seed=seed)
    b = random_tt(shape, small, seed=seed + 100, scale=eps)
    return lr.tt_add(a, b)


@pytest.mark.parametrize("shape,big,small,rmax", [
    ((9, 11, 13), [3, 3], [4, 4], 3),
    ((45, 27, 63), [4, 5], [6, 6], 5),
    ((31, 17), [5], [7], 5),
    ((243, 81, 45), [6, 6], [10, 10], 6),
])
def test_round_matches_oracle(ctx, shape, big, small, rmax):
    x = _gapped(shape, big, small, seed=sum(shape))
    ref = lr.tt_full(lr.tt_round(x, rmax=rmax))
    got = ctx.tt_round(T(x), rmax)
    assert max(got.ranks) <= rmax
    G = ctx.tt_expand(got).cpu().numpy()
    assert rel(G, ref) <= 1e-8
    # left carriages orthonormal
    for c in got.cores[:-1]:
        M = c.reshape(-1, c.shape[2])
        I = (M.T @ M).cpu().numpy()
        assert np.abs(I - np.eye(I.shape[0])).max() <= 1e-8  # Gram-based factor: eps * cond(bond)^2


def test_round_without_truncation_and_rank_deficient(ctx):
    shape = (7, 9, 11)
    x = random_tt(shape, [3, 4], seed=3)
    y = lr.tt_add(x, x)  # rank 6/8 frame of a rank 3/4 tensor
    got = ctx.tt_round(T(y), 10)
    assert rel(ctx.tt_expand(got).cpu().numpy(), 2 * lr.tt_full(x)) <= 1e-10
    # rmax larger than any rank: exact
    got = ctx.tt_round(T(x), 50)
    assert rel(ctx.tt_expand(got).cpu().numpy(), lr.tt_full(x)) <= 1e-10


@pytest.mark.parametrize("shape,rx,rmax,eps", [((15, 13, 11), [2, 3], 4, 0.1), ((45, 45), [3], 6, 0.01),
                                               ((63, 27, 45), [3, 3], 8, 0.1)])
def test_precond_matches_oracle(ctx, shape, rx, rmax, eps):
    x = random_tt(shape, rx, seed=5)
    d = len(shape)
    ones = [[np.ones(n) for n in shape]]
    op = lr.LowRankGaNi(lr.tt_from_separable(ones), shape, fmt="tt", rank=rmax, pinv_eps=eps)
    ref_h = op.T(lr.tt_hadamard(op.Pinv, lr.tt_dft(x)))
    ref = np.real(lr.tt_full(lr.tt_idft(ref_h)))
    got = ctx.tt_expand(ctx.tt_precond(T(x), eps, rmax)).cpu().numpy()
    assert rel(got, ref) <= 1e-7
    assert d in (2, 3)


@pytest.mark.parametrize("d,N,rmax", [(2, 63, 8), (3, 27, 6), (3, 45, 10)])
def test_compress_matches_oracle(ctx, d, N, rmax):
    A = lognormal_grf(d, N, ell=0.2, seed=9)
    ref = lr.tt_full(lr.tt_svd(A, rmax=rmax))
    got = ctx.tt_compress(torch.as_tensor(A, device="cuda"), rmax)
    G = ctx.tt_expand(got).cpu().numpy()
    assert rel(G, ref) <= 1e-8
    assert rel(G, A) <= 0.05
