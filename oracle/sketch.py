"""Randomised TT rounding (sketch, then orthogonalise) — FP64 oracle, test infrastructure only.

The paper truncates with the deterministic TT rounding of App. A.3.3 (QR sweep, then truncated SVDs), whose
cost grows like N s^3 in the input rank s; after the material product (s = r_A r) and the exponential-sum
preconditioner (s = R r) it is the dominant cost of one application of Eq. (Pls_lowrank).  The randomised
rounding "randomize-then-orthogonalize" of Al Daas, Ballard, Cazeaux, Hallman, Miedlar, Pasha, Reid and
Saibaba ("Randomized algorithms for rounding in the tensor-train format", SIAM J. Sci. Comput. 45 (2023)
A74-A95) replaces it for those products; this module restates it in plain NumPy:

  1. contract the input y (ranks s_j) with a random sketch TT omega (ranks l_j) from the right,
         W_{d-1} = [1],   W_{j-1} = sum_n y_j[:, n, :] W_j omega_j[:, n, :]^T        (s_{j-1} x l_{j-1});
  2. sweep from the left: with the current left carriage X_j (unfolded (a n) x s_j),
         A = X_j W_j,  Q = orth(A),  X_j <- Q,  X_{j+1} <- (Q^* X_j) X_{j+1};
  3. the result (ranks l_j, left-orthonormal) is truncated to the target rank or tolerance by the truncated
     SVDs of App. A.3.3 taken from the right (lowrank.tt_truncate_left_orth): its carriages are already
     left-orthonormal, so the orthogonalisation half of the deterministic rounding has nothing left to do,
     and one sweep of truncated SVDs from the right completes it.
When y has TT ranks <= l_j the sketch spans its unfoldings exactly and the result equals the deterministic
rounding taken in that direction (lowrank.tt_round_rl: orthogonalise from the left, truncate from the right);
otherwise it is a near-optimal approximation with high probability (op. cit.).

The sketch carriages have Rademacher entries +-1 from the counter-based generator SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value i of stream `seed` is
mix(seed + (i + 1) * 0x9E3779B97F4A7C15) with the finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;  z = (z ^ (z >> 27)) * 0x94D049BB133111EB;  z ^ (z >> 31)
(arithmetic modulo 2^64); the sign is the top bit.  Counter of entry t of carriage j: (j + 1) * 2^40 + t.
"""
from __future__ import annotations

import numpy as np

from . import lowrank as _lr

__all__ = ["splitmix64", "sketch_tt", "tt_round_sketch"]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters) -> np.ndarray:
    """Outputs of SplitMix64 stream `seed` at the given counters (uint64 array)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sketch_tt(shape, ell, seed: int):
    """Rademacher sketch TT of mode sizes `shape` and inner ranks `ell` (an int or one per bond):
    carriage j has shape (l_{j-1}, N_j, l_j), l_0 = l_d = 1, entries +-1 (top bit of SplitMix64: 1 -> -1)."""
    d = len(shape)
    ls = [ell] * (d - 1) if np.isscalar(ell) else list(ell)
    rr = [1] + [int(v) for v in ls] + [1]
    out = []
    for j in range(d):
        n = rr[j] * shape[j] * rr[j + 1]
        t = np.arange(n, dtype=np.uint64) + np.uint64(j + 1) * np.uint64(1 << 40)
        bits = splitmix64(seed, t) >> np.uint64(63)
        out.append((1.0 - 2.0 * bits.astype(np.float64)).reshape(rr[j], shape[j], rr[j + 1]))
    return out


def tt_round_sketch(y, omega, rmax=None, tol=None, final=True):
    """Randomised TT rounding of y with the sketch TT omega (randomize-then-orthogonalize, then the
    truncated SVDs of App. A.3.3 from the right to rank rmax / tolerance tol; final=False: the left-orthonormal
    result of the sketch, of the sketch's ranks, without that last step)."""
    d = len(y)
    if d == 1:
        return [y[0].copy()]
    W = [None] * d
    W[d - 1] = np.ones((1, 1))
    for j in range(d - 1, 0, -1):
        # W_{j-1}[a, l] = sum_{n, b, m} y_j[a, n, b] W_j[b, m] omega_j[l, n, m]
        W[j - 1] = np.einsum("anb,bm,lnm->al", y[j], W[j], omega[j], optimize=True)
    x = [np.array(G, copy=True) for G in y]
    for j in range(d - 1):
        a, n, b = x[j].shape
        X = x[j].reshape(a * n, b)
        Q, _ = np.linalg.qr(X @ W[j])
        M = Q.conj().T @ X
        x[j] = Q.reshape(a, n, Q.shape[1])
        x[j + 1] = np.tensordot(M, x[j + 1], axes=([1], [0]))
    if not final:
        return x
    return _lr.tt_truncate_left_orth(x, rmax=rmax, tol=tol)
