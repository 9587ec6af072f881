"""Low-rank formats and the truncated GaNi operator — FP64 oracle, test infrastructure only.

Restates Sec. 3 and App. A of arXiv:1902.07455 in plain NumPy, in Fourier space as the paper writes it.

Tensor train (App. A.3, Eq. (TT)): a list of carriages G_j of shape (r_{j-1}, N_j, r_j), r_0 = r_d = 1,
    v[k_1..k_d] = G_1[0,k_1,:] G_2[:,k_2,:] ... G_d[:,k_d,0].
Tucker (App. A.2, Eq. (tucker)): core c of shape (r_1..r_d) and factor matrices B_j of shape (N_j, r_j)
    (the paper stores b^(j) as r_j x N_j; the columns here are its rows).
CP, d = 2 only (Sec. 3.1.1, App. A.1, Eq. (cano)): weights c (r,) and factors B_1 (N_1, r), B_2 (N_2, r).

Operations (each cites its passage):
  * Hadamard product: CP (App. A.1.1), Tucker factor pairs + Kronecker core (App. A.2.1, with the
    0-based pair index l = i*s + k), TT Khatri–Rao product of carriages (App. A.3.1);
  * sum: CP concatenation (Sec. 3.1.1); Tucker concatenated factors with a block core; TT block
    carriages (the paper points to App. A.3 for the TT sum without printing it; we use the standard
    block form: first carriage concatenated along its last index, last along its first, middle
    block-diagonal);
  * d-dimensional DFT as mode-wise 1D DFTs of factors / carriage fibres (Sec. 3.1.1, App. A.1.2,
    A.2.2, A.3.2);
  * truncation T: CP (d=2) QR of both factor matrices + SVD of R1 diag(c) R2^T (App. A.1.3, with the
    weights c that the printed product omits); Tucker QR of every factor + HOSVD of the updated core
    (App. A.2.3); TT rounding: right-to-left QR orthogonalisation then left-to-right truncated SVDs of
    the unfolded carriages (App. A.3.3);
  * TT-SVD of a full tensor by d-1 sequential SVDs (App. A.3.3).

The truncated operator is Eq. (Pls_lowrank):
    C~ v ~= T P^-1 T grad^* F T A~ F^-1 grad^ v,      b~ = - T P^-1 grad^* F A~ E,
with the gradient a rank-1 element-wise product on mode a (Sec. 3.2: grad^ = [2 pi i K_1 x 1 x 1, ...]),
the divergence the sum of the per-mode products with -2 pi i K_a, and P^-1 the exponential sum of
``oracle.expsum``.  The solver is the minimal-residual iteration with truncation of Sec. 3.3:
    r_i = T(b - C u_i),  omega_i = (C r_i, r_i) / ||C r_i||^2,  u_{i+1} = T(u_i + omega_i r_i),
stopped when the residual norm fails to decrease (Sec. 4.3) — the iterate with the smallest residual
is returned — or when it drops below a relative tolerance, or after ``maxit`` iterations.

Readings (listed in the design notes): every T truncates to the fixed solution rank r (Sec. 4.2 fixes
the rank), or with ``rank_tol`` to the smallest ranks within that relative tolerance (tol / sqrt(d - 1) per
TT bond, tol / sqrt(d) per Tucker mode); the residual is recomputed from its definition each iteration
and truncated; inner products of Fourier tensors take the real part; the relative error of Eq.
(rel_error) is reported as an absolute value.  Also here: a constant anisotropic part B of the material
(Sec. 4.4), the rank-adapting iteration Sec. 4.3 proposes (``minres_rank_adaptive``), and Ga in the low-rank
formats (``LowRankGa``: TT, Tucker, CP for d = 2; Sec. 2.2.3 with the truncations of Eq. (Pls_lowrank)).
"""
from __future__ import annotations

import numpy as np

from . import expsum as _expsum
from . import fourier_galerkin as _fg

# ----------------------------------------------------------------------------------------------
# rank selection
# ----------------------------------------------------------------------------------------------


def _keep(sv: np.ndarray, rmax, tol) -> int:
    """Number of singular values kept: at most rmax, and enough that the dropped tail has
    Frobenius norm <= tol * ||sv|| when tol is given (App. A.3.3 error bound per SVD)."""
    n = len(sv)
    k = n if rmax is None else min(int(rmax), n)
    if tol is not None and n > 0:
        tail = np.sqrt(np.cumsum(sv[::-1] ** 2))[::-1]  # tail[i] = ||sv[i:]||
        total = np.sqrt(np.sum(sv ** 2))
        ok = np.nonzero(np.append(tail, 0.0) <= tol * total)[0]
        k = min(k, max(int(ok[0]), 1))
    return max(k, 1)


# ----------------------------------------------------------------------------------------------
# tensor train (App. A.3)
# ----------------------------------------------------------------------------------------------


def tt_full(cores) -> np.ndarray:
    """Contract the carriages into the full tensor v[k_1..k_d] (Eq. (TT))."""
    out = cores[0]  # (1, N1, r1)
    for G in cores[1:]:
        out = np.tensordot(out, G, axes=([out.ndim - 1], [0]))
    return out[0, ..., 0]


def tt_ranks(cores):
    return [G.shape[0] for G in cores] + [1]


def tt_svd(A: np.ndarray, rmax=None, tol=None):
    """TT-SVD: d-1 sequential SVDs of the unfoldings (App. A.3.3).  With ``tol`` each SVD drops a tail
    of relative norm <= tol / sqrt(d-1), so the total error is <= tol ||A|| (the bound of App. A.3.3)."""
    d = A.ndim
    shape = A.shape
    cores = []
    r = 1
    M = A.reshape(shape[0], -1)
    loc_tol = None if tol is None else tol / np.sqrt(max(d - 1, 1))
    for j in range(d - 1):
        M = M.reshape(r * shape[j], -1)
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        k = _keep(s, rmax, loc_tol)
        cores.append(U[:, :k].reshape(r, shape[j], k))
        M = s[:k, None] * Vt[:k]
        r = k
    cores.append(M.reshape(r, shape[-1], 1))
    return cores


def tt_add(x, y):
    """Sum of two TTs in block-carriage form (standard form; ranks add)."""
    d = len(x)
    dt = np.result_type(x[0], y[0])
    out = []
    for j, (G, H) in enumerate(zip(x, y)):
        a, n, b = G.shape
        c, _, e = H.shape
        if d == 1:
            out.append(G + H)
        elif j == 0:
            out.append(np.concatenate([G, H], axis=2).astype(dt))
        elif j == d - 1:
            out.append(np.concatenate([G, H], axis=0).astype(dt))
        else:
            Z = np.zeros((a + c, n, b + e), dtype=dt)
            Z[:a, :, :b] = G
            Z[a:, :, b:] = H
            out.append(Z)
    return out


def tt_scale(x, alpha):
    """alpha * v: scales the first carriage."""
    return [x[0] * alpha] + [G.copy() for G in x[1:]]


def tt_hadamard(x, y):
    """Element-wise product: carriages combine by the Khatri–Rao product of App. A.3.1, Kronecker in
    the rank indices, element-wise in the mode index; pair index l = i*s + k (0-based)."""
    out = []
    for G, H in zip(x, y):
        a, n, b = G.shape
        c, _, e = H.shape
        Z = np.einsum("inj,knl->iknjl", G, H).reshape(a * c, n, b * e)
        out.append(Z)
    return out


def tt_mode_multiply(x, j, m):
    """Multiply the fibres of carriage j by the vector m over the mode index (a rank-1 element-wise
    product acting on mode j only, e.g. 2 pi i K_j of the gradient, Sec. 3.2)."""
    out = [G.copy() for G in x]
    out[j] = x[j] * m[None, :, None]
    return out


def tt_dft(x):
    """F_N of a TT: 1D DFT F_{N_j} (1/N_j normalised) of every carriage fibre (App. A.3.2)."""
    return [np.fft.fft(G, axis=1) / G.shape[1] for G in x]


def tt_idft(x):
    """F_N^{-1} of a TT: unnormalised inverse 1D DFT of every carriage fibre (App. A.3.2)."""
    return [np.fft.ifft(G, axis=1) * G.shape[1] for G in x]


def tt_dot(x, y) -> complex:
    """<x, y> = sum_k conj(x[k]) y[k] by left-to-right carriage contraction."""
    W = np.ones((1, 1), dtype=np.result_type(x[0], y[0], np.complex128))
    for G, H in zip(x, y):
        # W[a, c] -> sum_{a,c,n} W[a,c] conj(G[a,n,b]) H[c,n,e]
        W = np.einsum("ac,anb,cne->be", W, np.conj(G), H)
    return W[0, 0]


def tt_norm(x) -> float:
    return float(np.sqrt(max(np.real(tt_dot(x, x)), 0.0)))


def tt_round(x, rmax=None, tol=None):
    """TT rounding (App. A.3.3): right-to-left re-orthogonalisation by QR, then d-1 sequential
    truncated SVDs of the unfolded carriages from left to right.  Fixed rank ``rmax`` and/or relative
    tolerance ``tol`` (split evenly over the d-1 SVDs)."""
    d = len(x)
    G = [g.copy() for g in x]
    # right-to-left orthogonalisation: G_j = L Q with Q row-orthonormal (QR of the transpose)
    for j in range(d - 1, 0, -1):
        a, n, b = G[j].shape
        Q, R = np.linalg.qr(G[j].reshape(a, n * b).T)  # (n b) x k, k x a
        k = Q.shape[1]
        G[j] = Q.T.reshape(k, n, b)
        G[j - 1] = np.tensordot(G[j - 1], R.T, axes=([2], [0]))  # (.., .., a) x (a, k)
    loc_tol = None if tol is None else tol / np.sqrt(max(d - 1, 1))
    for j in range(d - 1):
        a, n, b = G[j].shape
        U, s, Vt = np.linalg.svd(G[j].reshape(a * n, b), full_matrices=False)
        k = _keep(s, rmax, loc_tol)
        G[j] = U[:, :k].reshape(a, n, k)
        G[j + 1] = np.tensordot(s[:k, None] * Vt[:k], G[j + 1], axes=([1], [0]))
    return G


def tt_truncate_left_orth(x, rmax=None, tol=None):
    """Truncation of a TT whose carriages 1..d-1 are left-orthonormal (the second half of the rounding of
    App. A.3.3 run from the right): for j = d-1 down to 1, the truncated SVD of carriage j unfolded as
    r_{j-1} x (N_j r_j) = U S V^*, carriage j <- V^* (k rows), carriage j-1 <- carriage j-1 U S.  With the
    left part orthonormal, that SVD is the SVD of the whole unfolding at bond j.  Fixed rank ``rmax`` and/or
    relative tolerance ``tol`` (split evenly over the d-1 SVDs, as in tt_round)."""
    d = len(x)
    G = [g.copy() for g in x]
    loc_tol = None if tol is None else tol / np.sqrt(max(d - 1, 1))
    for j in range(d - 1, 0, -1):
        a, n, b = G[j].shape
        U, s, Vt = np.linalg.svd(G[j].reshape(a, n * b), full_matrices=False)
        k = _keep(s, rmax, loc_tol)
        G[j] = Vt[:k].reshape(k, n, b)
        G[j - 1] = np.tensordot(G[j - 1], U[:, :k] * s[:k], axes=([2], [0]))
    return G


def tt_round_rl(x, rmax=None, tol=None):
    """TT rounding in the other direction (App. A.3.3 mirrored): left-to-right orthogonalisation by QR, then
    the truncated SVDs from right to left (tt_truncate_left_orth)."""
    d = len(x)
    G = [g.copy() for g in x]
    for j in range(d - 1):
        a, n, b = G[j].shape
        Q, R = np.linalg.qr(G[j].reshape(a * n, b))
        G[j] = Q.reshape(a, n, Q.shape[1])
        G[j + 1] = np.tensordot(R, G[j + 1], axes=([1], [0]))
    return tt_truncate_left_orth(G, rmax=rmax, tol=tol)


def tt_zeros(shape, dtype=np.complex128):
    return [np.zeros((1, n, 1), dtype=dtype) for n in shape]


def tt_from_separable(terms, weights=None):
    """TT of a sum of separable terms sum_i w_i f_i^1 x ... x f_i^d (a CP form), in block form."""
    R = len(terms)
    d = len(terms[0])
    w = np.ones(R) if weights is None else np.asarray(weights, dtype=np.float64)
    cores = []
    for j in range(d):
        F = np.stack([np.asarray(t[j], dtype=np.float64) for t in terms], axis=1)  # (N, R)
        n = F.shape[0]
        if d == 1:
            cores.append((F @ w).reshape(1, n, 1))
        elif j == 0:
            cores.append((F * w[None, :]).reshape(1, n, R))
        elif j == d - 1:
            cores.append(F.T.reshape(R, n, 1))
        else:
            Z = np.zeros((R, n, R))
            for i in range(R):
                Z[i, :, i] = F[:, i]
            cores.append(Z)
    return cores


# ----------------------------------------------------------------------------------------------
# Tucker (App. A.2)
# ----------------------------------------------------------------------------------------------


def tucker_full(core, factors) -> np.ndarray:
    """sum_i c[i_1..i_d] b^(1)[i_1] x ... x b^(d)[i_d]  (Eq. (tucker))."""
    out = core
    for j, B in enumerate(factors):
        out = np.moveaxis(np.tensordot(B, out, axes=([1], [j])), 0, j)
    return out


def tucker_hosvd(A: np.ndarray, rmax=None, tol=None):
    """HOSVD of a full tensor (App. A.2.3): factors = leading left singular vectors of each mode
    unfolding, core = A contracted with the factors' transposes."""
    d = A.ndim
    factors = []
    loc_tol = None if tol is None else tol / np.sqrt(d)
    for j in range(d):
        M = np.moveaxis(A, j, 0).reshape(A.shape[j], -1)
        U, s, _ = np.linalg.svd(M, full_matrices=False)
        k = _keep(s, rmax, loc_tol)
        factors.append(U[:, :k])
    core = A
    for j, B in enumerate(factors):
        core = np.moveaxis(np.tensordot(B.conj().T, core, axes=([1], [j])), 0, j)
    return core, factors


def tucker_add(x, y):
    """Concatenated factors with a block-diagonal core (the frame of Sec. 3.1.2 / App. A.2)."""
    (c1, F1), (c2, F2) = x, y
    d = c1.ndim
    shape = tuple(a + b for a, b in zip(c1.shape, c2.shape))
    core = np.zeros(shape, dtype=np.result_type(c1, c2))
    core[tuple(slice(0, s) for s in c1.shape)] = c1
    core[tuple(slice(s, None) for s in c1.shape)] = c2
    factors = [np.concatenate([F1[j], F2[j]], axis=1) for j in range(d)]
    return core, factors


def tucker_hadamard(x, y):
    """Factor pairs b_v[i] * b_w[k] at column l = i*s + k and the Kronecker product of the cores
    (App. A.2.1, 0-based pair index)."""
    (c1, F1), (c2, F2) = x, y
    factors = [np.einsum("ni,nk->nik", A, B).reshape(A.shape[0], -1) for A, B in zip(F1, F2)]
    core = np.kron(c1, c2)
    return core, factors


def tucker_mode_multiply(x, j, m):
    c, F = x
    F = [f.copy() for f in F]
    F[j] = F[j] * m[:, None]
    return c.copy(), F


def tucker_dft(x):
    c, F = x
    return c.copy(), [np.fft.fft(f, axis=0) / f.shape[0] for f in F]


def tucker_idft(x):
    c, F = x
    return c.copy(), [np.fft.ifft(f, axis=0) * f.shape[0] for f in F]


def tucker_scale(x, alpha):
    c, F = x
    return c * alpha, [f.copy() for f in F]


def tucker_round(x, rmax=None, tol=None):
    """Truncation of App. A.2.3: QR of every factor (frame -> orthonormal basis), core updated by the
    R factors, then HOSVD of the core; factors become Q U_k."""
    c, F = x
    core = c
    Qs = []
    for j, B in enumerate(F):
        Q, R = np.linalg.qr(B)
        Qs.append(Q)
        core = np.moveaxis(np.tensordot(R, core, axes=([1], [j])), 0, j)
    cs, Us = tucker_hosvd(core, rmax=rmax, tol=tol)
    return cs, [Q @ U for Q, U in zip(Qs, Us)]


def tucker_dot(x, y) -> complex:
    """<x, y> via the factor Gram matrices and the cores."""
    (c1, F1), (c2, F2) = x, y
    t = c2
    for j in range(len(F1)):
        G = F1[j].conj().T @ F2[j]  # (r1_j, r2_j)
        t = np.moveaxis(np.tensordot(G, t, axes=([1], [j])), 0, j)
    return np.sum(np.conj(c1) * t)


def tucker_norm(x) -> float:
    return float(np.sqrt(max(np.real(tucker_dot(x, x)), 0.0)))


def tucker_from_separable(terms, weights=None):
    R = len(terms)
    d = len(terms[0])
    w = np.ones(R) if weights is None else np.asarray(weights, dtype=np.float64)
    factors = [np.stack([np.asarray(t[j], dtype=np.float64) for t in terms], axis=1) for j in range(d)]
    core = np.zeros((R,) * d)
    for i in range(R):
        core[(i,) * d] = w[i]
    return core, factors


def tucker_zeros(shape, dtype=np.complex128):
    return np.zeros((1,) * len(shape), dtype=dtype), [np.zeros((n, 1), dtype=dtype) for n in shape]


# ----------------------------------------------------------------------------------------------
# CP, d = 2 (Sec. 3.1.1, App. A.1)
# ----------------------------------------------------------------------------------------------


def cp_full(x) -> np.ndarray:
    c, B1, B2 = x
    return (B1 * c[None, :]) @ B2.T


def cp_add(x, y):
    return (np.concatenate([x[0], y[0]]), np.concatenate([x[1], y[1]], axis=1),
            np.concatenate([x[2], y[2]], axis=1))


def cp_hadamard(x, y):
    """sum_i sum_k c_v[i] c_w[k] (b1_v[i]*b1_w[k]) x (b2_v[i]*b2_w[k])  (Sec. 3.1.1, App. A.1.1)."""
    c = np.kron(x[0], y[0])
    B1 = np.einsum("ni,nk->nik", x[1], y[1]).reshape(x[1].shape[0], -1)
    B2 = np.einsum("ni,nk->nik", x[2], y[2]).reshape(x[2].shape[0], -1)
    return c, B1, B2


def cp_mode_multiply(x, j, m):
    c, B1, B2 = x
    if j == 0:
        return c.copy(), B1 * m[:, None], B2.copy()
    return c.copy(), B1.copy(), B2 * m[:, None]


def cp_dft(x):
    c, B1, B2 = x
    return c.copy(), np.fft.fft(B1, axis=0) / B1.shape[0], np.fft.fft(B2, axis=0) / B2.shape[0]


def cp_idft(x):
    c, B1, B2 = x
    return c.copy(), np.fft.ifft(B1, axis=0) * B1.shape[0], np.fft.ifft(B2, axis=0) * B2.shape[0]


def cp_scale(x, alpha):
    return x[0] * alpha, x[1].copy(), x[2].copy()


def cp_round(x, rmax=None, tol=None):
    """App. A.1.3: B1 = Q1 R1, B2 = Q2 R2, SVD of R1 diag(c) R2^T = U S V^T, keep k terms:
    weights S_k, factors Q1 U_k and Q2 conj(V_k)."""
    c, B1, B2 = x
    Q1, R1 = np.linalg.qr(B1)
    Q2, R2 = np.linalg.qr(B2)
    U, s, Vt = np.linalg.svd((R1 * c[None, :]) @ R2.T, full_matrices=False)
    k = _keep(s, rmax, tol)
    return s[:k].astype(np.result_type(c, B1, B2)), Q1 @ U[:, :k], Q2 @ Vt[:k].T


def cp_dot(x, y) -> complex:
    G1 = x[1].conj().T @ y[1]
    G2 = x[2].conj().T @ y[2]
    return np.sum(np.conj(x[0])[:, None] * G1 * G2 * y[0][None, :])


def cp_norm(x) -> float:
    return float(np.sqrt(max(np.real(cp_dot(x, x)), 0.0)))


def cp_from_separable(terms, weights=None):
    R = len(terms)
    w = np.ones(R) if weights is None else np.asarray(weights, dtype=np.float64)
    B1 = np.stack([np.asarray(t[0], dtype=np.float64) for t in terms], axis=1)
    B2 = np.stack([np.asarray(t[1], dtype=np.float64) for t in terms], axis=1)
    return w.copy(), B1, B2


def cp_zeros(shape, dtype=np.complex128):
    return np.zeros(1, dtype=dtype), np.zeros((shape[0], 1), dtype=dtype), np.zeros((shape[1], 1), dtype=dtype)


# ----------------------------------------------------------------------------------------------
# format dispatch
# ----------------------------------------------------------------------------------------------


class _Fmt:
    def __init__(self, full, add, had, mmul, dft, idft, scale, rnd, dot, norm, sep, zeros):
        self.full, self.add, self.had, self.mmul = full, add, had, mmul
        self.dft, self.idft, self.scale, self.round = dft, idft, scale, rnd
        self.dot, self.norm, self.sep, self.zeros = dot, norm, sep, zeros


FORMATS = {
    "tt": _Fmt(tt_full, tt_add, tt_hadamard, tt_mode_multiply, tt_dft, tt_idft, tt_scale, tt_round,
               tt_dot, tt_norm, tt_from_separable, tt_zeros),
    "tucker": _Fmt(lambda x: tucker_full(*x), tucker_add, tucker_hadamard, tucker_mode_multiply,
                   tucker_dft, tucker_idft, tucker_scale, tucker_round, tucker_dot, tucker_norm,
                   tucker_from_separable, tucker_zeros),
    "cp": _Fmt(cp_full, cp_add, cp_hadamard, cp_mode_multiply, cp_dft, cp_idft, cp_scale, cp_round,
               cp_dot, cp_norm, cp_from_separable, cp_zeros),
}


def compress(A: np.ndarray, fmt: str, rmax=None, tol=None):
    """Low-rank form of a full real tensor: TT-SVD, HOSVD, or (d=2) truncated SVD as CP."""
    if fmt == "tt":
        return tt_svd(A, rmax=rmax, tol=tol)
    if fmt == "tucker":
        return tucker_hosvd(A, rmax=rmax, tol=tol)
    if fmt == "cp":
        if A.ndim != 2:
            raise ValueError("CP is used for d = 2 only (Sec. 3.1)")
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
        k = _keep(s, rmax, tol)
        return s[:k].copy(), U[:, :k].copy(), Vt[:k].T.copy()
    raise ValueError(fmt)


# ----------------------------------------------------------------------------------------------
# the truncated operator (Eq. (Pls_lowrank)) and the minimal-residual iteration (Sec. 3.3)
# ----------------------------------------------------------------------------------------------


class LowRankGaNi:
    """Operator C~ and right-hand side b~ of Eq. (Pls_lowrank) for an isotropic coefficient a(x) I given
    in low-rank form ``a_lr`` (format ``fmt``), grid ``shape`` (odd sizes), solution rank ``rank`` and
    the exponential-sum accuracy ``pinv_eps`` of P~^-1.  All tensors are Fourier coefficient tensors
    except the coefficient, which holds grid values (as in the paper's A~)."""

    def __init__(self, a_lr, shape, fmt="tt", rank=10, pinv_eps=0.1, rank_tol=None, B=None, sketch=None):
        self.f = FORMATS[fmt]
        self.fmt = fmt
        # randomised rounding of the products (TT only): (oversampling p, seed[, keep]) or None.  The material
        # products and the P~^-1 product are then truncated by ``sketch.tt_round_sketch`` with a sketch of
        # ranks rank + p, acting on grid values (the material product is formed there; the P~^-1 product
        # is mapped there by F^-1 and back by F); every other T stays the deterministic rounding.  keep: those
        # two truncations return the sketch's rank rank + p (no final rounding to rank).
        if sketch is not None and fmt != "tt":
            raise ValueError("the randomised rounding is defined for the TT format")
        self.sketch = None if sketch is None else (int(sketch[0]), int(sketch[1]),
                                                   bool(sketch[2]) if len(sketch) > 2 else False)
        self.a = a_lr
        # constant anisotropic part: A~(x) = a(x) I + B (the modified materials of Sec. 4.4)
        self.B = None if B is None else np.asarray(B, dtype=np.float64)
        self.shape = tuple(int(n) for n in shape)
        self.d = len(self.shape)
        self.rank = rank
        self.rank_tol = rank_tol
        self.K = [_fg.frequencies(n).astype(np.float64) for n in self.shape]
        xmax = float(sum(((n - 1) // 2) ** 2 for n in self.shape))
        t, w = _expsum.expsum_inverse(xmax, pinv_eps)
        self.pinv_t, self.pinv_w = t, w
        terms = [[np.exp(-tm * K ** 2) for K in self.K] for tm in t]
        self.Pinv = self.f.sep(terms, w)

    def T(self, x):
        return self.f.round(x, rmax=self.rank, tol=self.rank_tol)

    def T_values(self, x):
        """T of a product held as grid values: the randomised rounding when ``sketch`` is set, else T."""
        if self.sketch is None:
            return self.T(x)
        from . import sketch as _sk
        over, seed, keep = self.sketch
        omega = _sk.sketch_tt(self.shape, self.rank + over, seed)
        return _sk.tt_round_sketch(x, omega, rmax=self.rank, tol=self.rank_tol, final=not keep)

    def T_pinv(self, sh):
        """T P~^-1 s for a Fourier tensor s: with ``sketch`` the product is truncated as grid values."""
        f = self.f
        if self.sketch is None:
            return self.T(f.had(self.Pinv, sh))
        return f.dft(self.T_values(f.idft(f.had(self.Pinv, sh))))

    def apply(self, vh):
        """T P~^-1 T grad^* F T A~ F^-1 grad^ v  (Eq. (Pls_lowrank)).  With the constant anisotropic part
        B, component a of A~ e is a e_a + sum_b B[a, b] e_b (zero entries of B skipped)."""
        f = self.f
        acc = None
        es = None
        if self.B is not None:
            es = [f.idft(f.mmul(vh, b, 2j * np.pi * self.K[b])) for b in range(self.d)]
        for a in range(self.d):
            g = f.mmul(vh, a, 2j * np.pi * self.K[a])      # gradient, mode a (rank unchanged)
            e = f.idft(g)                                   # F^-1, mode-wise
            ae = f.had(self.a, e)
            if self.B is not None:
                for b in range(self.d):
                    if self.B[a, b] != 0.0:
                        ae = f.add(ae, f.scale(es[b], float(self.B[a, b])))
            w = self.T_values(ae)                           # T A~ e_a
            wh = f.dft(w)                                   # F, mode-wise
            term = f.mmul(wh, a, -2j * np.pi * self.K[a])   # divergence, mode a
            acc = term if acc is None else f.add(acc, term)
        s = self.T(acc)                                     # T after the sum
        return self.T_pinv(s)                               # T P~^-1

    def rhs(self, E):
        """b~ = - T P~^-1 grad^* F A~ E  (Eq. (Pls_lowrank)).  A constant anisotropic part adds the constant
        field B E, whose divergence is zero, so B does not enter."""
        f = self.f
        acc = None
        ah = f.dft(self.a)
        for a in range(self.d):
            if E[a] == 0.0:
                continue
            term = f.mmul(f.scale(ah, float(E[a])), a, -2j * np.pi * self.K[a])
            acc = term if acc is None else f.add(acc, term)
        if acc is None:
            return f.zeros(self.shape)
        return f.scale(self.T_pinv(acc), -1.0)

    def homogenised_coefficient(self, uh, E) -> float:
        """A_eff E.E = (1/|N|) sum_k A~(x_k)(E + e(x_k)).(E + e(x_k)) with e_a = F^-1 grad^_a u^ (Eq. (homog)),
        evaluated by low-rank contractions without truncation:
        |E|^2 <a,1> + 2 sum_a E_a <a, e_a> + sum_a <a * e_a, e_a>  (+ E.B E + sum_ab B_ab <e_a, e_b>)."""
        f = self.f
        size = float(np.prod(self.shape))
        ones = f.sep([[np.ones(n) for n in self.shape]])
        a_mean = np.real(f.dot(ones, self.a)) / size
        val = float(np.dot(E, E)) * a_mean
        es = []
        for a in range(self.d):
            e = f.idft(f.mmul(uh, a, 2j * np.pi * self.K[a]))
            es.append(e)
            ae = f.had(self.a, e)
            val += 2.0 * float(E[a]) * np.real(f.dot(ones, ae)) / size
            val += np.real(f.dot(e, ae)) / size
        if self.B is not None:
            # (E + e).B(E + e) averaged: E.B E + sum_ab B[a, b] <e_a, e_b> / |N| (e has zero mean)
            val += float(E @ self.B @ E)
            for a in range(self.d):
                for b in range(self.d):
                    if self.B[a, b] != 0.0:
                        val += float(self.B[a, b]) * np.real(f.dot(es[a], es[b])) / size
        return float(val)

    def full_field(self, uh) -> np.ndarray:
        """Real grid values u = F^-1 u^ of a low-rank solution (for comparisons at small N)."""
        return np.real(_fg.idft(self.f.full(uh), self.d))


def minres(op: LowRankGaNi, E, tol=1e-10, maxit=200, stop_on_increase=True, callback=None):
    """Minimal-residual iteration with truncation (Sec. 3.3):
        r_i = T(b - C u_i),  omega_i = Re(C r_i, r_i) / ||C r_i||^2,  u_{i+1} = T(u_i + omega_i r_i).
    Stops when ||r_i|| fails to decrease (returning the iterate with the smallest residual, Sec. 4.3),
    when ||r_i|| <= tol ||b||, or after maxit iterations.  ``stop_on_increase`` = k > 1 (an int) stops after k
    consecutive iterations without a new smallest residual instead of at the first failure.  Returns dict(u,
    iters, rel_resid, history, Aeff)."""
    f = op.f
    E = np.asarray(E, dtype=np.float64)
    b = op.rhs(E)
    nb = f.norm(b)
    u = f.zeros(op.shape)
    best = (np.inf, u, 0)
    hist = []
    it = 0
    patience = int(stop_on_increase)
    since_best = 0
    while True:
        r = op.T(f.add(b, f.scale(op.apply(u), -1.0))) if it > 0 else b
        nr = f.norm(r) / nb if nb > 0 else 0.0
        hist.append(nr)
        if callback is not None:
            callback(it, u, nr)
        if nr < best[0]:
            best = (nr, u, it)
            since_best = 0
        elif patience:
            since_best += 1
            if since_best >= patience:
                break
        if nr <= tol or it >= maxit:
            break
        q = op.apply(r)
        qq = np.real(f.dot(q, q))
        if qq == 0.0:
            break
        omega = np.real(f.dot(q, r)) / qq
        u = op.T(f.add(u, f.scale(r, omega))) if it > 0 else op.T(f.scale(r, omega))
        it += 1
    nr, u, itb = best
    return dict(u=u, iters=itb, rel_resid=nr, history=hist, Aeff=op.homogenised_coefficient(u, E))


def minres_rank_adaptive(op: LowRankGaNi, E, rank_start, rank_step, tol=1e-10, maxit=200, stop_on_increase=True):
    """Rank-adapting minimal-residual iteration (the solver Sec. 4.3 proposes: start with a low solution
    rank and raise it during the iterations).  Reading: the iteration of ``minres`` runs with every T at
    the current rank r_c = rank_start; when the residual norm fails to decrease and r_c < op.rank (the
    cap), r_c rises by rank_step (at most to the cap), the right-hand side is rebuilt at the new rank, and
    the iteration restarts from the best iterate so far with its residual recomputed at the new rank
    (the comparison for "fails to decrease" starts again from there).  At the cap it is the fixed-rank
    iteration and stops as ``minres`` does: a failure to decrease ends it (``stop_on_increase`` = True),
    or k consecutive iterations without a new smallest residual (an int k > 1), or never (False / 0); so do
    the relative tolerance and ``maxit`` (iterations summed over all ranks).  The tolerance is read as a statement about the solution at the cap: below it, a
    residual within the tolerance raises the rank like a stagnation does (that residual is truncated at the
    lower rank and understates the one the cap gives), again after a raise while it stays within it; at the
    cap it ends the iteration only for an iterate of a step taken there (not for the restart point, which
    has the lower rank).  Returns dict(u, iters, rel_resid, rank, history, Aeff) for the best iterate of the
    last rank."""
    f = op.f
    E = np.asarray(E, dtype=np.float64)
    rmax = op.rank
    rc = min(int(rank_start), rmax)
    op.rank = rc
    try:
        b = op.rhs(E)
        nb = f.norm(b)
        u, u_zero = f.zeros(op.shape), True
        r = b
        best = (np.inf, u, 0, True)
        hist = []
        it = 0
        cap_steps = 0  # steps taken at the cap
        patience = int(stop_on_increase)
        since_best = 0  # iterations at the cap since the last new smallest residual
        while True:
            nr = f.norm(r) / nb if nb > 0 else 0.0
            hist.append(nr)
            improved = nr < best[0]
            if improved:
                best = (nr, u, it, u_zero)
                since_best = 0
            if rc < rmax and (not improved or nr <= tol):
                # stagnation, or the tolerance met, below the cap: raise the rank and restart from the best
                # iterate (again while the restarted residual is within the tolerance below the cap)
                while True:
                    rc = min(rc + int(rank_step), rmax)
                    op.rank = rc
                    b = op.rhs(E)
                    nb = f.norm(b)
                    u, u_zero = best[1], best[3]
                    r = b if u_zero else op.T(f.add(b, f.scale(op.apply(u), -1.0)))
                    nr = f.norm(r) / nb if nb > 0 else 0.0
                    hist.append(nr)
                    best = (nr, u, best[2], u_zero)
                    since_best = 0
                    if not (rc < rmax and nr <= tol):
                        break
            elif not improved and patience:
                since_best += 1
                if since_best >= patience:
                    break
            if (nr <= tol and rc >= rmax and cap_steps > 0) or it >= maxit:
                break
            q = op.apply(r)
            qq = np.real(f.dot(q, q))
            if qq == 0.0:
                break
            omega = np.real(f.dot(q, r)) / qq
            u = op.T(f.scale(r, omega)) if u_zero else op.T(f.add(u, f.scale(r, omega)))
            u_zero = False
            it += 1
            cap_steps += rc >= rmax
            r = op.T(f.add(b, f.scale(op.apply(u), -1.0)))
        nr, u, itb, _ = best
        return dict(u=u, iters=itb, rel_resid=nr, rank=rc, history=hist, Aeff=op.homogenised_coefficient(u, E))
    finally:
        op.rank = rmax


# ----------------------------------------------------------------------------------------------
# Ga (exact integration on the double grid, Sec. 2.2.3) in the low-rank formats
# ----------------------------------------------------------------------------------------------


def tt_mode_map(x, j, L):
    """Carriage j's fibres mapped by the matrix L (M x N): G_j[a, :, b] <- L G_j[a, :, b] — a linear map on
    mode j only, which may change that mode's size (zero padding, projection)."""
    out = [G.copy() for G in x]
    out[j] = np.einsum("mn,anb->amb", L, x[j])
    return out


def tucker_mode_map(x, j, L):
    """The same linear map on mode j of a Tucker tensor: factor B_j <- L B_j (core unchanged)."""
    c, F = x
    F = [f.copy() for f in F]
    F[j] = L @ F[j]
    return c.copy(), F


def cp_mode_map(x, j, L):
    """The same on mode j of a CP tensor (d = 2): factor B_j <- L B_j (weights unchanged)."""
    c, B1, B2 = x
    if j == 0:
        return c.copy(), L @ B1, B2.copy()
    return c.copy(), B1.copy(), L @ B2


MODE_MAPS = {"tt": tt_mode_map, "tucker": tucker_mode_map, "cp": cp_mode_map}


def ga_matrices(N: int):
    """Per-mode matrices of Ga for one axis of N points and the double grid M = 2N - 1 (storage order):
    inject (M x N) zero-pads Fourier coefficients, project (N x M) is its adjoint, and extend (M x N) maps
    pixel values g_p of a pixel-wise constant factor to int g(t) phi^j_M(t) dt,
        extend[j, p] = M^-1 sum_{m in Z_M} s(m) e^{2 pi i m (x_p - y_j)},  s(m) = sin(pi m / N) / (pi m),
    the one-axis form of the modified coefficient of Sec. 2.2.3."""
    M = 2 * N - 1
    kN = _fg.frequencies(N)
    inj = np.zeros((M, N))
    inj[kN % M, np.arange(N)] = 1.0
    ms = _fg.frequencies(M).astype(np.float64)
    s = np.full(M, 1.0 / N)
    nz = ms != 0
    s[nz] = np.sin(np.pi * ms[nz] / N) / (np.pi * ms[nz])
    xp = _fg.grid_points(N)
    yj = _fg.grid_points(M)
    ph = np.exp(2j * np.pi * ms[None, None, :] * (xp[None, :, None] - yj[:, None, None]))
    ext = (ph * s[None, None, :]).sum(axis=2) / M
    return inj, inj.T.copy(), np.real(ext)


class LowRankGa:
    """Ga in a low-rank format (TT, Tucker, or CP for d = 2): C~ v ~= T P~^-1 T grad^* I* F_M T A~ F_M^-1 I grad^ v
    and b~ = - T P~^-1 grad^* I* F_M A~ E (Eq. (ls_Ga_fourier) with the truncations placed as in Eq.
    (Pls_lowrank)), A~ the modified coefficient of a pixel-wise constant a given in the same format as its
    pixel values on the grid N; I, I* and the DFTs act mode by mode (on carriage fibres or factor columns).
    Interface of ``LowRankGaNi`` (for ``minres``).  A constant anisotropic part B (Sec. 4.4) is part of the
    material A = a I + B whose modified coefficient is taken: A~ = a~ I + B 1~, 1~ the modified coefficient of the
    constant 1 (the same mode maps applied to the all-ones tensor), so component a of the product on the double
    grid is a~ e_a + sum_b B[a, b] 1~ e_b before its T."""

    def __init__(self, a_tt, shape, rank=10, pinv_eps=0.1, rank_tol=None, fmt="tt", B=None):
        self.f = FORMATS[fmt]
        self.fmt = fmt
        self._map = MODE_MAPS[fmt]
        self.shape = tuple(int(n) for n in shape)
        self.d = len(self.shape)
        self.rank = rank
        self.rank_tol = rank_tol
        self.B = None if B is None else np.asarray(B, dtype=np.float64)
        self.K = [_fg.frequencies(n).astype(np.float64) for n in self.shape]
        self.mats = [ga_matrices(n) for n in self.shape]
        At = _as_float(fmt, a_tt)
        Ones = self.f.sep([[np.ones(n) for n in self.shape]])
        for j in range(self.d):
            At = self._map(At, j, self.mats[j][2])
            Ones = self._map(Ones, j, self.mats[j][2])
        self.At = At                                             # values on the double grid
        self.Ones = Ones                                         # 1~, the modified coefficient of 1
        xmax = float(sum(((n - 1) // 2) ** 2 for n in self.shape))
        t, w = _expsum.expsum_inverse(xmax, pinv_eps)
        self.pinv_t, self.pinv_w = t, w
        self.Pinv = self.f.sep([[np.exp(-tm * K ** 2) for K in self.K] for tm in t], w)

    def T(self, x):
        return self.f.round(x, rmax=self.rank, tol=self.rank_tol)

    def _inject(self, xh):
        for j in range(self.d):
            xh = self._map(xh, j, self.mats[j][0])
        return xh

    def _project(self, xh):
        for j in range(self.d):
            xh = self._map(xh, j, self.mats[j][1])
        return xh

    def _grad_double(self, vh, a):
        """e_a on the double grid: F_M^-1 I grad^_a v^ (values)."""
        return self.f.idft(self._inject(self.f.mmul(vh, a, 2j * np.pi * self.K[a])))

    def apply(self, vh):
        f = self.f
        acc = None
        eds = [self._grad_double(vh, a) for a in range(self.d)] if self.B is not None else None
        for a in range(self.d):
            ed = eds[a] if eds is not None else self._grad_double(vh, a)
            m = f.had(self.At, ed)
            if self.B is not None:
                for b in range(self.d):
                    if self.B[a, b] != 0.0:
                        m = f.add(m, f.scale(f.had(self.Ones, eds[b]), float(self.B[a, b])))
            w = self.T(m)                                            # T A~ e_a on the double grid
            wh = self._project(f.dft(w))                           # I* F_M
            term = f.mmul(wh, a, -2j * np.pi * self.K[a])
            acc = term if acc is None else f.add(acc, term)
        s = self.T(acc)
        return self.T(f.had(self.Pinv, s))

    def rhs(self, E):
        f = self.f
        ah = self._project(f.dft(self.At))
        acc = None
        for a in range(self.d):
            if E[a] == 0.0:
                continue
            term = f.mmul(f.scale(ah, float(E[a])), a, -2j * np.pi * self.K[a])
            acc = term if acc is None else f.add(acc, term)
        if acc is None:
            return f.zeros(self.shape)
        return f.scale(self.T(f.had(self.Pinv, acc)), -1.0)

    def homogenised_coefficient(self, uh, E) -> float:
        """sum over the double grid of A~ |E + e|^2 (exact integration), by low-rank contractions:
        |E|^2 <A~, 1> + 2 sum_a E_a <A~, e_a> + sum_a <A~ e_a, e_a>; with B also
        E.B E <1~, 1> + 2 sum_ab E_a B[a, b] <1~, e_b> + sum_ab B[a, b] <1~ e_a, e_b>."""
        f = self.f
        E = np.asarray(E, dtype=np.float64)
        ones = f.sep([[np.ones(2 * n - 1) for n in self.shape]])
        val = float(E @ E) * np.real(f.dot(ones, self.At))
        es = []
        for a in range(self.d):
            e = self._grad_double(uh, a)
            es.append(e)
            ae = f.had(self.At, e)
            val += 2.0 * float(E[a]) * np.real(f.dot(ones, ae))
            val += np.real(f.dot(e, ae))
        if self.B is not None:
            val += float(E @ self.B @ E) * np.real(f.dot(ones, self.Ones))
            for a in range(self.d):
                for b in range(self.d):
                    if self.B[a, b] == 0.0:
                        continue
                    oe = f.had(self.Ones, es[a])
                    val += 2.0 * float(E[b] * self.B[b, a]) * np.real(f.dot(ones, oe))
                    val += float(self.B[a, b]) * np.real(f.dot(oe, es[b]))
        return float(val)

    def full_field(self, uh) -> np.ndarray:
        return np.real(_fg.idft(self.f.full(uh), self.d))


LowRankGaTT = LowRankGa  # the TT instance (fmt="tt"), under its earlier name


def _as_float(fmt, x):
    """A real FP64 copy of a low-rank tensor of the given format."""
    if fmt == "tt":
        return [np.asarray(G, dtype=np.float64) for G in x]
    if fmt == "tucker":
        c, F = x
        return np.asarray(c, dtype=np.float64), [np.asarray(f, dtype=np.float64) for f in F]
    c, B1, B2 = x
    return np.asarray(c, dtype=np.float64), np.asarray(B1, dtype=np.float64), np.asarray(B2, dtype=np.float64)


def relative_error(A_full: float, A_lowrank: float) -> float:
    """|A_N - A_{N,r}| / A_N  (Eq. (rel_error), reported as an absolute value)."""
    return abs(A_full - A_lowrank) / abs(A_full)
