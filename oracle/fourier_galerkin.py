"""Full-format Fourier–Galerkin (GaNi) oracle, FP64 — test infrastructure only.

Restates Sec. 2 of arXiv:1902.07455 ("FFT-based homogenisation accelerated by low-rank tensor
approximations") in plain NumPy:

* odd grid sizes N, frequencies Z_N = {k : |k| < N/2}, grid points x_k = k/N (Sec. 2.2.1);
* DFT matrices F_N[m,k] = w^{-mk}/|N| and F_N^{-1}[m,k] = w^{mk} (Sec. 2.2.1);
* Fourier gradient (grad^ v)[a,k] = 2 pi i k_a v[k] and its adjoint, the divergence
  (grad^* w)[k] = sum_a -2 pi i k_a w[a,k] (Sec. 2.2.1);
* the GaNi linear system, Eq. (ls_GaNi_fourier):
      grad^* F A~ F^{-1} grad^ u^ = - grad^* F A~ E;
* the Laplacian preconditioner P^[k,k] = k.k with pseudo-inverse 1/(k.k), 0 at k = 0 (Sec. 2.3,
  Eq. (Pls_GaNi_fourier));
* preconditioned CG (Sec. 3.3 and 4: the full systems are solved by CG on Eq. (Pls_fourier));
* the homogenised coefficient A_eff E.E = (1/|N|) sum_k A(x_k)(E + e(x_k)).(E + e(x_k)) with the
  gradient field e = F^{-1} grad^ u^ (Eq. (homog), (bilinear) with the rectangle rule of Sec. 2.2.2).

Storage: a scalar grid function is an ndarray of shape (N,)*d whose entry at storage index i along an
axis belongs to frequency / grid index k = i if i <= (N-1)/2 else i - N (so k = i mod N).  Vector
fields carry a leading axis of length d.

Readings where the paper is silent (each is listed in the design notes):
* the GaNi quadrature weight 1/|N| missing from the printed bilinear form is restored in A_eff
  (the printed sum would make A_eff = |N| A for a constant A, contradicting "exact for constant A");
* the CG stopping test is relative, on the preconditioned residual: ||P^-1 r|| <= tol ||P^-1 b||;
* inner products of Fourier fields take the real part (fields are Hermitian-symmetric).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "frequencies", "grid_points", "dft", "idft", "grad_hat", "div_hat", "precond_inv",
    "gani_operator", "gani_rhs", "pcg", "homogenised_coefficient", "solve_gani",
]


def frequencies(N: int) -> np.ndarray:
    """Z_N in storage order: k = i for i <= (N-1)/2, else i - N (Sec. 2.2.1, N odd)."""
    if N % 2 != 1 or N < 1:
        raise ValueError("the GaNi discretisation uses odd N only (Sec. 2.2.1)")
    k = np.arange(N, dtype=np.int64)
    k[k > (N - 1) // 2] -= N
    return k


def grid_points(N: int) -> np.ndarray:
    """x_k = k/N for k in Z_N, in storage order (Sec. 2.2.1)."""
    return frequencies(N) / N


def _axes(v: np.ndarray, d: int):
    return tuple(range(v.ndim - d, v.ndim))


def dft(v: np.ndarray, d: int) -> np.ndarray:
    """F_N v with F_N[m,k] = w^{-mk} / |N| over the last d axes (Sec. 2.2.1)."""
    ax = _axes(v, d)
    size = int(np.prod([v.shape[a] for a in ax]))
    return np.fft.fftn(v, axes=ax) / size


def idft(vh: np.ndarray, d: int) -> np.ndarray:
    """F_N^{-1} v^ with F_N^{-1}[m,k] = w^{mk} over the last d axes (Sec. 2.2.1)."""
    ax = _axes(vh, d)
    size = int(np.prod([vh.shape[a] for a in ax]))
    return np.fft.ifftn(vh, axes=ax) * size


def _kgrid(shape):
    """Per-axis frequency arrays broadcast to the grid: K[a] has k_a at every grid index."""
    d = len(shape)
    ks = [frequencies(n) for n in shape]
    return np.stack(np.meshgrid(*ks, indexing="ij")).reshape((d,) + tuple(shape))


def grad_hat(uh: np.ndarray) -> np.ndarray:
    """(grad^ u^)[a,k] = 2 pi i k_a u^[k] (Sec. 2.2.1)."""
    K = _kgrid(uh.shape)
    return 2j * np.pi * K * uh[None]


def div_hat(wh: np.ndarray) -> np.ndarray:
    """(grad^* w^)[k] = sum_a -2 pi i k_a w^[a,k] (Sec. 2.2.1)."""
    K = _kgrid(wh.shape[1:])
    return np.sum(-2j * np.pi * K * wh, axis=0)


def precond_inv(shape) -> np.ndarray:
    """Moore–Penrose inverse of P^[k,k] = k.k: 1/(k.k), and 0 at k = 0 (Sec. 2.3)."""
    K = _kgrid(shape)
    kk = np.sum(K.astype(np.float64) ** 2, axis=0)
    out = np.zeros_like(kk)
    nz = kk > 0
    out[nz] = 1.0 / kk[nz]
    return out


def gani_operator(uh: np.ndarray, A: np.ndarray) -> np.ndarray:
    """grad^* F A~ F^{-1} grad^ u^ of Eq. (ls_GaNi_fourier).

    ``A`` holds the grid samples A(x_k): shape (N,)*d for an isotropic coefficient a(x) I, or
    (d, d, N, ..., N) for a full symmetric tensor (stored diagonals of the block-diagonal A~, Sec. 2.2.2).
    """
    d = uh.ndim
    e = idft(grad_hat(uh), d)
    if A.ndim == d:
        w = A[None] * e
    else:
        w = np.einsum("ab...,b...->a...", A, e)
    return div_hat(dft(w, d))


def gani_rhs(A: np.ndarray, E) -> np.ndarray:
    """- grad^* F A~ E of Eq. (ls_GaNi_fourier); E is the constant macroscopic gradient."""
    E = np.asarray(E, dtype=np.float64)
    d = E.shape[0]
    if A.ndim == d:
        AE = A[None] * E.reshape((d,) + (1,) * d)
    else:
        AE = np.einsum("ab...,b->a...", A, E)
    return -div_hat(dft(AE.astype(np.complex128), d))


def _dot(x: np.ndarray, y: np.ndarray) -> float:
    """Real part of the Euclidean inner product of Fourier coefficient arrays (Sec. 4.2 norm)."""
    return float(np.real(np.vdot(x, y)))


def pcg(apply_C, b: np.ndarray, Pinv: np.ndarray, tol: float = 1e-8, maxit: int = 1000):
    """Conjugate gradients on the preconditioned system P^-1 C u = P^-1 b (Eq. (Pls_fourier)).

    CG on the left-preconditioned system in the P-inner product is ordinary PCG with M^-1 = P^-1.
    Starts from u = 0; stops when ||P^-1 r|| <= tol ||P^-1 b|| (the norm of the preconditioned
    residuum, Sec. 4.3) or after ``maxit`` iterations.  Returns (u, iterations, relative residual,
    history of relative residuals).
    """
    u = np.zeros_like(b)
    r = b.copy()
    z = Pinv * r
    nb = np.sqrt(_dot(z, z))
    hist = [1.0]
    if nb == 0.0:
        return u, 0, 0.0, hist
    p = z.copy()
    rz = _dot(r, z)
    it = 0
    rel = 1.0
    while it < maxit:
        q = apply_C(p)
        alpha = rz / _dot(p, q)
        u = u + alpha * p
        r = r - alpha * q
        z = Pinv * r
        it += 1
        rel = np.sqrt(_dot(z, z)) / nb
        hist.append(rel)
        if rel <= tol:
            break
        rz_new = _dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return u, it, rel, hist


def homogenised_coefficient(uh: np.ndarray, A: np.ndarray, E) -> float:
    """A_eff E.E = (1/|N|) sum_k A(x_k)(E + e_k).(E + e_k), e = F^{-1} grad^ u^ (Eq. (homog)).

    The rectangle-rule bilinear form of Sec. 2.2.2 with the cell-average weight 1/|N|.
    """
    E = np.asarray(E, dtype=np.float64)
    d = E.shape[0]
    e = np.real(idft(grad_hat(uh), d))
    f = e + E.reshape((d,) + (1,) * d)
    if A.ndim == d:
        dens = A * np.sum(f * f, axis=0)
    else:
        dens = np.einsum("ab...,a...,b...->...", A, f, f)
    return float(np.mean(dens))


def solve_gani(A: np.ndarray, E, tol: float = 1e-8, maxit: int = 1000):
    """Full-format GaNi solve by PCG: returns dict(Aeff, uh, iters, rel_resid, history)."""
    E = np.asarray(E, dtype=np.float64)
    d = E.shape[0]
    shape = A.shape[-d:]
    b = gani_rhs(A, E)
    Pinv = precond_inv(shape)
    uh, it, rel, hist = pcg(lambda v: gani_operator(v, A), b, Pinv, tol=tol, maxit=maxit)
    return dict(Aeff=homogenised_coefficient(uh, A, E), uh=uh, iters=it, rel_resid=rel, history=hist)
