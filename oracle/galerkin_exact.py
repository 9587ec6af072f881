"""Fourier–Galerkin method with exact integration (Ga) in full format, FP64 — test infrastructure only.

Restates Sec. 2.2.3 of arXiv:1902.07455 in plain NumPy for a pixel-wise constant coefficient: a(x) = a_p on the
cell of side 1/N centred at the grid point x_p (p in Z_N^d), the image-based composite with coefficients
constant over pixels that the paper lists among the materials whose integrals are exact.

Double grid integration with projection (DoGIP), M = 2N - 1 per axis:
* modified coefficient on the double grid, A~[j] = int_Y a(x) phi^j_M(x) dx, with phi^j_M the fundamental
  trigonometric polynomial of T_M at x^j_M = j/M (phi^j_M(x^l_M) = delta_jl);
* zero-padding injection I from the frequencies Z_N to Z_M and its adjoint I* (projection on Z_N);
* the linear system Eq. (ls_Ga_fourier):
      grad^*_N I* F_M A~ F_M^{-1} I grad^_N u^ = - grad^*_N I* F_M A~ E,
  preconditioned by the same Fourier Laplacian as GaNi (Sec. 2.3) and solved by PCG;
* A_eff E.E = int_Y a |E + grad u|^2 dx = sum_j A~[j] |E + e(x^j_M)|^2 — exact, because |E + grad u|^2
  lies in T_M when u lies in T_N.

The integrals: with A^(m) = int_Y a(x) e^{2 pi i m.x} dx = abar(m) prod_a s(m_a), abar(m) = sum_p a_p
e^{2 pi i m.x_p} and s(m) = sin(pi m / N) / (pi m) (s(0) = 1/N), the definition of phi^j_M,
phi^j_M(x) = |M|^-1 sum_{m in Z_M} e^{2 pi i m.(x - x^j_M)}, gives A~[j] = |M|^-1 sum_m e^{-2 pi i m.x^j_M} A^(m).

Conventions as in ``oracle.fourier_galerkin`` (storage order, F normalised by 1/|N|, F^-1 not).
"""
from __future__ import annotations

import numpy as np

from . import fourier_galerkin as fg

__all__ = ["pixel_fourier", "ga_coefficient", "inject", "project", "ga_operator", "ga_rhs",
           "homogenised_coefficient_ga", "solve_ga"]


def _sinc_cell(m: np.ndarray, N: int) -> np.ndarray:
    """s(m) = int_{-1/(2N)}^{1/(2N)} e^{2 pi i m t} dt = sin(pi m / N) / (pi m), 1/N at m = 0."""
    m = np.asarray(m, dtype=np.float64)
    out = np.full(m.shape, 1.0 / N)
    nz = m != 0
    out[nz] = np.sin(np.pi * m[nz] / N) / (np.pi * m[nz])
    return out


def pixel_fourier(a: np.ndarray, M: int) -> np.ndarray:
    """A^(m) = int_Y a(x) e^{2 pi i m.x} dx for m in Z_M^d (storage order), a pixel-wise constant on the
    N^d cells centred at the grid points."""
    d = a.ndim
    N = a.shape[0]
    abar_N = np.fft.ifftn(a) * float(N) ** d        # abar(m) for m in Z_N, periodic in m with period N
    ms = fg.frequencies(M)
    idx = np.ix_(*([ms % N] * d))
    abar = abar_N[idx]
    S = np.ones((M,) * d)
    for ax in range(d):
        shape = [1] * d
        shape[ax] = M
        S = S * _sinc_cell(ms, N).reshape(shape)
    return abar * S


def ga_coefficient(a: np.ndarray) -> np.ndarray:
    """A~[j] = int_Y a phi^j_M dx on the double grid M = 2N - 1 (storage order), real."""
    d = a.ndim
    M = 2 * a.shape[0] - 1
    Ah = pixel_fourier(a, M)
    At = np.fft.fftn(Ah) / float(M) ** d              # |M|^-1 sum_m e^{-2 pi i m j / M} A^(m)
    if np.abs(At.imag).max() > 1e-12 * max(1.0, np.abs(At.real).max()):
        raise ValueError("modified coefficient is not real")
    return At.real


def inject(vh: np.ndarray, M: int, d: int) -> np.ndarray:
    """Zero padding I: coefficients on Z_N (last d axes) placed at the same frequencies of Z_M."""
    N = vh.shape[-1]
    out = np.zeros(vh.shape[:-d] + (M,) * d, dtype=np.complex128)
    kN = fg.frequencies(N)
    idx_out = np.ix_(*([kN % M] * d))
    out[(Ellipsis,) + idx_out] = vh
    return out


def project(wh: np.ndarray, N: int, d: int) -> np.ndarray:
    """Adjoint I*: the coefficients of the frequencies Z_N out of Z_M (last d axes)."""
    M = wh.shape[-1]
    kN = fg.frequencies(N)
    idx = np.ix_(*([kN % M] * d))
    return wh[(Ellipsis,) + idx]


def ga_operator(uh: np.ndarray, At: np.ndarray) -> np.ndarray:
    """grad^*_N I* F_M A~ F_M^{-1} I grad^_N u^ of Eq. (ls_Ga_fourier)."""
    d = uh.ndim
    N = uh.shape[0]
    M = At.shape[0]
    e = fg.idft(inject(fg.grad_hat(uh), M, d), d)    # gradient values on the double grid
    w = At[None] * e
    return fg.div_hat(project(fg.dft(w, d), N, d))


def ga_rhs(At: np.ndarray, E, N: int) -> np.ndarray:
    """- grad^*_N I* F_M A~ E of Eq. (ls_Ga_fourier)."""
    E = np.asarray(E, dtype=np.float64)
    d = E.shape[0]
    AE = At[None] * E.reshape((d,) + (1,) * d)
    return -fg.div_hat(project(fg.dft(AE.astype(np.complex128), d), N, d))


def homogenised_coefficient_ga(uh: np.ndarray, At: np.ndarray, E) -> float:
    """A_eff E.E = sum_j A~[j] |E + e(x^j_M)|^2 (exact integration of a |E + grad u|^2)."""
    E = np.asarray(E, dtype=np.float64)
    d = E.shape[0]
    M = At.shape[0]
    e = np.real(fg.idft(inject(fg.grad_hat(uh), M, d), d))
    f = e + E.reshape((d,) + (1,) * d)
    return float(np.sum(At * np.sum(f * f, axis=0)))


def solve_ga(a: np.ndarray, E, tol: float = 1e-8, maxit: int = 1000):
    """Ga solve by PCG with the Laplacian preconditioner: dict(Aeff, uh, iters, rel_resid, At)."""
    E = np.asarray(E, dtype=np.float64)
    d = E.shape[0]
    N = a.shape[0]
    At = ga_coefficient(a)
    b = ga_rhs(At, E, N)
    Pinv = fg.precond_inv((N,) * d)
    uh, it, rel, hist = fg.pcg(lambda v: ga_operator(v, At), b, Pinv, tol=tol, maxit=maxit)
    return dict(Aeff=homogenised_coefficient_ga(uh, At, E), uh=uh, iters=it, rel_resid=rel, At=At, history=hist)
