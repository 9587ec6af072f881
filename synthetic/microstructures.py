"""Microstructure generators on the periodic cell Y = (-1/2, 1/2)^d, sampled at x_k = k/N.

Storage order along each axis: index i holds grid point k/N with k = i for i <= (N-1)/2 and k = i - N
otherwise (the usual DFT order, N odd).  Every generator is deterministic given its arguments; random
ones take an explicit seed (NumPy PCG64).

Workloads (recipes, with the paper's materials as the pattern, Sec. 4.1):
* ``square_inclusion``: centred square/cube of volume fraction vf with phases (p0 matrix, p1 inclusion);
  separable: a = p0 * 1x..x1 + (p1 - p0) * chi x .. x chi  (rank 2, as the paper notes for its
  inclusion material).
* ``smoothed_cube``: a = 1 + (contrast - 1) prod_a h(x_a), h(t) = (tanh((t+c)/w) - tanh((t-c)/w))/2.
* ``laminate``: a(x) = f(x_1), rank 1.
* ``smoothed_sphere``: a = 1 + (contrast - 1) (1 - tanh((|x| - R)/w))/2 (not separable).
* ``lognormal_grf``: a = exp(g), g a periodic Gaussian random field with squared-exponential covariance
  sigma^2 exp(-|x-y|^2 / (2 l^2)), realised through its spectral density
  lambda_k ~ prod_a exp(-2 pi^2 l^2 k_a^2) normalised to sum_k lambda_k = sigma^2 (modes with
  lambda_k < 1e-16 max dropped).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 19020745


def _k(N: int) -> np.ndarray:
    if N % 2 != 1:
        raise ValueError("odd N only")
    k = np.arange(N, dtype=np.int64)
    k[k > (N - 1) // 2] -= N
    return k


def grid_points(N: int) -> np.ndarray:
    return _k(N) / N


def _outer(vecs):
    out = vecs[0]
    for v in vecs[1:]:
        out = np.multiply.outer(out, v)
    return out


def square_inclusion(d: int, N: int, vf: float = 0.5, phases=(1.0, 10.0)):
    """Centred square (d=2) / cube (d=3) of volume fraction ``vf``: half side h = vf^(1/d)/2.
    Returns (a_full, terms, weights) with a = sum_i weights[i] * outer(terms[i])."""
    h = vf ** (1.0 / d) / 2.0
    x = grid_points(N)
    chi = (np.abs(x) < h).astype(np.float64)
    one = np.ones(N)
    p0, p1 = float(phases[0]), float(phases[1])
    terms = [[one] * d, [chi] * d]
    weights = [p0, p1 - p0]
    a = p0 + (p1 - p0) * _outer([chi] * d)
    return a, terms, weights


def smoothed_cube(d: int, N: int, contrast: float = 100.0, c: float = 0.3, width=None, full: bool = True):
    """a = 1 + (contrast-1) prod_a h(x_a) with a tanh-smoothed indicator of |t| < c, width 2/N by
    default.  Returns (a_full, terms, weights); a_full is None when full=False (large N)."""
    w = 2.0 / N if width is None else float(width)
    x = grid_points(N)
    h = 0.5 * (np.tanh((x + c) / w) - np.tanh((x - c) / w))
    one = np.ones(N)
    terms = [[one] * d, [h] * d]
    weights = [1.0, contrast - 1.0]
    a = 1.0 + (contrast - 1.0) * _outer([h] * d) if full else None
    return a, terms, weights


def laminate(d: int, N: int, contrast: float = 10.0, c: float = 0.25, full: bool = True):
    """Layered medium a(x) = 1 + (contrast-1) [|x_1| < c].  Returns (a_full, terms, weights); a_full is
    None when full=False (large N)."""
    x = grid_points(N)
    f = 1.0 + (contrast - 1.0) * (np.abs(x) < c)
    one = np.ones(N)
    terms = [[f] + [one] * (d - 1)]
    a = _outer([f] + [one] * (d - 1)) if full else None
    return a, terms, [1.0]


def smoothed_sphere(d: int, N: int, contrast: float = 10.0, radius: float = 0.3, width=None):
    """a = 1 + (contrast-1) s(|x|), s a tanh-smoothed indicator of the ball |x| < radius (width 2/N by
    default, distances periodic on the cell).  Returns the full grid array (not separable)."""
    w = 2.0 / N if width is None else float(width)
    x = grid_points(N)
    r2 = np.zeros((N,) * d)
    for a in range(d):
        shape = [1] * d
        shape[a] = N
        r2 = r2 + (x ** 2).reshape(shape)
    s = 0.5 * (1.0 - np.tanh((np.sqrt(r2) - radius) / w))
    return 1.0 + (contrast - 1.0) * s


def lognormal_grf(d: int, N: int, ell: float = 0.2, var: float = 1.0, seed: int = BASE_SEED,
                  mean: float = 0.0):
    """a = exp(g) with g a seeded periodic Gaussian random field of squared-exponential covariance
    (correlation length ``ell``, variance ``var``).  Returns the full grid array."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = _k(N).astype(np.float64)
    lam1 = np.exp(-2.0 * np.pi ** 2 * ell ** 2 * k ** 2)
    lam = _outer([lam1] * d)
    lam[lam < 1e-16 * lam.max()] = 0.0
    lam *= var / lam.sum()
    white = rng.standard_normal((N,) * d)
    wh = np.fft.fftn(white)                      # Hermitian, E|wh_k|^2 = N^d
    g = np.real(np.fft.ifftn(wh * np.sqrt(lam * N ** d)))
    return np.exp(mean + g)


def random_field(shape, seed: int = BASE_SEED, low: float = 1.0, high: float = 10.0):
    """Uniform random positive coefficient on the grid (for operator tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(low, high, size=tuple(shape))


def random_tt(shape, ranks, seed: int = BASE_SEED, scale: float = 1.0):
    """Random real TT carriages (r_{j-1}, N_j, r_j), entries N(0, scale^2 / r_{j-1})."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = len(shape)
    rr = [1] + list(ranks) + [1]
    if len(rr) != d + 1:
        raise ValueError("need d-1 interior ranks")
    return [rng.standard_normal((rr[j], shape[j], rr[j + 1])) * scale / np.sqrt(rr[j]) for j in range(d)]
