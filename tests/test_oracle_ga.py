"""Pins of the Ga oracle (exact integration on the double grid, Sec. 2.2.3) against routes that do not use it:
Gauss-Legendre quadrature of the pixel-wise constant coefficient against the closed-form Dirichlet kernel,
a dense Galerkin solve assembled from quadrature Fourier coefficients (K[l,k] = 4 pi^2 (k.l) A^(k - l)),
closed forms (constant coefficient, laminate along its layers) and the variational bounds of a Galerkin
method on nested spaces."""
import numpy as np
import pytest

from oracle import fourier_galerkin as fg
from oracle import galerkin_exact as ga
from oracle import lowrank as lr
from synthetic import random_field, smoothed_cube, square_inclusion

GL_X, GL_W = np.polynomial.legendre.leggauss(12)


def cell_nodes(N):
    """Gauss-Legendre nodes and weights on every cell [x_p - 1/(2N), x_p + 1/(2N)] (1D), per cell."""
    xs = fg.grid_points(N)
    h = 0.5 / N
    return xs[:, None] + h * GL_X[None, :], h * GL_W


def dirichlet(t, M):
    """D_M(t) = sum_{m in Z_M} e^{2 pi i m t} = sin(M pi t) / sin(pi t) (M at integer t), M odd."""
    t = np.asarray(t, dtype=np.float64)
    s = np.sin(np.pi * t)
    out = np.full(t.shape, float(M))
    nz = np.abs(s) > 1e-14
    out[nz] = np.sin(M * np.pi * t[nz]) / s[nz]
    return out


def quad_fourier(a, m):
    """A^(m) = int a e^{2 pi i m.x} dx by cell-wise Gauss-Legendre quadrature (d = 2)."""
    N = a.shape[0]
    X, W = cell_nodes(N)
    f0 = (np.exp(2j * np.pi * m[0] * X) * W[None]).sum(axis=1)  # per cell, axis 0
    f1 = (np.exp(2j * np.pi * m[1] * X) * W[None]).sum(axis=1)
    return np.sum(a * np.outer(f0, f1))


def test_coefficient_sums_to_the_mean():
    a = random_field((7, 7), seed=3)
    At = ga.ga_coefficient(a)
    assert At.shape == (13, 13)
    assert abs(At.sum() - a.mean()) <= 1e-14 * a.mean()


def test_coefficient_matches_quadrature_of_the_dirichlet_kernel():
    """A~[j] = int a phi^j_M with phi^j_M(x) = |M|^-1 prod_a D_M(x_a - x^j_a), integrated cell by cell."""
    N = 5
    M = 2 * N - 1
    a = random_field((N, N), seed=4)
    At = ga.ga_coefficient(a)
    X, W = cell_nodes(N)
    xj = fg.grid_points(M)
    ref = np.zeros((M, M))
    for j0 in range(M):
        g0 = (dirichlet(X - xj[j0], M) * W[None]).sum(axis=1)
        for j1 in range(M):
            g1 = (dirichlet(X - xj[j1], M) * W[None]).sum(axis=1)
            ref[j0, j1] = np.sum(a * np.outer(g0, g1)) / M ** 2
    assert np.abs(At - ref).max() <= 1e-13 * np.abs(ref).max()
    Ah = ga.pixel_fourier(a, M)
    ks = fg.frequencies(M)
    for i0, i1 in [(0, 0), (1, 3), (4, 8), (7, 2)]:
        assert abs(Ah[i0, i1] - quad_fourier(a, (ks[i0], ks[i1]))) <= 1e-13 * abs(Ah[0, 0])


def dense_galerkin(a, E, B=None):
    """Minimise int (E + grad u).(a I + B)(E + grad u) over u in T_N by the dense Galerkin system with quadrature
    A^(k - l); a constant B adds 4 pi^2 l.B k on the diagonal (k = l) and E.B E to the energy."""
    N = a.shape[0]
    ks = fg.frequencies(N)
    K2 = [(k0, k1) for k0 in ks for k1 in ks if (k0, k1) != (0, 0)]
    n = len(K2)
    K = np.zeros((n, n), dtype=np.complex128)
    rhs = np.zeros(n, dtype=np.complex128)
    cache = {}

    def Ahat(m):
        if m not in cache:
            cache[m] = quad_fourier(a, m)
        return cache[m]

    for i, l in enumerate(K2):
        for j, k in enumerate(K2):
            K[i, j] = 4 * np.pi ** 2 * (k[0] * l[0] + k[1] * l[1]) * Ahat((k[0] - l[0], k[1] - l[1]))
            if B is not None and i == j:
                K[i, j] += 4 * np.pi ** 2 * (np.array(l) @ B @ np.array(k))
        rhs[i] = 2j * np.pi * (E[0] * l[0] + E[1] * l[1]) * Ahat((-l[0], -l[1]))
    u = np.linalg.solve(K, rhs)
    eBe = 0.0 if B is None else float(E @ B @ E)
    return float(np.real(Ahat((0, 0)) * (E @ E) + eBe - np.vdot(u, K @ u)))


@pytest.mark.parametrize("N,seed", [(5, 1), (7, 2)])
def test_ga_solve_matches_dense_galerkin(N, seed):
    a = random_field((N, N), seed=seed)
    for E in (np.array([1.0, 0.0]), np.array([0.3, -1.2])):
        ref = dense_galerkin(a, E)
        res = ga.solve_ga(a, E, tol=1e-14, maxit=2000)
        assert abs(res["Aeff"] - ref) <= 1e-10 * ref


def test_constant_coefficient_exact():
    a = np.full((9, 9, 9), 2.5)
    E = np.array([1.0, 2.0, -1.0])
    res = ga.solve_ga(a, E)
    assert abs(res["Aeff"] - 2.5 * E @ E) <= 1e-13 * 2.5 * E @ E
    assert np.abs(res["uh"]).max() <= 1e-12


def test_laminate_along_layers_is_the_mean():
    N = 15
    f = 1.0 + 9.0 * (np.abs(fg.grid_points(N)) < 0.25)
    a = np.outer(f, np.ones(N))
    res = ga.solve_ga(a, [0.0, 1.0], tol=1e-12)
    assert abs(res["Aeff"] - a.mean()) <= 1e-12 * a.mean()


def refine(a, q):
    """The same pixel material on the solution grid q N (q odd): each cell split into q^d sub-cells."""
    N = a.shape[0]
    kf = fg.frequencies(q * N)
    kc = np.rint(kf / q).astype(int) % N
    return a[np.ix_(*([kc] * a.ndim))]


def test_galerkin_bounds_on_nested_spaces():
    """T_N is contained in T_3N and the bilinear form is integrated exactly, so A_eff(3N) <= A_eff(N); every
    Galerkin value lies above the Reuss bound and below the Voigt bound of the pixel material."""
    a = random_field((5, 5), seed=9)
    E = np.array([1.0, 0.0])
    coarse = ga.solve_ga(a, E, tol=1e-13)["Aeff"]
    fine = ga.solve_ga(refine(a, 3), E, tol=1e-13)["Aeff"]
    assert fine <= coarse * (1 + 1e-12)
    assert coarse - fine > 1e-6 * coarse  # the bigger space lowers the energy
    harm = 1.0 / np.mean(1.0 / a)
    assert harm <= fine and coarse <= a.mean()


def test_tt_modified_coefficient_matches_the_full_one():
    """The mode-wise (dense matrix) route of the TT Ga coefficient against the FFT route of the full one."""
    N = 9
    a, terms, w = smoothed_cube(3, N, contrast=10.0)
    op = lr.LowRankGaTT(lr.tt_from_separable(terms, w), (N,) * 3, rank=None)
    ref = ga.ga_coefficient(a)
    assert np.abs(lr.tt_full(op.At) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("d,N", [(2, 13), (3, 9)])
def test_untruncated_tt_ga_equals_full_ga(d, N):
    """Untruncated TT Ga MinRes reaches the full-format Ga solution (pinned above) to 1e-10."""
    a, terms, w = square_inclusion(d, N)
    E = np.eye(d)[0]
    full = ga.solve_ga(a, E, tol=1e-13, maxit=3000)
    op = lr.LowRankGaTT(lr.tt_from_separable(terms, w), (N,) * d, rank=None, rank_tol=1e-15)
    out = lr.minres(op, E, tol=1e-13, maxit=600, stop_on_increase=False)
    assert abs(out["Aeff"] - full["Aeff"]) <= 1e-10 * full["Aeff"]


@pytest.mark.parametrize("fmt,d,N", [("tucker", 3, 9), ("tucker", 2, 13), ("cp", 2, 13)])
def test_tucker_cp_modified_coefficient_matches_the_full_one(fmt, d, N):
    """The modified coefficient formed factor by factor (Tucker, CP) against the FFT route of the full one."""
    a, terms, w = smoothed_cube(d, N, contrast=10.0)
    a_lr = lr.tucker_from_separable(terms, w) if fmt == "tucker" else lr.cp_from_separable(terms, w)
    op = lr.LowRankGa(a_lr, (N,) * d, rank=None, fmt=fmt)
    ref = ga.ga_coefficient(a)
    assert np.abs(np.real(op.f.full(op.At)) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("fmt,d,N", [("tucker", 2, 13), ("tucker", 3, 9), ("cp", 2, 13)])
def test_untruncated_tucker_cp_ga_equals_full_ga(fmt, d, N):
    """Untruncated Tucker / CP Ga MinRes reaches the full-format Ga solution (pinned above) to 1e-10."""
    a, terms, w = square_inclusion(d, N)
    E = np.eye(d)[0]
    full = ga.solve_ga(a, E, tol=1e-13, maxit=3000)
    a_lr = lr.tucker_from_separable(terms, w) if fmt == "tucker" else lr.cp_from_separable(terms, w)
    op = lr.LowRankGa(a_lr, (N,) * d, rank=None, rank_tol=1e-15, fmt=fmt)
    out = lr.minres(op, E, tol=1e-13, maxit=600, stop_on_increase=False)
    assert abs(out["Aeff"] - full["Aeff"]) <= 1e-10 * full["Aeff"]


@pytest.mark.parametrize("fmt,N", [("tt", 5), ("tt", 7), ("tucker", 7), ("cp", 5)])
def test_untruncated_lowrank_ga_with_anisotropy_matches_dense_galerkin(fmt, N):
    """Low-rank Ga with a constant anisotropic part B (A~ = a~ I + B 1~), untruncated, against the dense
    Galerkin solve of the anisotropic material assembled from quadrature (d = 2)."""
    a, terms, w = square_inclusion(2, N)
    B = np.array([[0.7, 0.25], [0.25, 0.4]])
    a_lr = {"tt": lr.tt_from_separable, "tucker": lr.tucker_from_separable, "cp": lr.cp_from_separable}[fmt](terms, w)
    op = lr.LowRankGa(a_lr, (N, N), rank=None, rank_tol=1e-15, fmt=fmt, B=B)
    for E in (np.array([1.0, 0.0]), np.array([0.3, -1.2])):
        ref = dense_galerkin(a, E, B)
        out = lr.minres(op, E, tol=1e-13, maxit=600, stop_on_increase=False)
        assert abs(out["Aeff"] - ref) <= 1e-10 * ref, (out["Aeff"], ref)
    # B changes the answer (the pin is not vacuous)
    assert abs(dense_galerkin(a, np.array([1.0, 0.0])) - dense_galerkin(a, np.array([1.0, 0.0]), B)) > 0.1
