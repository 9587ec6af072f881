"""Pins of the full-format FP64 oracle against facts that do not come from the oracle itself.

* DFT: the paper's matrices F_N[m,k] = w^{-mk}/|N|, F_N^{-1}[m,k] = w^{mk} written as explicit sums.
* Gradient: the closed-form odd-N spectral differentiation matrix (Trefethen, "Spectral Methods in
  MATLAB", 2000, ch. 3, rescaled from period 2 pi to period 1): D[j,l] = pi (-1)^(j-l) / sin(pi (j-l)/N).
* Solve: a dense direct solve of the GaNi minimisation assembled from that matrix.
* Closed forms: constant coefficient (Sec. 2.2.2: GaNi is exact for constant A), laminates (harmonic /
  arithmetic means), Voigt–Reuss bounds, symmetry of the square inclusion.
"""
import numpy as np
import pytest

from oracle import fourier_galerkin as fg
from synthetic import laminate, lognormal_grf, random_field, square_inclusion


def _dft_matrix(N):
    k = fg.frequencies(N)
    w = np.exp(2j * np.pi / N)
    F = w ** (-np.outer(k, k)) / N
    Finv = w ** (np.outer(k, k))
    return F, Finv


@pytest.mark.parametrize("N", [1, 3, 5, 9, 15, 21, 27, 35, 45, 49])
def test_dft_matches_paper_matrices(N):
    rng = np.random.default_rng(N)
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    F, Finv = _dft_matrix(N)
    assert np.allclose(fg.dft(v, 1), F @ v, atol=1e-14, rtol=0)
    assert np.allclose(fg.idft(v, 1), Finv @ v, atol=1e-12, rtol=0)
    assert np.allclose(fg.idft(fg.dft(v, 1), 1), v, atol=1e-13)
    # Parseval with the paper's scaling: sum |F v|^2 = (1/N) sum |v|^2
    assert np.isclose(np.sum(np.abs(fg.dft(v, 1)) ** 2), np.sum(np.abs(v) ** 2) / N, rtol=1e-13)


def test_dft_2d_3d_separable():
    rng = np.random.default_rng(0)
    for shape in [(5, 7), (3, 5, 7)]:
        v = rng.standard_normal(shape)
        ref = v.astype(np.complex128)
        for ax, n in enumerate(shape):
            F, _ = _dft_matrix(n)
            ref = np.moveaxis(np.tensordot(F, np.moveaxis(ref, ax, 0), axes=([1], [0])), 0, ax)
        assert np.allclose(fg.dft(v, len(shape)), ref, atol=1e-14)


def test_frequencies_and_even_rejected():
    assert list(fg.frequencies(5)) == [0, 1, 2, -2, -1]
    with pytest.raises(ValueError):
        fg.frequencies(4)


def trefethen_D(N):
    """Closed-form odd-N Fourier differentiation matrix on x_j = j/N, period 1."""
    j = np.arange(N)
    m = j[:, None] - j[None, :]
    D = np.zeros((N, N))
    off = m != 0
    D[off] = np.pi * (-1.0) ** m[off] / np.sin(np.pi * m[off] / N)
    return D


@pytest.mark.parametrize("N", [3, 5, 7, 9, 15, 31])
def test_gradient_matches_closed_form_differentiation(N):
    rng = np.random.default_rng(N)
    u = rng.standard_normal(N)
    e = np.real(fg.idft(fg.grad_hat(fg.dft(u, 1)), 1))[0]
    assert np.allclose(e, trefethen_D(N) @ u, atol=1e-11)
    # divergence is the adjoint of the gradient: <grad^ u, w> = <u, grad^* w>
    uh = fg.dft(u, 1)
    wh = fg.dft(rng.standard_normal((1, N)), 1)
    assert np.isclose(np.vdot(fg.grad_hat(uh), wh), np.vdot(uh, fg.div_hat(wh)), atol=1e-14)


def test_gradient_exact_on_trig_polynomial():
    N = 11
    x = fg.grid_points(N)
    X, Y = np.meshgrid(x, x, indexing="ij")
    u = np.sin(2 * np.pi * 3 * X) * np.cos(2 * np.pi * 2 * Y)
    e = np.real(fg.idft(fg.grad_hat(fg.dft(u, 2)), 2))
    assert np.allclose(e[0], 6 * np.pi * np.cos(2 * np.pi * 3 * X) * np.cos(2 * np.pi * 2 * Y), atol=1e-11)
    assert np.allclose(e[1], -4 * np.pi * np.sin(2 * np.pi * 3 * X) * np.sin(2 * np.pi * 2 * Y), atol=1e-11)


def dense_direct(A, E):
    """Minimise (1/|N|) sum_k a_k |E + D u|_k^2 over grid vectors u by a dense least-squares solve."""
    d = A.ndim
    N = A.shape[0]
    D1 = trefethen_D(N)
    I = np.eye(N)
    Ds = []
    for ax in range(d):
        mats = [I] * d
        mats[ax] = D1
        M = mats[0]
        for m in mats[1:]:
            M = np.kron(M, m)
        Ds.append(M)
    a = A.ravel()
    K = sum(Dm.T @ (a[:, None] * Dm) for Dm in Ds)
    b = -sum(Dm.T @ (a * E[i]) for i, Dm in enumerate(Ds))
    u = np.linalg.lstsq(K, b, rcond=1e-13)[0]
    u -= u.mean()
    f = np.stack([E[i] + Ds[i] @ u for i in range(d)])
    return float(np.mean(a * np.sum(f * f, axis=0))), u.reshape(A.shape)


@pytest.mark.parametrize("d,N,kind", [(2, 9, "sq"), (2, 15, "rand"), (2, 13, "grf"), (3, 5, "sq"),
                                      (3, 7, "rand"), (3, 7, "grf")])
def test_pcg_matches_dense_direct_solve(d, N, kind):
    if kind == "sq":
        A = square_inclusion(d, N)[0]
    elif kind == "rand":
        A = random_field((N,) * d, seed=7 + N)
    else:
        A = lognormal_grf(d, N, ell=0.3, seed=11)
    E = np.zeros(d)
    E[0] = 1.0
    ref, u_ref = dense_direct(A, E)
    res = fg.solve_gani(A, E, tol=1e-14, maxit=2000)
    assert abs(res["Aeff"] - ref) <= 1e-12 * ref
    u = np.real(fg.idft(res["uh"], d))
    assert np.abs(u - u_ref).max() <= 1e-9 * max(1.0, np.abs(u_ref).max())


@pytest.mark.parametrize("d,N", [(2, 15), (3, 9)])
def test_constant_coefficient_exact(d, N):
    A = np.full((N,) * d, 3.7)
    E = np.arange(1, d + 1, dtype=np.float64)
    res = fg.solve_gani(A, E)
    assert abs(res["Aeff"] - 3.7 * E @ E) <= 1e-13 * 3.7 * E @ E
    assert np.abs(res["uh"]).max() <= 1e-12  # the right-hand side vanishes: u = 0


@pytest.mark.parametrize("d,N", [(2, 63), (3, 15)])
def test_laminate_harmonic_and_arithmetic_means(d, N):
    A = laminate(d, N, contrast=10.0)[0]
    f = A[(slice(None),) + (0,) * (d - 1)]
    harm = 1.0 / np.mean(1.0 / f)
    arith = np.mean(f)
    E1 = np.eye(d)[0]
    E2 = np.eye(d)[1]
    r1 = fg.solve_gani(A, E1, tol=1e-12)
    r2 = fg.solve_gani(A, E2, tol=1e-12)
    assert abs(r1["Aeff"] - harm) <= 1e-10 * harm
    assert abs(r2["Aeff"] - arith) <= 1e-12 * arith


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_voigt_reuss_bounds(seed):
    d, N = 2, 21
    A = lognormal_grf(d, N, ell=0.15, var=1.0, seed=seed)
    res = fg.solve_gani(A, [1.0, 0.0], tol=1e-10)
    harm = 1.0 / np.mean(1.0 / A)
    assert harm - 1e-12 <= res["Aeff"] <= np.mean(A) + 1e-12
    assert res["Aeff"] < np.mean(A) - 1e-3  # strictly inside for a heterogeneous field


def test_square_inclusion_isotropic_and_symmetric():
    d, N = 2, 31
    A = square_inclusion(d, N)[0]
    r1 = fg.solve_gani(A, [1.0, 0.0], tol=1e-12)["Aeff"]
    r2 = fg.solve_gani(A, [0.0, 1.0], tol=1e-12)["Aeff"]
    r12 = fg.solve_gani(A, [1.0, 1.0], tol=1e-12)["Aeff"]
    assert abs(r1 - r2) <= 1e-10 * r1
    # polarisation: A12 = (A(e1+e2).(e1+e2) - A11 - A22)/2 is 0 by the x1 -> -x1 reflection symmetry
    assert abs(0.5 * (r12 - r1 - r2)) <= 1e-9 * r1


def test_general_field_symmetry_of_tensor():
    d, N = 2, 15
    A = lognormal_grf(d, N, ell=0.2, seed=5)
    vals = {}
    for E in [(1.0, 0.0), (0.0, 1.0), (1.0, 1.0), (1.0, -1.0)]:
        vals[E] = fg.solve_gani(A, E, tol=1e-13)["Aeff"]
    a12_plus = 0.5 * (vals[(1.0, 1.0)] - vals[(1.0, 0.0)] - vals[(0.0, 1.0)])
    a12_minus = -0.5 * (vals[(1.0, -1.0)] - vals[(1.0, 0.0)] - vals[(0.0, 1.0)])
    assert abs(a12_plus - a12_minus) <= 1e-10 * vals[(1.0, 0.0)]


def test_config1_square_63():
    """d=2, N=63, centred square of volume fraction 0.5, phases 1 and 10: 45x45 inclusion nodes."""
    A = square_inclusion(2, 63)[0]
    assert int(np.sum(A > 5)) == 45 * 45
    res = fg.solve_gani(A, [1.0, 0.0], tol=1e-8)
    assert res["rel_resid"] <= 1e-8
    harm = 1.0 / np.mean(1.0 / A)
    assert harm < res["Aeff"] < np.mean(A)


# the constant anisotropic parts of the modified materials of Sec. 4.4 (eigenvalues (1, 10) and (1, 5, 10))
B2 = np.array([[5.5, -4.5], [-4.5, 5.5]])
B3 = np.array([[4.25, -3.25, -1.25 * np.sqrt(2.0)], [-3.25, 4.25, 1.25 * np.sqrt(2.0)],
               [-1.25 * np.sqrt(2.0), 1.25 * np.sqrt(2.0), 7.5]])


def test_anisotropic_parts_have_the_stated_eigenvalues():
    assert np.allclose(np.linalg.eigvalsh(B2), [1.0, 10.0], atol=1e-13)
    assert np.allclose(np.linalg.eigvalsh(B3), [1.0, 5.0, 10.0], atol=1e-13)


def dense_direct_tensor(At, E):
    """Minimise (1/|N|) sum_k (E + D u)_k.A_k (E + D u)_k for a tensor field At (d, d, N..) by a dense
    least-squares solve: K = sum_ab D_a^T diag(A_ab) D_b, b = -sum_ab D_a^T (A_ab E_b)."""
    d = At.shape[0]
    N = At.shape[-1]
    D1 = trefethen_D(N)
    I = np.eye(N)
    Ds = []
    for ax in range(d):
        mats = [I] * d
        mats[ax] = D1
        M = mats[0]
        for m in mats[1:]:
            M = np.kron(M, m)
        Ds.append(M)
    K = sum(Ds[a].T @ (At[a, b].ravel()[:, None] * Ds[b]) for a in range(d) for b in range(d))
    rhs = -sum(Ds[a].T @ (At[a, b].ravel() * E[b]) for a in range(d) for b in range(d))
    u = np.linalg.lstsq(K, rhs, rcond=1e-13)[0]
    u -= u.mean()
    f = np.stack([E[i] + Ds[i] @ u for i in range(d)])
    dens = np.einsum("abk,ak,bk->k", At.reshape(d, d, -1), f, f)
    return float(np.mean(dens)), u.reshape(At.shape[2:])


@pytest.mark.parametrize("d,N", [(2, 9), (2, 13), (3, 5)])
def test_anisotropic_pcg_matches_dense_direct_solve(d, N):
    """The tensor-coefficient path of the full oracle (A~ = a I + B, Sec. 4.4) against a dense direct
    solve of the same minimisation."""
    a = square_inclusion(d, N)[0]
    B = B2 if d == 2 else B3
    At = a[None, None] * np.eye(d).reshape((d, d) + (1,) * d) + B.reshape((d, d) + (1,) * d)
    for E in (np.eye(d)[0], np.ones(d)):
        ref, u_ref = dense_direct_tensor(At, E)
        res = fg.solve_gani(At, E, tol=1e-14, maxit=3000)
        assert abs(res["Aeff"] - ref) <= 1e-12 * ref
        u = np.real(fg.idft(res["uh"], d))
        assert np.abs(u - u_ref).max() <= 1e-9 * max(1.0, np.abs(u_ref).max())


def test_anisotropic_constant_coefficient_exact():
    d, N = 3, 7
    At = 2.0 * np.eye(d).reshape((d, d) + (1,) * d) + B3.reshape((d, d) + (1,) * d) + np.zeros((d, d) + (N,) * d)
    E = np.array([1.0, -2.0, 0.5])
    res = fg.solve_gani(At, E)
    ref = float(E @ (2.0 * np.eye(d) + B3) @ E)
    assert abs(res["Aeff"] - ref) <= 1e-13 * ref
