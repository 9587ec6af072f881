"""The symmetric eigensolver inside every truncation (lrfg_sym_eig: the k largest eigenpairs of the Gram cores of
the Gram-SVD rounding, App. A.3.3) against LAPACK's (numpy.linalg.eigh).

Eigenvalues agree within c n eps ||A||; the returned vectors are orthonormal to 1e-12 and have residuals
||A v - w v|| within c n eps ||A||; where an eigenvalue is separated from its neighbours by more than 1e-3 ||A||
its vector matches LAPACK's up to sign.  Inputs: Gaussian symmetric matrices (both signs), Gram-like positive
semidefinite matrices with geometric spectra down to 1e-16, rank-deficient Gram matrices (a cluster of exact
zeros), repeated eigenvalues, diagonal matrices (nothing to reduce) and the zero matrix."""
import numpy as np
import pytest

import paper_1902_07455_gb300 as lrfg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS = np.finfo(np.float64).eps


def _orth(n, rng):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def _matrix(kind, n, rng):
    if kind == "gauss":
        a = rng.standard_normal((n, n))
        return 0.5 * (a + a.T)
    if kind == "graded":
        q = _orth(n, rng)
        return (q * 10.0 ** (-16.0 * np.arange(n) / max(n, 1))) @ q.T
    if kind == "lowrank":
        b = rng.standard_normal((n, max(1, n // 3)))
        return b @ b.T
    if kind == "repeated":
        q = _orth(n, rng)
        lam = np.repeat([3.0, 1.0, 0.25, 0.0], (n + 3) // 4)[:n]
        return (q * lam) @ q.T
    if kind == "diagonal":
        return np.diag(rng.permutation(np.linspace(-1.0, 2.0, n)))
    if kind == "zero":
        return np.zeros((n, n))
    raise ValueError(kind)


def _check(A, w, V, k):
    n = A.shape[0]
    anorm = max(np.linalg.norm(A, 2), 1e-300)
    ref = np.linalg.eigh(A)
    lam = ref[0][::-1][:k]
    tol = 64 * n * EPS * anorm
    assert np.all(np.abs(w - lam) <= tol), (np.max(np.abs(w - lam)) / anorm, n, k)
    assert np.all(np.diff(w) <= tol)  # descending
    assert np.max(np.abs(V.T @ V - np.eye(k))) <= 1e-12
    res = np.linalg.norm(A @ V - V * w, axis=0)
    assert np.all(res <= tol), (np.max(res) / anorm, n, k)
    # isolated eigenvalues: the vector itself, up to sign
    full = ref[0][::-1]
    U = ref[1][:, ::-1]
    for t in range(k):
        gap = min(abs(full[t] - full[s]) for s in range(n) if s != t) if n > 1 else np.inf
        if gap > 1e-3 * anorm:
            assert abs(abs(U[:, t] @ V[:, t]) - 1.0) <= 1e-10, (t, n, k)


@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (3, 2), (5, 5), (17, 9), (30, 20), (32, 32), (33, 20), (45, 30),
                                 (60, 20), (64, 32), (64, 1), (100, 20), (80, 40)])
@pytest.mark.parametrize("kind", ["gauss", "graded", "lowrank", "repeated", "diagonal", "zero"])
def test_sym_eig_matches_lapack(ctx, n, k, kind):
    rng = np.random.default_rng(1000 * n + k)
    As = np.stack([_matrix(kind, n, rng) for _ in range(3)])
    w, V = ctx.sym_eig(torch.as_tensor(As, device="cuda"), k)
    w, V = w.cpu().numpy(), V.cpu().numpy()
    for b in range(3):
        _check(As[b], w[b], V[b], k)


def test_sym_eig_batch_items_are_independent(ctx):
    # each item alone gives the same result as inside a batch of unlike matrices
    rng = np.random.default_rng(7)
    As = np.stack([_matrix("graded", 60, rng), _matrix("lowrank", 60, rng), _matrix("gauss", 60, rng)])
    w, V = ctx.sym_eig(torch.as_tensor(As, device="cuda"), 20)
    for b in range(3):
        w1, V1 = ctx.sym_eig(torch.as_tensor(As[b], device="cuda"), 20)
        assert torch.equal(w1, w[b]) and torch.equal(V1, V[b])


def test_sym_eig_rejects_bad_sizes(ctx):
    with pytest.raises(lrfg.LrfgError):
        ctx.sym_eig(torch.zeros((4, 0, 0), dtype=torch.float64, device="cuda"), 1)
    with pytest.raises(lrfg.LrfgError):
        ctx.sym_eig(torch.eye(4, dtype=torch.float64, device="cuda"), 0)
