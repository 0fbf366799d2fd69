"""Pins of the two-sided Petrov-Galerkin recycle update (the reading of the
RBiCG generator): exact invariant subspaces inside the search spaces are
recovered exactly, with their eigenvalues, on both sides; and for a
symmetric matrix with W~ = W the two sides coincide (Rayleigh-Ritz)."""
import numpy as np

from oracle.dense import principal_cosines
from oracle.recycle_two_sided import petrov_galerkin_update


def test_recovers_exact_left_and_right_eigenvectors():
    rng = np.random.default_rng(11)
    n, k = 30, 3
    lam = np.concatenate([[0.1, 0.2, 0.3], np.linspace(5.0, 10.0, n - k)])
    V = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    Vi = np.linalg.inv(V)
    A = V @ np.diag(lam) @ Vi
    R, L = V[:, :k], Vi[:k, :].T                      # right and left eigenvectors
    W = np.column_stack([R, rng.standard_normal((n, 6))]) @ rng.standard_normal((k + 6, k + 6))
    Wt = np.column_stack([L, rng.standard_normal((n, 6))]) @ rng.standard_normal((k + 6, k + 6))
    U, Ut, th = petrov_galerkin_update(A, W, Wt, k)
    assert U.shape[1] == Ut.shape[1] == k
    assert np.allclose(np.sort(th.real), lam[:k], rtol=1e-9) and np.all(np.abs(th.imag) <= 1e-9)
    assert np.min(principal_cosines(U, R)) >= 1 - 1e-10
    assert np.min(principal_cosines(Ut, L)) >= 1 - 1e-10


def test_symmetric_matrix_two_sides_coincide():
    rng = np.random.default_rng(12)
    n, m, k = 40, 10, 4
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    W = rng.standard_normal((n, m))
    U, Ut, th = petrov_galerkin_update(A, W, W, k)
    assert np.all(np.abs(th.imag) <= 1e-12 * np.abs(th.real))
    assert np.min(principal_cosines(U, Ut)) >= 1 - 1e-10
    # Rayleigh-Ritz: the smallest Ritz values of A on range(W)
    Q, _ = np.linalg.qr(W)
    ritz = np.sort(np.linalg.eigvalsh(Q.T @ A @ Q))[:k]
    assert np.allclose(np.sort(th.real), ritz, rtol=1e-10)
