"""Pins of the Alg. 1 (RBiCG) oracle against what the paper and the
mathematics fix: the solutions of the primary and dual systems (dense LU),
the residual identity of the final correction for both systems, the bi-orthogonality of
the BiCG residuals (the bi-Lanczos relations of Sec. 2), the orthogonality
of the residuals to the recycle space (Sec. 3), the reduction to CG for a
symmetric positive definite matrix with b~ = b and k = 0 (a library
routine), and finite termination after n - k steps when U, U~ span exact
invariant subspaces of A, A^T."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import rbicg as orc
from oracle import rbicgstab as orb
from paper_1406_2831_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _problem(N=12, p=10.0, k=0, seed=3):
    A = inputs.conv_diff_2d(N, p).to_scipy()
    b = inputs.gaussian_rhs(A.shape[0], seed)
    bt = inputs.gaussian_rhs(A.shape[0], seed + 50)
    rec = orb.recycle_setup(A, inputs.random_recycle_basis(A.shape[0], k, seed + 7)) if k else None
    return A, b, bt, rec


@pytest.mark.parametrize("k", [0, 6])
def test_rbicg_solves_primary_and_dual(k):
    A, b, bt, rec = _problem(k=k)
    x, xt, info = orc.rbicg(A, b, bt, rec, tol=1e-11)
    D = A.toarray()
    assert info.status == orc.OK
    assert _rel(x, sla.solve(D, b)) <= 1e-8
    assert _rel(xt, sla.solve(D.T, bt)) <= 1e-8
    assert info.relres <= 1e-11 and info.relres_dual <= 1e-11


@pytest.mark.parametrize("k", [0, 6])
def test_rbicg_residual_identity_of_step7(k):
    """b - A (x_i - U zeta_c) = r_i and b~ - A^T (x~_i - U~ zeta~_c) = r~_i at
    every iterate: pins the signs of the updates and of the final correction in both columns."""
    A, b, bt, rec = _problem(k=k)
    U = rec.U if rec else np.zeros((A.shape[0], 0))
    Ut = rec.Ut if rec else U
    _, _, info = orc.rbicg(A, b, bt, rec, tol=1e-10, record=True)
    for x, zc, r, xt, ztc, rt in info.iterates:
        assert np.linalg.norm(b - A @ (x - U @ zc) - r) <= 1e-10 * np.linalg.norm(b)
        assert np.linalg.norm(bt - A.T @ (xt - Ut @ ztc) - rt) <= 1e-10 * np.linalg.norm(bt)


@pytest.mark.parametrize("k", [0, 4])
def test_rbicg_residuals_biorthogonal(k):
    """(r~_j, r_i) = 0 for i != j (bi-Lanczos) on a small well-conditioned
    system, over the first iterations."""
    A, b, bt, rec = _problem(N=8, p=3.0, k=k)
    _, _, info = orc.rbicg(A, b, bt, rec, tol=1e-14, max_itn=8, record=True)
    R = info.residuals
    for i in range(len(R)):
        for j in range(len(R)):
            if i != j:
                ri, rtj = R[i][0], R[j][1]
                assert abs(np.dot(rtj, ri)) <= 1e-9 * np.linalg.norm(rtj) * np.linalg.norm(ri), (i, j)


def test_rbicg_residuals_orthogonal_to_recycle_space():
    """C~^T r_i = 0 and C^T r~_i = 0 for every i (eq. (3.5) starts them there
    and the projected products keep them there)."""
    A, b, bt, rec = _problem(k=6)
    _, _, info = orc.rbicg(A, b, bt, rec, tol=1e-10, record=True)
    for r, rt in info.residuals:
        assert np.linalg.norm(rec.Ct.T @ r) <= 1e-10 * np.linalg.norm(rec.Ct) * np.linalg.norm(b)
        assert np.linalg.norm(rec.C.T @ rt) <= 1e-10 * np.linalg.norm(rec.C) * np.linalg.norm(bt)


def test_rbicg_is_cg_for_spd_with_equal_right_hand_sides():
    """k = 0, A symmetric positive definite, b~ = b: BiCG's primary iterates
    are CG's (compared with SciPy's CG, iterate by iterate)."""
    N = 14
    T = sp.diags([-np.ones(N - 1), 2.0 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    A = (sp.kron(sp.identity(N), T) + sp.kron(T, sp.identity(N))).tocsr()
    b = inputs.gaussian_rhs(A.shape[0], 9)
    ref = []
    spla.cg(A, b, rtol=1e-30, atol=0.0, maxiter=12, callback=lambda xk: ref.append(xk.copy()))
    _, _, info = orc.rbicg(A, b, b.copy(), None, tol=1e-30, max_itn=12, record=True)
    assert len(info.iterates) == len(ref) == 12
    for (x, *_), xr in zip(info.iterates, ref):
        assert _rel(x, xr) <= 1e-10


def test_rbicg_exact_deflation_terminates_after_n_minus_k():
    """A = V diag(lambda) V^{-1} with distinct real eigenvalues; U = k right
    and U~ = k left eigenvectors.  The projected iteration then works on the
    remaining n - k eigenvalues and terminates after n - k steps; without
    recycling it needs n."""
    rng = np.random.default_rng(5)
    n, k = 24, 6
    V = np.eye(n) + 0.2 * rng.standard_normal((n, n))
    lam = np.linspace(1.0, 6.0, n)
    A = sp.csr_matrix(V @ np.diag(lam) @ np.linalg.inv(V))
    Winv = np.linalg.inv(V)
    U = V[:, :k]
    Ut = Winv[:k, :].T
    b = rng.standard_normal(n)
    bt = rng.standard_normal(n)
    rec = orb.recycle_setup(A, U, Ut)
    _, _, info = orc.rbicg(A, b, bt, rec, tol=1e-9)
    _, _, plain = orc.rbicg(A, b, bt, None, tol=1e-9)
    assert info.status == orc.OK
    assert info.iters <= n - k
    assert plain.iters > n - k


def test_rbicg_redraws_the_dual_start_when_rho_is_zero():
    """(r_0, r~_0) = 0 exactly (b and b~ with disjoint supports, x~_{-1} = 0):
    Alg. 1 takes a new x~_{-1}; the dual system is still solved."""
    A, b, _, _ = _problem()
    n = A.shape[0]
    bt = inputs.gaussian_rhs(n, 77)
    b[n // 2:] = 0.0
    bt[: n // 2] = 0.0
    x, xt, info = orc.rbicg(A, b, bt, None, tol=1e-11)
    D = A.toarray()
    assert info.seeds_used == 1
    assert _rel(x, sla.solve(D, b)) <= 1e-8
    assert _rel(xt, sla.solve(D.T, bt)) <= 1e-8
