"""Pins of the adjoint-gradient oracle (the dual system of Sec. 2 with
b~ = dL/dx) against what the mathematics fixes: central finite differences of
L(p) and L(b) with direct sparse LU solves (no Krylov method, no adjoint),
the chain rule from the pattern gradient to the parameters, the linearity of
the parametrised operator, and finite termination of the dual solve when its
swapped recycle space (right U~, left U) holds exact eigenvectors."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import adjoint as oad
from oracle import rbicgstab as orb
from oracle.dense import principal_cosines
from paper_1406_2831_gb300 import inputs


def _spec(N=6, m_out=4):
    return inputs.config_param_3d(N=N, m_out=m_out)


def _A(spec, p):
    P = spec.pattern
    return sp.csr_matrix((spec.values(p), P.col, P.row_ptr), shape=(P.n, P.n))


def _loss_direct(spec, p, b=None):
    """L(p) with a direct sparse LU solve."""
    A = _A(spec, p).tocsc()
    x = spla.spsolve(A, spec.b if b is None else b)
    return oad.loss(spec.C_out, x)


def test_param_operator_is_linear_in_p():
    """sum_k p_k A_k equals the operator assembled directly with the regional
    coefficients (per-cell kappa and c), for a generic p."""
    N = 8
    spec = inputs.config_param_3d(N=N)
    h = 1.0 / (N + 1)
    idx = np.arange(N ** 3)
    region = 2 * ((idx % N + 1) * h >= 0.5) + (((idx // N) % N + 1) * h >= 0.5)
    p = np.array([0.7, 1.3, 2.0, 0.4, 3.0, 11.0, 7.5, 0.2])
    A = inputs.conv_diff_3d(N, p[4:][region], kappa=p[:4][region])
    assert np.array_equal(A.col, spec.pattern.col) and np.array_equal(A.row_ptr, spec.pattern.row_ptr)
    assert np.max(np.abs(A.val - spec.values(p))) <= 1e-14 * np.max(np.abs(A.val))
    assert sorted(np.bincount(region)) == [N ** 3 // 4] * 4


def test_gradient_matches_central_differences():
    """dL/dp_k from one dual solve against central differences of L(p) with
    h = 1e-6 max(1, |p_k|): within 1e-5 relative (the differences' own error
    is O(h^2) plus rounding / h)."""
    spec = _spec()
    p = spec.p0
    g = oad.adjoint_gradient(_A(spec, p), spec.b, spec.C_out, spec.basis, tol=1e-13)
    fd = np.empty(len(p))
    for kk in range(len(p)):
        hk = 1e-6 * max(1.0, abs(p[kk]))
        e = np.zeros(len(p))
        e[kk] = hk
        fd[kk] = (_loss_direct(spec, p + e) - _loss_direct(spec, p - e)) / (2 * hk)
    assert g.info.status == orb.OK and g.info_dual.status == orb.OK
    assert np.linalg.norm(g.grad_p - fd) <= 1e-5 * np.linalg.norm(fd)
    assert np.max(np.abs(g.grad_p - fd)) <= 1e-5 * np.max(np.abs(fd))


def test_difference_pin_catches_an_untransposed_dual_solve():
    """The finite-difference pin separates A from A^T (A is non-symmetric
    through the upwind convection): a dual solve with A instead of A^T is off
    by far more than the tolerance."""
    spec = _spec()
    p = spec.p0
    A = _A(spec, p)
    g = oad.adjoint_gradient(A, spec.b, spec.C_out, spec.basis, tol=1e-13)
    lam_wrong = spla.spsolve(A.tocsc(), 2.0 * spec.C_out.T @ (spec.C_out @ g.x))
    P = spec.pattern
    wrong = np.array([-(lam_wrong @ (sp.csr_matrix((Ak, P.col, P.row_ptr), shape=A.shape) @ g.x))
                      for Ak in spec.basis])
    assert np.linalg.norm(wrong - g.grad_p) > 1e-3 * np.linalg.norm(g.grad_p)


def test_gradient_in_b_is_the_dual_solution():
    """dL/db = lam: L is quadratic in b, so a central difference along a
    random direction is exact up to rounding."""
    spec = _spec()
    p = spec.p0
    g = oad.adjoint_gradient(_A(spec, p), spec.b, spec.C_out, spec.basis, tol=1e-13)
    d = np.random.default_rng(8).standard_normal(spec.b.shape[0])
    eps = 1e-3
    fd = (_loss_direct(spec, p, spec.b + eps * d) - _loss_direct(spec, p, spec.b - eps * d)) / (2 * eps)
    assert abs(g.lam @ d - fd) <= 1e-8 * abs(fd)


def test_pattern_gradient_contracts_to_parameter_gradient():
    """dL/dp_k = sum_ij dL/dA_ij (A_k)_ij: the pattern gradient and the
    parameter gradient agree through the chain rule."""
    spec = _spec()
    g = oad.adjoint_gradient(_A(spec, spec.p0), spec.b, spec.C_out, spec.basis, tol=1e-12)
    via_pattern = np.array([g.grad_vals @ Ak for Ak in spec.basis])
    assert np.max(np.abs(via_pattern - g.grad_p)) <= 1e-12 * np.max(np.abs(g.grad_p))


def test_gradient_with_recycling_equals_gradient_without():
    """A random right-only space (U~ = U) for the primary solve and the same
    space with roles swapped for the dual solve change the iterations, not
    the gradient."""
    spec = _spec()
    A = _A(spec, spec.p0)
    rec = orb.recycle_setup(A, inputs.random_recycle_basis(A.shape[0], 6, 12))
    g0 = oad.adjoint_gradient(A, spec.b, spec.C_out, spec.basis, tol=1e-12)
    g1 = oad.adjoint_gradient(A, spec.b, spec.C_out, spec.basis, rec=rec, tol=1e-12)
    assert np.linalg.norm(g1.grad_p - g0.grad_p) <= 1e-8 * np.linalg.norm(g0.grad_p)
    assert np.linalg.norm(g1.lam - g0.lam) <= 1e-8 * np.linalg.norm(g0.lam)


def test_dual_space_reuses_the_primary_products():
    """The dual operator's C is the primary's C~ and its C~ the primary's C
    (as spaces): A^T U~ and (A^T)^T U."""
    spec = _spec()
    A = _A(spec, spec.p0)
    n = A.shape[0]
    rec = orb.recycle_setup(A, inputs.random_recycle_basis(n, 5, 1), inputs.random_recycle_basis(n, 5, 2))
    dual = oad.dual_space(A, rec)
    assert dual.k == rec.k
    assert np.min(principal_cosines(dual.C, rec.Ct)) >= 1 - 1e-12
    assert np.min(principal_cosines(dual.Ct, rec.C)) >= 1 - 1e-12


@pytest.mark.parametrize("k", [4, 6])
def test_dual_solve_with_exact_left_eigenvectors_terminates_after_n_minus_k(k):
    """A = V diag(lambda) V^{-1}: with U = k right and U~ = k left
    eigenvectors, the swapped space deflates k eigenvalues of A^T, so the
    dual solve ends within n - k iterations."""
    rng = np.random.default_rng(5)
    n = 24
    V = np.eye(n) + 0.2 * rng.standard_normal((n, n))
    A = sp.csr_matrix(V @ np.diag(np.linspace(1.0, 6.0, n)) @ np.linalg.inv(V))
    U = V[:, :k]
    Ut = np.linalg.inv(V)[:k, :].T
    rec = orb.recycle_setup(A, U, Ut)
    C_out = rng.standard_normal((3, n))
    b = rng.standard_normal(n)
    basis = [A]
    g = oad.adjoint_gradient(A, b, C_out, basis, rec=rec, tol=1e-10)
    assert g.info.status == orb.OK and g.info_dual.status == orb.OK
    assert g.info.iters <= n - k and g.info_dual.iters <= n - k
    lam = np.linalg.solve(A.toarray().T, 2.0 * C_out.T @ (C_out @ np.linalg.solve(A.toarray(), b)))
    assert np.linalg.norm(g.lam - lam) <= 1e-7 * np.linalg.norm(lam)
