"""Pins of the BiCGstab(l) oracle, plain and on the recycling projected
operator: dense LU solutions; l = 1 reproduces the separately written
BiCGSTAB and, with a recycle space, Alg. 2 iterate by iterate; the recursive
residual equals the true residual of x = x_0 + y - U C-hat^T A y (pins the
recycle bookkeeping); and on a nearly skew-symmetric operator, where
BiCGSTAB's omega collapses, l = 2 and 4 converge while l = 1 does not."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import bicgstab as ob
from oracle import bicgstab_l as obl
from oracle import rbicgstab as orb
from paper_1406_2831_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _problem(N=20, p=10.0, seed=3):
    A = inputs.conv_diff_2d(N, p).to_scipy()
    return A, inputs.gaussian_rhs(A.shape[0], seed)


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_plain_matches_dense_lu(ell):
    A, b = _problem()
    x, info = obl.bicgstab_l(A, b, ell, tol=1e-12)
    assert info.status == orb.OK and info.iters % ell == 0
    assert _rel(x, np.linalg.solve(A.toarray(), b)) <= 1e-9


def test_ell1_is_bicgstab():
    A, b = _problem()
    _, ref = ob.bicgstab(A, b, tol=1e-12, record=True)
    _, got = obl.bicgstab_l(A, b, 1, tol=1e-12, record=True)
    for j in range(20):
        assert _rel(got.iterates[j], ref.iterates[j]) <= 1e-10, j   # rounding grows to ~1e-11


def test_recycled_ell1_is_alg2():
    A, b = _problem()
    rec = orb.recycle_setup(A, inputs.random_recycle_basis(A.shape[0], 6, 4))
    _, ref = orb.rbicgstab(A, b, rec, tol=1e-12, record=True)
    _, got = obl.bicgstab_l(A, b, 1, rec=rec, tol=1e-12, record=True)
    for j in range(20):
        xi, xc, _ = ref.iterates[j]
        assert _rel(got.iterates[j], xi - rec.U @ xc) <= 1e-10, j


@pytest.mark.parametrize("ell", [2, 3])
def test_recycled_matches_dense_lu_and_true_residual(ell):
    A, b = _problem()
    n = A.shape[0]
    rec = orb.recycle_setup(A, inputs.random_recycle_basis(n, 6, 4))
    x, info = obl.bicgstab_l(A, b, ell, rec=rec, tol=1e-12)
    assert info.status == orb.OK
    assert _rel(x, np.linalg.solve(A.toarray(), b)) <= 1e-9
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(true - info.relres) <= 1e-3 * info.relres + 1e-15


def test_ell2_survives_where_bicgstab_collapses():
    """A = S + 1e-3 I with S the skew-symmetric central-difference convection
    operator on a 20 x 20 grid: (t, s) = 1e-3 ||s||^2, so BiCGSTAB's omega is
    nearly 0 and l = 1 breaks down or stalls; l = 2 and 4 minimise over two
    and four directions and converge."""
    N = 20
    I = sp.identity(N)
    D1 = sp.diags([-1.0, 1.0], [-1, 1], shape=(N, N)) * 0.5
    A = (sp.kron(I, D1) + sp.kron(D1, I) + 1e-3 * sp.identity(N * N)).tocsr()
    b = inputs.gaussian_rhs(N * N, 1)
    x1, i1 = obl.bicgstab_l(A, b, 1, tol=1e-8, max_itn=2000)
    assert i1.status != orb.OK or np.linalg.norm(b - A @ x1) > 1e-6 * np.linalg.norm(b)
    # Alg. 2 itself stops at its breakdown guards with finite iterates
    with np.errstate(divide="raise", invalid="raise", over="raise"):
        xa, ia = orb.rbicgstab(A, b, None, tol=1e-8, max_itn=2000)
    assert ia.status in (orb.BREAKDOWN_RHO, orb.BREAKDOWN_OMEGA, orb.NOTCONV)
    assert np.all(np.isfinite(xa))
    for ell in (2, 4):
        x, info = obl.bicgstab_l(A, b, ell, tol=1e-8, max_itn=2000)
        assert info.status == orb.OK, ell
        assert np.linalg.norm(b - A @ x) <= 2e-8 * np.linalg.norm(b), ell
