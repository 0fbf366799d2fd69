"""Recycled BiCGstab(l) on the GPU (rbicgstab_solve_l) against the FP64
oracle (oracle/bicgstab_l.py) and dense LU: the breakdown-robust variant of
Alg. 2 (Sec. 4's omega = 0 remark, Sec. 7).  The library minimises over the
residual block through its Gram matrix where the oracle orthogonalises it
(modified Gram-Schmidt): the same minimiser, other rounding.  Sizes are
ragged; l = 1 must behave as Alg. 2 on the GPU; on a nearly skew operator,
where BiCGSTAB's omega collapses, l = 2 and 4 must converge."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import bicgstab_l as obl
from oracle import rbicgstab as orb
from paper_1406_2831_gb300 import build as rbuild
from paper_1406_2831_gb300 import inputs
from paper_1406_2831_gb300 import rbicgstab as rb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    rbuild.build()
    rb.lib()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _csr(S):
    S = S.tocsr()
    S.sort_indices()
    return inputs.CSR(S.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


@pytest.mark.parametrize("ell,k", [(1, 0), (2, 0), (4, 0), (2, 5), (3, 5)])
def test_solve_l_matches_oracle_and_dense_lu(ell, k):
    A = inputs.conv_diff_2d(33, 10.0)
    S = A.to_scipy()
    b = inputs.gaussian_rhs(A.n, 3)
    s = rb.Solver(recycle="fixed" if k else "none", k_max=k, tol=1e-10)
    s.set_matrix(A.row_ptr, A.col, A.val)
    rec = None
    if k:
        U = inputs.random_recycle_basis(A.n, k, 8)
        s.set_recycle(U)
        rec = orb.recycle_setup(S, U)
    res = s.solve_l(b, ell)
    st = res.stats
    xo, io = obl.bicgstab_l(S, b, ell, rec=rec, tol=1e-10)
    assert st["status"] == rb.RB_OK and io.status == orb.OK
    assert st["iters"] % ell == 0
    assert abs(st["iters"] - io.iters) <= max(ell, int(0.05 * io.iters)), (st["iters"], io.iters)
    xs = sla.solve(S.toarray(), b)
    assert _rel(res.x, xs) <= max(2.0 * _rel(xo, xs), 1e-7)
    assert _rel(res.x, xo) <= 1e-7
    # the recursive residual is the true residual of x = x_0 + y - U x_c
    assert abs(st["relres_true"] - st["relres_rec"]) <= 1e-3 * st["relres_rec"] + 1e-14


def test_ell1_behaves_as_alg2_on_the_gpu():
    A = inputs.conv_diff_2d(40, 13.0)
    b = inputs.gaussian_rhs(A.n, 5)
    U = inputs.random_recycle_basis(A.n, 6, 2)
    s = rb.Solver(recycle="fixed", k_max=6, tol=1e-9)
    s.set_matrix(A.row_ptr, A.col, A.val)
    s.set_recycle(U)
    r1 = s.solve_l(b, 1)
    r2 = s.solve(b)
    assert r1.stats["status"] == r2.stats["status"] == rb.RB_OK
    assert abs(r1.stats["iters"] - r2.stats["iters"]) <= 1
    assert _rel(r1.x, r2.x) <= 1e-7


def test_ell2_survives_where_bicgstab_collapses():
    """S + 1e-3 I, S the skew-symmetric central-difference convection
    operator on a 20 x 20 grid: l = 1 stalls or breaks down; l = 2 and 4
    converge and are as accurate as the oracle's l = 2 answer."""
    N = 20
    I = sp.identity(N)
    D1 = sp.diags([-1.0, 1.0], [-1, 1], shape=(N, N)) * 0.5
    S = (sp.kron(I, D1) + sp.kron(D1, I) + 1e-3 * sp.identity(N * N)).tocsr()
    A = _csr(S)
    b = inputs.gaussian_rhs(N * N, 1)
    s = rb.Solver(recycle="none", tol=1e-8, max_itn=2000)
    s.set_matrix(A.row_ptr, A.col, A.val)
    r1 = s.solve_l(b, 1)
    assert r1.stats["status"] != rb.RB_OK or np.linalg.norm(b - S @ r1.x) > 1e-6 * np.linalg.norm(b)
    xs = sla.solve(S.toarray(), b)
    xo, io = obl.bicgstab_l(S, b, 2, tol=1e-8, max_itn=2000)
    for ell in (2, 4):
        r = s.solve_l(b, ell)
        assert r.stats["status"] == rb.RB_OK, (ell, r.stats)
        assert np.linalg.norm(b - S @ r.x) <= 2e-8 * np.linalg.norm(b), ell
        assert _rel(r.x, xs) <= max(10.0 * _rel(xo, xs), 1e-6), ell


def test_solve_l_rejects_bad_ell():
    A = inputs.conv_diff_2d(10, 5.0)
    s = rb.Solver()
    s.set_matrix(A.row_ptr, A.col, A.val)
    for ell in (0, 9):
        with pytest.raises(rb.RbError):
            s.solve_l(inputs.gaussian_rhs(A.n, 1), ell)
