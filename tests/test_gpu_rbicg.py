"""GPU parity of Alg. 1 (RBiCG, rbicg_solve): the primary system A x = b and
the dual A^T x~ = b~ against the FP64 oracle's Alg. 1 (same starts, same
recycle space), at ragged sizes (n not a multiple of the 32-row slice):
iterations within 5%, both solutions within 1e-7, the iterates after exactly
j iterations, the redraw of x~_{-1} when (r_0, r~_0) = 0, the shadow dual right-hand side, initial
guesses, and exact deflation."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import rbicg as orc
from oracle import rbicgstab as orb
from oracle.shadow import DEFAULT_SEED, shadow_vector
from paper_1406_2831_gb300 import build as rbuild
from paper_1406_2831_gb300 import inputs
from paper_1406_2831_gb300 import rbicgstab as rb

pytestmark = pytest.mark.gpu

XTOL = 1e-7


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    rbuild.build()
    rb.lib()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _iters_close(a, b):
    return abs(a - b) <= max(1, int(0.05 * max(a, b)))


def _solver(A, U=None, Ut=None, **kw):
    k = 0 if U is None else U.shape[1]
    s = rb.Solver(recycle="fixed" if k else "none", k_max=k, **kw)
    s.set_matrix(A.row_ptr, A.col, A.val)
    if k:
        s.set_recycle(U, Ut)
    return s


@pytest.mark.parametrize("k", [0, 8])
def test_rbicg_parity(k):
    A = inputs.conv_diff_2d(45, 15.0)
    S = A.to_scipy()
    b = inputs.gaussian_rhs(A.n, 5)
    bt = inputs.gaussian_rhs(A.n, 6)
    U = inputs.random_recycle_basis(A.n, k, 21) if k else None
    rx, rxt = _solver(A, U).solve_dual(b, bt)
    rec = orb.recycle_setup(S, U) if k else None
    xo, xto, io = orc.rbicg(S, b, bt, rec, tol=1e-8)
    st = rx.stats
    assert st["status"] == rb.RB_OK and io.status == orc.OK
    assert _iters_close(st["iters"], io.iters), (st["iters"], io.iters)
    assert _rel(rx.x, xo) <= XTOL
    assert _rel(rxt.x, xto) <= XTOL
    assert np.linalg.norm(b - S @ rx.x) / np.linalg.norm(b) <= 1.5e-8
    assert np.linalg.norm(bt - S.T @ rxt.x) / np.linalg.norm(bt) <= 1.5e-8
    assert abs(st["relres_true"] - np.linalg.norm(b - S @ rx.x) / np.linalg.norm(b)) <= 1e-12
    assert abs(rxt.stats["relres_true"] - np.linalg.norm(bt - S.T @ rxt.x) / np.linalg.norm(bt)) <= 1e-12
    assert st["k_used"] == k and st["matvecs"] == 2 * st["iters"]


@pytest.mark.parametrize("j", [1, 5, 20])
def test_rbicg_truncated_iterates_track_oracle(j):
    """x_j and x~_j (after the final correction) after exactly j iterations, k = 8."""
    A = inputs.conv_diff_2d(40, 12.0)
    S = A.to_scipy()
    b = inputs.gaussian_rhs(A.n, 1)
    bt = inputs.gaussian_rhs(A.n, 2)
    U = inputs.random_recycle_basis(A.n, 8, 3)
    rx, rxt = _solver(A, U, max_itn=j).solve_dual(b, bt)
    xo, xto, io = orc.rbicg(S, b, bt, orb.recycle_setup(S, U), tol=1e-8, max_itn=j)
    assert rx.stats["iters"] == io.iters == j
    assert rx.stats["status"] == rb.C["RB_ENOTCONV"]
    bound = {1: 1e-12, 5: 1e-12, 20: 1e-10}[j]
    assert _rel(rx.x, xo) <= bound
    assert _rel(rxt.x, xto) <= bound


def test_rbicg_two_sided_space_first_iterates():
    """Independent random U, U~: the oblique projector amplifies rounding in
    any implementation (see the parity notes), so only the first iterates are
    compared."""
    A = inputs.conv_diff_2d(36, 10.0)
    S = A.to_scipy()
    b = inputs.gaussian_rhs(A.n, 11)
    bt = inputs.gaussian_rhs(A.n, 12)
    U = inputs.random_recycle_basis(A.n, 6, 13)
    Ut = inputs.random_recycle_basis(A.n, 6, 14)
    for j in (1, 3):
        rx, rxt = _solver(A, U, Ut, max_itn=j).solve_dual(b, bt)
        xo, xto, _ = orc.rbicg(S, b, bt, orb.recycle_setup(S, U, Ut), tol=1e-8, max_itn=j)
        assert _rel(rx.x, xo) <= 1e-8
        assert _rel(rxt.x, xto) <= 1e-8


def test_rbicg_shadow_dual_and_initial_guesses():
    """b~ omitted (the shadow vector serves) and non-zero x_{-1}, x~_{-1}."""
    A = inputs.conv_diff_2d(30, 9.0)
    S = A.to_scipy()
    b = inputs.gaussian_rhs(A.n, 21)
    x0 = inputs.gaussian_rhs(A.n, 22)
    xt0 = inputs.gaussian_rhs(A.n, 23)
    U = inputs.random_recycle_basis(A.n, 4, 24)
    rx, rxt = _solver(A, U).solve_dual(b, None, x0.copy(), xt0.copy())
    bt = shadow_vector(A.n, DEFAULT_SEED)
    xo, xto, io = orc.rbicg(S, b, bt, orb.recycle_setup(S, U), x_m1=x0, xt_m1=xt0, tol=1e-8)
    assert _iters_close(rx.stats["iters"], io.iters)
    assert _rel(rx.x, xo) <= XTOL
    assert _rel(rxt.x, xto) <= XTOL


def test_rbicg_redraw_when_rho_is_zero():
    A = inputs.conv_diff_2d(24, 8.0)
    S = A.to_scipy()
    n = A.n
    b = inputs.gaussian_rhs(n, 31)
    bt = inputs.gaussian_rhs(n, 32)
    b[n // 2:] = 0.0
    bt[: n // 2] = 0.0
    rx, rxt = _solver(A).solve_dual(b, bt)
    xo, xto, io = orc.rbicg(S, b, bt, None, tol=1e-8)
    assert io.seeds_used == 1 and rx.stats["seeds_used"] == 2
    assert _rel(rx.x, xo) <= XTOL
    assert _rel(rxt.x, xto) <= XTOL


def test_rbicg_exact_deflation():
    """U, U~ = exact right / left eigenvectors: at most n - k iterations."""
    rng = np.random.default_rng(5)
    n, k = 24, 6
    V = np.eye(n) + 0.2 * rng.standard_normal((n, n))
    M = V @ np.diag(np.linspace(1.0, 6.0, n)) @ np.linalg.inv(V)
    S = sp.csr_matrix(M)
    A = inputs.CSR(n=n, row_ptr=S.indptr.astype(np.int32), col=S.indices.astype(np.int32), val=S.data.copy())
    U = V[:, :k]
    Ut = np.linalg.inv(V)[:k, :].T
    b = rng.standard_normal(n)
    bt = rng.standard_normal(n)
    rx, rxt = _solver(A, U, Ut, tol=1e-9).solve_dual(b, bt)
    assert rx.stats["status"] == rb.RB_OK
    assert rx.stats["iters"] <= n - k
    assert np.linalg.norm(b - M @ rx.x) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(bt - M.T @ rxt.x) <= 1e-8 * np.linalg.norm(bt)


def test_rbicg_device_arrays_and_determinism():
    import torch
    A = inputs.conv_diff_2d(33, 11.0)
    b = inputs.gaussian_rhs(A.n, 41)
    bt = inputs.gaussian_rhs(A.n, 42)
    U = inputs.random_recycle_basis(A.n, 5, 43)
    s = _solver(A, U)
    x1, xt1 = (r.x.copy() for r in s.solve_dual(b, bt))
    x2, xt2 = (r.x.copy() for r in s.solve_dual(b, bt))
    assert np.array_equal(x1, x2) and np.array_equal(xt1, xt2)
    rd, rdt = s.solve_dual(torch.from_numpy(b).cuda(), torch.from_numpy(bt).cuda())
    assert np.array_equal(rd.x.cpu().numpy(), x1) and np.array_equal(rdt.x.cpu().numpy(), xt1)
