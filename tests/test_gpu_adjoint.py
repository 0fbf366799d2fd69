"""GPU parity of the adjoint gradient (autograd.RecycledSolve) against the
oracle's adjoint gradient and central differences (direct sparse LU), on the
parametrised 3D operator with 8 regional coefficients; and the pattern outer
product against its definition."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import adjoint as oad
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


def _A(spec, p):
    P = spec.pattern
    return sp.csr_matrix((spec.values(p), P.col, P.row_ptr), shape=(P.n, P.n))


def test_pattern_outer_matches_definition():
    import torch
    A = inputs.conv_diff_2d(37, 11.0)
    s = rb.Solver()
    s.set_matrix(A.row_ptr, A.col, A.val)
    u = torch.from_numpy(inputs.gaussian_rhs(A.n, 1)).cuda()
    v = torch.from_numpy(inputs.gaussian_rhs(A.n, 2)).cuda()
    out = s.pattern_outer(u, v, -1.0).cpu().numpy()
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    want = (-u.cpu().numpy()[rows]) * v.cpu().numpy()[A.col]
    assert np.array_equal(out, want)


@pytest.mark.parametrize("k", [0, 6])
def test_autograd_gradient_matches_oracle_and_differences(k):
    import torch
    from paper_1406_2831_gb300 import autograd as rag
    spec = inputs.config_param_3d(N=9, m_out=4)
    P = spec.pattern
    s = rb.Solver(recycle="fixed" if k else "none", k_max=k, tol=1e-12)
    s.set_matrix(P.row_ptr, P.col, spec.values(spec.p0))
    rec = None
    if k:
        U = inputs.random_recycle_basis(P.n, k, 7)
        s.set_recycle(U)
        from oracle import rbicgstab as orb
        rec = orb.recycle_setup(_A(spec, spec.p0), U)
    dev = torch.device("cuda")
    basis = torch.from_numpy(np.stack(spec.basis)).to(dev)
    p = torch.tensor(spec.p0, dtype=torch.float64, device=dev, requires_grad=True)
    b = torch.from_numpy(spec.b).to(dev).requires_grad_(True)
    Cout = torch.from_numpy(spec.C_out).to(dev)
    vals = (p[:, None] * basis).sum(0)
    x = rag.solve(s, vals, b)
    L = (Cout @ x).square().sum()
    L.backward()
    g = oad.adjoint_gradient(_A(spec, spec.p0), spec.b, spec.C_out, spec.basis, rec=rec, tol=1e-13)
    gp = p.grad.cpu().numpy()
    assert np.linalg.norm(gp - g.grad_p) <= 1e-7 * np.linalg.norm(g.grad_p)
    assert np.linalg.norm(b.grad.cpu().numpy() - g.lam) <= 1e-7 * np.linalg.norm(g.lam)
    fd = np.empty(8)
    for kk in range(8):
        h = 1e-6 * max(1.0, abs(spec.p0[kk]))
        e = np.zeros(8)
        e[kk] = h
        Lp = oad.loss(spec.C_out, spla.spsolve(_A(spec, spec.p0 + e).tocsc(), spec.b))
        Lm = oad.loss(spec.C_out, spla.spsolve(_A(spec, spec.p0 - e).tocsc(), spec.b))
        fd[kk] = (Lp - Lm) / (2 * h)
    assert np.max(np.abs(gp - fd)) <= 1e-5 * np.max(np.abs(fd))


@pytest.mark.parametrize("two_sided", [False, True])
def test_adjoint_solve_matches_oracle_dual(two_sided):
    """rbicgstab_solve_adjoint: Alg. 2 on A^T with the swapped space (right
    U~, left U) against the oracle's dual solve of the same construction
    (iterations within 5%, lam within 1e-7), ragged n = 13^3."""
    spec = inputs.config_param_3d(N=13, m_out=4)
    P = spec.pattern
    A = _A(spec, spec.p0)
    U = inputs.random_recycle_basis(P.n, 8, 17)
    Ut = inputs.random_recycle_basis(P.n, 8, 18) if two_sided else None
    from oracle import rbicgstab as orb
    rec = orb.recycle_setup(A, U, Ut)
    g = inputs.gaussian_rhs(P.n, 21)
    lo, io = orb.rbicgstab(sp.csr_matrix(A.T), g, oad.dual_space(A, rec), tol=1e-8)
    s = rb.Solver(recycle="fixed", k_max=8, tol=1e-8)
    s.set_matrix(P.row_ptr, P.col, spec.values(spec.p0))
    s.set_recycle(U, Ut)
    r = s.solve_adjoint(g)
    assert r.stats["status"] == rb.RB_OK
    assert abs(r.stats["iters"] - io.iters) <= max(1, int(0.05 * io.iters)), (r.stats["iters"], io.iters)
    assert np.linalg.norm(r.x - lo) <= 1e-7 * np.linalg.norm(lo)
    assert np.linalg.norm(g - A.T @ r.x) <= 1.5e-8 * np.linalg.norm(g)
    # the handle is back in its primary orientation
    b = inputs.gaussian_rhs(P.n, 22)
    xp = s.solve(b).x
    assert np.linalg.norm(b - A @ xp) <= 1.5e-8 * np.linalg.norm(b)
