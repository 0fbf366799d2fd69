"""Host logic of the autograd function (``autograd.RecycledSolve``) on CPU:
its backward wiring (adjoint solve -> dL/db, pattern product -> dL/dvalues) is
checked by torch's numerical gradient check with a dense stand-in for the
solver handle, and a solver that moved on to another matrix is put back to
the forward's matrix before the dual solve."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from paper_1406_2831_gb300 import autograd as rag  # noqa: E402
from paper_1406_2831_gb300 import inputs  # noqa: E402
from paper_1406_2831_gb300 import rbicgstab as rb  # noqa: E402


class _Res:
    def __init__(self, x):
        self.x = x
        self.stats = {"status": rb.RB_OK}


class DenseStandIn:
    """The Solver methods the function calls, with dense solves (CPU tensors)."""

    def __init__(self, A):
        self.row_ptr, self.col = A.row_ptr, A.col
        self.rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
        self.values_version = 0
        self.log = []

    def _M(self):
        n = len(self.row_ptr) - 1
        return sp.csr_matrix((self.vals, self.col, self.row_ptr), shape=(n, n)).toarray()

    def set_values(self, v):
        self.vals = v.detach().numpy().copy()
        self.values_version += 1
        self.log.append("set_values")

    def solve(self, b):
        return _Res(torch.from_numpy(np.linalg.solve(self._M(), b.numpy())))

    def solve_adjoint(self, g):
        self.log.append("solve_adjoint")
        return _Res(torch.from_numpy(np.linalg.solve(self._M().T, g.numpy())))

    def pattern_outer(self, u, v, scale):
        return torch.from_numpy(scale * u.numpy()[self.rows] * v.numpy()[self.col])


def test_backward_wiring_passes_gradcheck():
    A = inputs.conv_diff_2d(5, 7.0)
    s = DenseStandIn(A)
    vals = torch.from_numpy(A.val.copy()).requires_grad_(True)
    b = torch.from_numpy(inputs.gaussian_rhs(A.n, 3)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v, bb: rag.RecycledSolve.apply(v, bb, s), (vals, b),
                                    eps=1e-6, atol=1e-8, rtol=1e-6)


def test_backward_restores_the_forward_matrix():
    A = inputs.conv_diff_2d(4, 5.0)
    s = DenseStandIn(A)
    v0 = torch.from_numpy(A.val.copy()).requires_grad_(True)
    b = torch.from_numpy(inputs.gaussian_rhs(A.n, 1))
    x0 = rag.solve(s, v0, b)
    # the solver moves on to another matrix before the backward of x0
    rag.solve(s, torch.from_numpy(2.0 * A.val), b)
    s.log.clear()
    x0.sum().backward()
    assert s.log == ["set_values", "solve_adjoint"]
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()
    lam = np.linalg.solve(M.T, np.ones(A.n))
    x = np.linalg.solve(M, b.numpy())
    want = -lam[s.rows] * x[A.col]
    assert np.allclose(v0.grad.numpy(), want, rtol=1e-12, atol=1e-14)


def test_checkpointing_recomputes_x_with_the_same_gradient():
    """With checkpoint=True the forward keeps no solution; backward solves
    for it again (after the dual solve) and returns the same gradients."""
    A = inputs.conv_diff_2d(5, 3.0)
    b0 = torch.from_numpy(inputs.gaussian_rhs(A.n, 1))
    grads = []
    for ck in (False, True):
        s = DenseStandIn(A)
        vals = torch.from_numpy(A.val.copy()).requires_grad_(True)
        b = b0.clone().requires_grad_(True)
        x = rag.solve(s, vals, b, checkpoint=ck)
        (x.square().sum()).backward()
        grads.append((vals.grad.clone(), b.grad.clone()))
        assert s.log.count("solve_adjoint") == 1
    assert torch.allclose(grads[0][0], grads[1][0], rtol=1e-12, atol=0)
    assert torch.allclose(grads[0][1], grads[1][1], rtol=1e-12, atol=0)
