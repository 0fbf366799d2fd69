"""The mixed modes on an ill-conditioned system: FP32 inner iterations meet
their accuracy floor (about u_32 times the condition number) on the
diffusion-dominated 2D operator at N = 300 (condition ~4e4), where one
replacement interval can no longer gain a decade.  The solver must then
finish in FP64 from its current x: the answer meets the tolerance, its
error against a tight FP64 reference is that of an FP64 solve at the same
tolerance, and the work stays within a small multiple of the FP64 solve's.
The recycle-update path and the batched solver take the same route."""
import numpy as np
import pytest

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


def _solve(A, b, tol, **kw):
    with rb.Solver(tol=tol, **kw) as s:
        s.set_matrix(A.row_ptr, A.col, A.val)
        r = s.solve(b)
        return np.asarray(r.x), r.stats


@pytest.fixture(scope="module")
def hard():
    A = inputs.conv_diff_2d(300, 4.0)
    b = inputs.gaussian_rhs(A.n, 7)
    xstar, st = _solve(A, b, 1e-13, precision="fp64")
    assert st["status"] == rb.RB_OK
    x64, st64 = _solve(A, b, 1e-8, precision="fp64")
    err64 = np.linalg.norm(x64 - xstar) / np.linalg.norm(xstar)
    return A, b, xstar, st64["iters"], err64


def _check(A, b, x, xstar, err64):
    S = A.to_scipy()
    assert np.linalg.norm(b - S @ x) <= 1.5e-8 * np.linalg.norm(b)   # FP64 finish: recursive criterion
    err = np.linalg.norm(x - xstar) / np.linalg.norm(xstar)
    assert err <= max(2.0 * err64, 1e-9), (err, err64)


def test_mixed_finishes_in_fp64_when_fp32_stalls(hard):
    A, b, xstar, it64, err64 = hard
    x, st = _solve(A, b, 1e-8, precision="mixed")
    assert st["status"] == rb.RB_OK, st
    _check(A, b, x, xstar, err64)
    # FP32 iterations cost about half an FP64 one; the whole solve stays
    # within a small multiple of the FP64 solve's work
    assert st["iters"] <= 3 * it64, (st["iters"], it64)


def test_mixed_update_path_finishes_in_fp64(hard):
    A, b, xstar, it64, err64 = hard
    x, st = _solve(A, b, 1e-8, precision="mixed", k_max=10, recycle="update_first")
    assert st["status"] == rb.RB_OK, st
    _check(A, b, x, xstar, err64)


def test_batched_mixed_finishes_hard_systems_in_fp64(hard):
    A, b, xstar, it64, err64 = hard
    easy = [inputs.conv_diff_2d(40, 10.0), inputs.conv_diff_2d(23, 3.0)]
    mats = [easy[0], A, easy[1]]
    bs = [inputs.gaussian_rhs(easy[0].n, 3), b, inputs.gaussian_rhs(easy[1].n, 4)]
    B = rb.Batch(mats, precision="mixed", tol=1e-8)
    xs, sts = B.solve(bs)
    for i, (M, bb) in enumerate(zip(mats, bs)):
        assert sts[i]["status"] == rb.RB_OK, (i, sts[i])
        assert np.linalg.norm(bb - M.to_scipy() @ xs[i]) <= 1.5e-8 * np.linalg.norm(bb)
    _check(A, b, xs[1], xstar, err64)
