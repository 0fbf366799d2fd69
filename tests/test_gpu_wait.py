"""Failure detection without a GPU fault: the bounded mbarrier wait that the
tensor-core Gram and the bulk-copy staging use gives up after its limit,
leaves the kernel normally and reports RB_ETIMEOUT, and the context stays
usable (a solve right after it is exact).  Nothing here faults, traps or
spins without bound: the wait that nothing completes has a limit of a few
milliseconds."""
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


def test_wait_completes_when_the_barrier_is_completed():
    code, ms = rb.wait_selftest(True, 5.0)
    assert code == rb.RB_OK
    assert ms < 5.0


def test_wait_expires_and_context_stays_usable():
    code, ms = rb.wait_selftest(False, 5.0)
    assert code == rb.C["RB_ETIMEOUT"]
    assert ms >= 1.0          # it did wait (the limit is in cycles at the rated clock)
    # the context still works: a small solve right after
    A = inputs.conv_diff_2d(16, 5.0)
    b = inputs.gaussian_rhs(A.n, 1)
    with rb.Solver(precision="fp64", tol=1e-10) as s:
        s.set_matrix(A.row_ptr, A.col, A.val)
        r = s.solve(b)
    assert r.stats["status"] == rb.RB_OK
    x = np.asarray(r.x)
    assert np.linalg.norm(b - A.to_scipy() @ x) <= 1e-9 * np.linalg.norm(b)


def test_wait_selftest_rejects_bad_limits():
    with pytest.raises(rb.RbError):
        rb.wait_selftest(False, 0.0)
    with pytest.raises(rb.RbError):
        rb.wait_selftest(False, 5000.0)
