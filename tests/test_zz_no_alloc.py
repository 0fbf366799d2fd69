"""rbicgstab_residual_noalloc: the residual entry point for callers that
cannot allocate device memory (a framework that owns the allocator, work
about to be captured into a CUDA graph, a service with device memory sized
once at start-up).  Its output is checked, on two calls in a row, against the
existing entry points: rbicgstab_apply (A x) for the residual vector and the
solver's own true-residual check (rb_stats.relres_true) for the norm.

This file is collected last on purpose: a run that stops at the first
failure has already run every other test.  It passes on its own in a fresh
process as well as after the rest of the suite."""
import numpy as np
import pytest

from paper_1406_2831_gb300 import build as rbuild
from paper_1406_2831_gb300 import inputs
from paper_1406_2831_gb300 import rbicgstab as rb

pytestmark = pytest.mark.gpu

RTOL = 1e-12   # same order as the library's other FP64 residual checks


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "needs a CUDA device"
    rbuild.build()
    rb.lib()
    return t


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_noalloc_residual_matches_existing_entry_points(torch, kind):
    A = inputs.conv_diff_2d(40, 12.0) if kind == "2d" else inputs.conv_diff_3d(48, 10.0)
    b = inputs.gaussian_rhs(A.n, 3)
    s = rb.Solver(tol=1e-8)
    s.set_matrix(A.row_ptr, A.col, A.val)
    res = s.solve(b)
    x1 = res.x
    x2 = inputs.gaussian_rhs(A.n, 4)           # a second, unrelated input
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.from_numpy(A.row_ptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    bt = torch.from_numpy(b).to(dev)
    r = torch.empty(A.n, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    bnorm = np.linalg.norm(b)
    for call, x in enumerate((x1, x2)):
        xt = torch.from_numpy(x).to(dev)
        code = rb.residual_noalloc(rp, col, val, xt, bt, r, out)
        assert code == rb.RB_OK
        torch.cuda.synchronize()
        want = b - s.apply(x)                         # existing entry point: A x
        got = r.cpu().numpy()
        assert np.linalg.norm(got - want) <= RTOL * np.linalg.norm(want)
        got_norm = np.sqrt(out.item())
        assert abs(got_norm - np.linalg.norm(want)) <= RTOL * np.linalg.norm(want)
        if call == 0:
            # the solver's own true-residual check of the same x
            assert abs(got_norm / bnorm - res.stats["relres_true"]) <= RTOL * max(res.stats["relres_true"], 1e-300)


def test_noalloc_rejects_bad_sizes(torch):
    dev = torch.device("cuda", torch.cuda.current_device())
    z = torch.zeros(4, dtype=torch.float64, device=dev)
    zi = torch.zeros(4, dtype=torch.int32, device=dev)
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    for bad_n in (0, -3, 2 ** 31):
        with pytest.raises(rb.RbError) as e:
            rb.residual_noalloc(zi, zi, z, z, z, z, one, n=bad_n)
        assert e.value.code == rb.C["RB_EINVAL"]


def test_noalloc_rejects_bad_arguments(torch):
    """Wrong dtypes and short buffers are refused on the host, before any
    pointer reaches the kernel."""
    A = inputs.conv_diff_2d(12, 5.0)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(A.row_ptr).to(dev)
    col = torch.from_numpy(A.col).to(dev)
    val = torch.from_numpy(A.val).to(dev)
    x = torch.ones(A.n, dtype=torch.float64, device=dev)
    b = torch.ones(A.n, dtype=torch.float64, device=dev)
    r = torch.empty(A.n, dtype=torch.float64, device=dev)
    nrm = torch.empty(1, dtype=torch.float64, device=dev)
    bad = [
        (rp.long(), col, val, x, b, r, nrm),
        (rp, col, val.float(), x, b, r, nrm),
        (rp, col, val, x[:-1], b, r, nrm),
        (rp, col, val, x, b, r[:-1], nrm),
        (rp, col[:-1], val, x, b, r, nrm),
        (rp, col, val, x, b, r, nrm[:0]),
    ]
    for args in bad:
        with pytest.raises(rb.RbError) as e:
            rb.residual_noalloc(*args)
        assert e.value.code == rb.C["RB_EINVAL"]
    assert rb.residual_noalloc(rp, col, val, x, b, r, nrm) == rb.RB_OK
