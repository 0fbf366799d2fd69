"""Batched solves of many independent systems of uneven sizes
(rbicgstab_batch_*): one persistent launch per pass over a work list of
tiles, per-system reductions, scalars and convergence.  Every system of the
batch must follow Alg. 2 on its own: in FP64 it is compared with the
oracle's solve of that system alone (iterations within 5%, x within 1e-7),
plain and with a fixed right-only recycle space per system; in the mixed
mode (FP32 iteration, FP64 restarts) every solution must be as close to the
exact one (dense LU) as the FP64 oracle's, or within 1e-7.  Sizes are ragged
and uneven (one system of a single slice, one with a zero right-hand side)."""
import numpy as np
import pytest
import scipy.linalg as sla

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
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _batch(nsys=9, seed=3):
    rng = np.random.default_rng(seed)
    mats = [inputs.conv_diff_2d(int(N), float(p)) for N, p in zip(rng.integers(5, 37, nsys), rng.uniform(1, 40, nsys))]
    mats.append(inputs.conv_diff_3d(11, 8.0))
    mats.append(inputs.conv_diff_2d(4, 3.0))          # 16 rows: one partial slice
    bs = [inputs.gaussian_rhs(A.n, 50 + i) for i, A in enumerate(mats)]
    bs[2] = np.zeros(mats[2].n)                         # finishes at once
    return mats, bs


@pytest.mark.parametrize("k", [0, 6])
def test_batch_fp64_matches_oracle_per_system(k):
    mats, bs = _batch()
    Us = [inputs.random_recycle_basis(A.n, k, 100 + i) for i, A in enumerate(mats)] if k else None
    B = rb.Batch(mats, k_max=k, precision="fp64", tol=1e-8)
    if k:
        B.set_recycle(Us)
    xs, sts = B.solve(bs)
    info = B.info()
    assert info["tiles"] > 0 and info["tile_slices"] in (16, 32, 64, 128, 256, 512, 1024)
    for i, (A, b) in enumerate(zip(mats, bs)):
        S = A.to_scipy()
        rec = orb.recycle_setup(S, Us[i]) if k else None
        xo, io = orb.rbicgstab(S, b, rec, tol=1e-8)
        st = sts[i]
        assert st["status"] == rb.RB_OK, (i, st)
        if np.linalg.norm(b) == 0:
            assert np.all(xs[i] == 0) and st["iters"] == 0
            continue
        assert abs(st["iters"] - io.iters) <= max(1, int(0.05 * io.iters)), (i, st["iters"], io.iters)
        assert _rel(xs[i], xo) <= 1e-7, (i, _rel(xs[i], xo))
        assert st["relres_true"] <= 1.5e-8
    # deterministic: the same batch twice gives bitwise-equal solutions
    xs2, _ = B.solve(bs)
    assert all(np.array_equal(a, c) for a, c in zip(xs, xs2))


@pytest.mark.parametrize("k", [0, 6])
def test_batch_mixed_against_dense_lu(k):
    mats, bs = _batch(seed=5)
    Us = [inputs.random_recycle_basis(A.n, k, 200 + i) for i, A in enumerate(mats)] if k else None
    B = rb.Batch(mats, k_max=k, precision="mixed", tol=1e-8)
    if k:
        B.set_recycle(Us)
    xs, sts = B.solve(bs)
    for i, (A, b) in enumerate(zip(mats, bs)):
        st = sts[i]
        assert st["status"] == rb.RB_OK, (i, st)
        if np.linalg.norm(b) == 0:
            continue
        S = A.to_scipy()
        assert np.linalg.norm(b - S @ xs[i]) <= 1e-8 * np.linalg.norm(b), (i, st)
        xstar = sla.solve(S.toarray(), b)
        xo, _ = orb.rbicgstab(S, b, orb.recycle_setup(S, Us[i]) if k else None, tol=1e-8)
        assert _rel(xs[i], xstar) <= max(2.0 * _rel(xo, xstar), 1e-7), (i, _rel(xs[i], xstar), _rel(xo, xstar))


def test_batch_values_and_device_arrays():
    """New values on the same patterns (a shift of every system), inputs as
    one concatenated CUDA tensor."""
    import torch
    mats, bs = _batch(nsys=5, seed=7)
    B = rb.Batch(mats, precision="fp64", tol=1e-8)
    shifted = [inputs.shifted_values(A, np.ones(A.n), 0.5) for A in mats]
    B.set_values(shifted)
    bt = torch.from_numpy(np.concatenate(bs)).cuda()
    xs, sts = B.solve(bt)
    for i, (A, b) in enumerate(zip(mats, bs)):
        S = inputs.CSR(A.n, A.row_ptr, A.col, shifted[i]).to_scipy()
        x = xs[i].cpu().numpy()
        assert sts[i]["status"] == rb.RB_OK
        assert np.linalg.norm(b - S @ x) <= 1.5e-8 * max(np.linalg.norm(b), 1e-300)
