"""Stencil slices of the SELL-32 layout.  A slice whose rows share one set of
column offsets (col - row) of the slice's width, all of them inside the
matrix, is stored in offset order with explicit zeros where a row lacks an
offset; the fused SpMV passes then form column indices from the offsets
instead of loading them.  Stencil operators qualify except near the first
and last grid planes.  The layout only reorders the zero terms of each row's
sum, so solves are bitwise equal to the CSR-order layout (RB_SELL_GENERIC);
a matrix without stencil structure keeps the generic layout and still
matches the oracle."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

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


def _solve(A, B, U, precision, generic):
    if generic:
        os.environ["RB_SELL_GENERIC"] = "1"
    try:
        s = rb.Solver(precision=precision, recycle="fixed", k_max=U.shape[1], tol=1e-8)
        s.set_matrix(A.row_ptr, A.col, A.val)
    finally:
        os.environ.pop("RB_SELL_GENERIC", None)
    s.set_recycle(U)
    return s, s.solve_block(B)


def _mats():
    spec = inputs.config_shifted_3d(N=21, n_shifts=3, n_rhs=1, k=20)
    P = spec.pattern
    yield "7pt-21^3", inputs.CSR(P.n, P.row_ptr, P.col, spec.values[1]())
    yield "5pt-45^2", inputs.conv_diff_2d(45, 15.0)
    yield "27pt-17x15x13", inputs.stencil27_noisy(17, 15, 13, 10.0)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_stencil_layout_is_bitwise_equal(precision):
    for name, A in _mats():
        U = inputs.random_recycle_basis(A.n, 20, 3)
        B = np.stack([inputs.gaussian_rhs(A.n, 70 + i) for i in range(4)])
        s1, r1 = _solve(A, B, U, precision, generic=False)
        s2, r2 = _solve(A, B, U, precision, generic=True)
        nsl, nst = s1.sell_stats()
        assert s2.sell_stats() == (nsl, 0)
        # every slice away from the first and last planes qualifies
        assert nst >= nsl // 2, (name, nsl, nst)
        for i in range(4):
            assert r1.stats[i]["iters"] == r2.stats[i]["iters"], name
            assert np.array_equal(r1.x[i], r2.x[i]), name
        v = inputs.gaussian_rhs(A.n, 5)
        assert np.array_equal(s1.apply(v), s2.apply(v))


def test_non_stencil_matrix_keeps_generic_layout():
    """Random sparsity: no slice shares an offset set of its width; the
    solve still matches the oracle."""
    rng = np.random.default_rng(4)
    n = 3000
    R = sp.random(n, n, density=2.0 / n, random_state=rng, format="csr")
    S = (R + sp.diags(np.full(n, 4.0)) + sp.diags(np.full(n - 1, -1.0), 1)).tocsr()
    S.sort_indices()
    A = inputs.CSR(n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))
    b = inputs.gaussian_rhs(n, 1)
    s = rb.Solver(recycle="none", tol=1e-10)
    s.set_matrix(A.row_ptr, A.col, A.val)
    nsl, nst = s.sell_stats()
    assert nst < nsl // 4
    res = s.solve(b)
    xo, io = orb.rbicgstab(S, b, None, tol=1e-10)
    assert res.stats["status"] == rb.RB_OK
    assert np.linalg.norm(res.x - xo) <= 1e-7 * np.linalg.norm(xo)
