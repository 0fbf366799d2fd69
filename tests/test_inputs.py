"""The seeded workload generators: sizes, structure and determinism of the
batched sweep of uneven 2D systems and of the large 27-point sequence (the
values their own docstrings state), checked on small instances and, for the
sweep's drawn sizes, at full size."""
import numpy as np

from paper_1406_2831_gb300 import inputs


def test_batch_sweep_sizes_and_shifts():
    specs = inputs.config_batch_2d(n_systems=6, side_lo=10, side_hi=20)
    again = inputs.config_batch_2d(n_systems=6, side_lo=10, side_hi=20)
    assert [s.label for s in specs] == [s.label for s in again]          # seeded
    for s in specs:
        P = s.pattern()
        N = int(round(np.sqrt(P.n)))
        assert N * N == P.n and 10 <= N <= 20
        assert P.nnz == 5 * N * N - 4 * N                                # 5-point, Dirichlet
        vals = [f() for f in s.values]
        d = P.diag_index()
        for v, sig in zip(vals, (0.0, 1e-2, 1e-1, 1.0)):
            dv = v - vals[0]
            assert np.allclose(dv[d], sig, rtol=0, atol=1e-15)          # sigma on the diagonal
            off = np.ones(P.nnz, bool)
            off[d] = False
            assert not np.any(dv[off])                                   # nothing else moves
        b = s.rhs[0][0]()
        assert b.shape == (P.n,) and np.array_equal(b, s.rhs[3][0]())   # one RHS per system
        assert s.k == 10


def test_batch_sweep_full_size_statistics():
    """256 systems with sides U{100..450}: about 22.5M unknowns and 112M
    nonzeros in all, mean n about 88k (from the drawn sides alone)."""
    specs = inputs.config_batch_2d()
    sides = np.array([int(s.label.split("x")[0].split("-")[1]) for s in specs])
    assert len(specs) == 256 and sides.min() >= 100 and sides.max() <= 450
    assert 20e6 < (sides ** 2).sum() < 25e6
    assert 100e6 < (5 * sides ** 2 - 4 * sides).sum() < 125e6


def test_large_27pt_sequence_structure():
    spec = inputs.config_large_27pt(8, 6, 5, n_systems=3)
    P = spec.pattern()
    assert P.n == 8 * 6 * 5
    assert P.nnz == (3 * 8 - 2) * (3 * 6 - 2) * (3 * 5 - 2)            # 27-point, Dirichlet
    v0, v1, v2 = (f() for f in spec.values)
    # only the centre and the three upwind face entries carry convection
    rows = np.repeat(np.arange(P.n), np.diff(P.row_ptr))
    moved = np.nonzero(v1 != v0)[0]
    d = P.col[moved] - rows[moved]
    assert set(np.unique(d)) <= {0, -1, -8, -8 * 6}
    assert np.array_equal(np.nonzero(v2 != v0)[0], moved)
    # the noise draw is shared: the diffusion-only entries are identical
    assert np.array_equal(np.delete(v0, moved), np.delete(v2, moved))
    assert spec.k == 30
    # the same count formula at another size (256 x 256 x 128 gives 224,140,792)
    Q = inputs.config_large_27pt(5, 4, 3, n_systems=1).pattern()
    assert Q.nnz == (3 * 5 - 2) * (3 * 4 - 2) * (3 * 3 - 2)



def test_stencil27_noisy_is_a_diagonally_dominant_m_matrix():
    """Off-diagonal couplings negative, interior row sums zero, boundary rows
    strictly dominant, non-symmetric; the oracle's BiCGSTAB solves it."""
    import scipy.sparse as sp
    from oracle import bicgstab as obs
    A = inputs.stencil27_noisy(9, 8, 7, 10.0)
    S = A.to_scipy()
    d = S.diagonal()
    off = S - sp.diags(d)
    assert off.max() <= 0.0 and d.min() > 0
    rowsum = np.asarray(S.sum(axis=1)).ravel()
    interior = np.array([(r % 9 not in (0, 8)) and ((r // 9) % 8 not in (0, 7)) and (r // 72 not in (0, 6))
                         for r in range(A.n)])
    assert np.abs(rowsum[interior]).max() <= 1e-12 * d.max()
    assert rowsum[~interior].min() > 0.1
    assert abs(S - S.T).max() > 0.01
    b = inputs.gaussian_rhs(A.n, 3)
    x, info = obs.bicgstab(S, b, tol=1e-10)
    assert np.linalg.norm(b - S @ x) <= 1e-9 * np.linalg.norm(b)
