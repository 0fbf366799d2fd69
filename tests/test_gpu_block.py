"""GPU parity of blocked solves (rbicgstab_solve_block): up to four
right-hand sides of one matrix iterate together, sharing every pass over A,
C and C-hat.  Each system must still follow Alg. 2 on its own: it is
compared with the FP64 oracle's single solve of that system (same shadow
seed, same recycle space), with the tolerances of the single-RHS parity
tests.  The blocked kernels project column per lane, so their rounding
differs from the single-RHS FP64 path; truncated iterates bound how far that
moves x_j.  Sizes are ragged (n not a multiple of the 32-row slice)."""
import numpy as np
import pytest

from oracle import rbicgstab as orb
from oracle import recycle as orc
from oracle.dense import principal_cosines
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


def _solver(A, **kw):
    s = rb.Solver(**kw)
    s.set_matrix(A.row_ptr, A.col, A.val)
    return s


def _rhs_block(n, nrhs, seed0=40):
    return np.stack([inputs.gaussian_rhs(n, seed0 + i) for i in range(nrhs)])


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4])
def test_block_fixed_space_parity(nrhs):
    """Right-only random space, k = 20: every system of the block against the
    oracle's single solve (iterations within 5%, x within 1e-7)."""
    A = inputs.conv_diff_2d(45, 15.0)
    S = A.to_scipy()
    U = inputs.random_recycle_basis(A.n, 20, 21)
    B = _rhs_block(A.n, nrhs)
    s = _solver(A, recycle="fixed", k_max=20)
    s.set_recycle(U)
    res = s.solve_block(B)
    rec = orb.recycle_setup(S, U)
    for i in range(nrhs):
        st = res.stats[i]
        xo, io = orb.rbicgstab(S, B[i], rec, tol=1e-8)
        assert st["status"] == rb.RB_OK
        assert _iters_close(st["iters"], io.iters), (i, st["iters"], io.iters)
        assert _rel(res.x[i], xo) <= XTOL
        assert np.linalg.norm(B[i] - S @ res.x[i]) / np.linalg.norm(B[i]) <= 1.5e-8
        assert abs(st["relres_true"] - np.linalg.norm(B[i] - S @ res.x[i]) / np.linalg.norm(B[i])) <= 1e-12


def test_block_plain_parity():
    A = inputs.conv_diff_2d(33, 13.0)
    S = A.to_scipy()
    B = _rhs_block(A.n, 4)
    res = _solver(A).solve_block(B)
    for i in range(4):
        xo, io = orb.rbicgstab(S, B[i], None, tol=1e-8)
        assert _iters_close(res.stats[i]["iters"], io.iters)
        assert _rel(res.x[i], xo) <= XTOL


@pytest.mark.parametrize("j", [1, 5, 20])
def test_block_truncated_iterates_track_oracle(j):
    """x_j after exactly j iterations of each system of a 4-block (k = 20)."""
    A = inputs.conv_diff_2d(45, 15.0)
    S = A.to_scipy()
    U = inputs.random_recycle_basis(A.n, 20, 21)
    B = _rhs_block(A.n, 4, seed0=1)
    s = _solver(A, recycle="fixed", k_max=20, max_itn=j)
    s.set_recycle(U)
    res = s.solve_block(B)
    rec = orb.recycle_setup(S, U)
    for i in range(4):
        xo, io = orb.rbicgstab(S, B[i], rec, tol=1e-8, max_itn=j)
        assert res.stats[i]["iters"] == io.iters == j
        assert res.stats[i]["status"] == rb.C["RB_ENOTCONV"]
        assert _rel(res.x[i], xo) <= {1: 1e-12, 5: 1e-12, 20: 1e-10}[j]


def test_block_matches_single_solves_and_masks_finished_systems():
    """A zero right-hand side finishes at once (x = 0) and a duplicated one
    gives the same x bitwise; the rest match the library's single solves."""
    A = inputs.conv_diff_2d(40, 12.0)
    U = inputs.random_recycle_basis(A.n, 8, 3)
    b0 = inputs.gaussian_rhs(A.n, 7)
    b2 = inputs.gaussian_rhs(A.n, 8)
    B = np.stack([b0, np.zeros(A.n), b2, b0])
    s = _solver(A, recycle="fixed", k_max=8)
    s.set_recycle(U)
    res = s.solve_block(B)
    assert res.stats[1]["iters"] == 0 and np.all(res.x[1] == 0)
    assert np.array_equal(res.x[0], res.x[3])
    for i in (0, 2):
        single = s.solve(B[i])
        assert _iters_close(res.stats[i]["iters"], single.stats["iters"])
        assert _rel(res.x[i], single.x) <= XTOL


def test_block_deterministic_and_device_arrays():
    import torch
    A = inputs.conv_diff_2d(36, 14.0)
    U = inputs.random_recycle_basis(A.n, 6, 3)
    B = _rhs_block(A.n, 3)
    s = _solver(A, recycle="fixed", k_max=8)
    s.set_recycle(U)
    x1 = s.solve_block(B).x.copy()
    x2 = s.solve_block(B).x.copy()
    assert np.array_equal(x1, x2)
    Bt = torch.from_numpy(B).cuda()
    xt = s.solve_block(Bt).x.cpu().numpy()
    assert np.array_equal(x1, xt)


def test_block_nonzero_initial_guesses():
    A = inputs.conv_diff_2d(30, 12.0)
    S = A.to_scipy()
    U = inputs.random_recycle_basis(A.n, 4, 9)
    B = _rhs_block(A.n, 2)
    X0 = _rhs_block(A.n, 2, seed0=90)
    s = _solver(A, recycle="fixed", k_max=8)
    s.set_recycle(U)
    res = s.solve_block(B, X0.copy())
    rec = orb.recycle_setup(S, U)
    for i in range(2):
        xo, io = orb.rbicgstab(S, B[i], rec, x_m1=X0[i], tol=1e-8)
        assert _iters_close(res.stats[i]["iters"], io.iters)
        assert _rel(res.x[i], xo) <= XTOL


def test_block_mixed_refinement():
    """FP32 inner block + FP64 refinement per system: every refined x meets
    the FP64 tolerance and is as close to the exact solution as the FP64
    oracle's answer (within 2x, or 1e-7 relative)."""
    import scipy.linalg as sla
    A = inputs.conv_diff_2d(48, 12.0)
    S = A.to_scipy()
    D = S.toarray()
    U = inputs.random_recycle_basis(A.n, 8, 4)
    B = _rhs_block(A.n, 4)
    s = _solver(A, precision="mixed", recycle="fixed", k_max=8)
    s.set_recycle(U)
    res = s.solve_block(B)
    rec = orb.recycle_setup(S, U)
    for i in range(4):
        st = res.stats[i]
        assert st["status"] == rb.RB_OK
        assert np.linalg.norm(B[i] - S @ res.x[i]) / np.linalg.norm(B[i]) <= 1e-8
        xstar = sla.solve(D, B[i])
        xo, _ = orb.rbicgstab(S, B[i], rec, tol=1e-8)
        assert _rel(res.x[i], xstar) <= max(2.0 * _rel(xo, xstar), 1e-7)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_sequence_update_parity(precision):
    """Shifted 3D sequence (13^3, 5 shifts x 4 RHS, k = 8, s = 25) solved one
    block per shift with the update built from each block's first system;
    the oracle runs the same order (policy "first_block").  The first block
    has no recycle space and must track the oracle closely; later spaces come
    out of an ill-conditioned harmonic-Ritz problem, so U is compared by
    principal angles and later solves by iteration counts and residuals."""
    spec = inputs.config_shifted_3d(N=13, n_shifts=5, n_rhs=4, k=8, lazy_rhs=False)
    P = spec.pattern
    import scipy.sparse as sp
    mats = [sp.csr_matrix((v(), P.col, P.row_ptr), shape=(P.n, P.n)) for v in spec.values]
    ref = orc.solve_sequence(mats, spec.rhs, k=spec.k, cycle_s=spec.cycle_s, tol=spec.tol, policy="first_block")
    s = rb.Solver(k_max=spec.k, cycle_s=spec.cycle_s, recycle="update_first", tol=spec.tol, precision=precision)
    got, Us = [], []
    for i, (M, bs) in enumerate(zip(mats, spec.rhs)):
        if i == 0:
            s.set_matrix(P.row_ptr, P.col, M.data)
        else:
            s.set_values(M.data)
        B = np.stack(bs)
        r = s.solve_block(B)
        for j in range(len(bs)):
            assert r.stats[j]["status"] == rb.RB_OK
            assert np.linalg.norm(B[j] - M @ r.x[j]) / np.linalg.norm(B[j]) <= 1.5e-8
            got.append(r.stats[j]["iters"])
        Us.append(s.get_recycle()[0])
    if precision == "fp64":
        assert got[:4] == ref.iters[:4]
        for gi, oi in zip(got, ref.iters):
            assert abs(gi - oi) <= max(3, int(0.1 * oi)), (got, ref.iters)
        assert abs(sum(got) - sum(ref.iters)) <= 0.05 * sum(ref.iters)
    else:
        # FP32 iterations follow another trajectory than the FP64 oracle's:
        # check the recycling effect (later blocks need fewer iterations than
        # the first, which has no recycle space)
        assert np.mean(got[4:]) < np.mean(got[:4])
    # the update of the first block spans the oracle's harmonic-Ritz space.
    # FP64: every principal angle is small.  Mixed: the Krylov vectors are
    # FP32 and the update runs over every cycle of the first system's solve;
    # the FP32 basis drifts from the FP64 one over those cycles, which moves
    # the weakest harmonic Ritz pairs, and pairs at the selection boundary
    # (the k-th smallest |theta|, or the end of a complex pair) can trade
    # places with their neighbours.  The leading directions must agree: all
    # but the last two have cosine >= 0.99.
    U1 = orc.solve_sequence(mats[:1], [spec.rhs[0][:1]], k=spec.k, cycle_s=spec.cycle_s, tol=spec.tol).U_final
    c = np.sort(principal_cosines(Us[0], U1))[::-1]
    if precision == "fp64":
        assert np.sqrt(max(0.0, 1 - c.min() ** 2)) <= 1e-5
    else:
        assert c[: max(1, len(c) - 2)].min() >= 0.99, c


def test_block_rejects_bad_sizes():
    A = inputs.conv_diff_2d(10, 10.0)
    s = _solver(A)
    L = rb.lib()
    B = np.zeros((5, A.n))
    X = np.zeros((5, A.n))
    for nrhs, ld in ((0, A.n), (5, A.n), (2, A.n - 1)):
        code = L.rbicgstab_solve_block(s._h, nrhs, B.ctypes.data, X.ctypes.data, ld, rb.RB_HOST, None)
        assert code == rb.C["RB_EINVAL"], (nrhs, ld, code)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_time_passes_block(precision):
    A = inputs.conv_diff_2d(64, 12.0)
    U = inputs.random_recycle_basis(A.n, 20, 5)
    s = _solver(A, recycle="fixed", k_max=20, precision=precision)
    s.set_recycle(U)
    ms, code = rb.time_passes(s, _rhs_block(A.n, 4), reps=3)
    assert code == rb.RB_OK
    assert np.all(ms > 0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("grid", ["2d-45", "3d-13"])
def test_block_benchmark_kernels_small(precision, grid):
    """The benchmark's kernel configuration at sizes dense LU can check:
    k = 20 (the 24-column kernel bucket), a block of R = 4 right-hand sides,
    ragged n (2025 = 63 slices + 9 rows; 2197 = 68 slices + 21 rows).  Every
    slot's solution is as close to the exact one (dense LU) as the FP64
    oracle's answer with the same space (within 2x), or within 1e-7.  FP64
    slots also track the oracle's own solve: iterations within 5%, x within
    1e-7."""
    import scipy.linalg as sla
    if grid == "2d-45":
        A = inputs.conv_diff_2d(45, 15.0)
    else:
        spec = inputs.config_shifted_3d(N=13, n_shifts=5, n_rhs=1, k=20)
        P = spec.pattern
        A = inputs.CSR(P.n, P.row_ptr, P.col, spec.values[2]())
    S = A.to_scipy()
    D = S.toarray()
    U = inputs.random_recycle_basis(A.n, 20, 23)
    B = _rhs_block(A.n, 4, seed0=60)
    s = _solver(A, precision=precision, recycle="fixed", k_max=20, tol=1e-8)
    s.set_recycle(U)
    res = s.solve_block(B)
    rec = orb.recycle_setup(S, U)
    for i in range(4):
        st = res.stats[i]
        assert st["status"] == rb.RB_OK, st
        assert st["k_used"] == 20
        assert np.linalg.norm(B[i] - S @ res.x[i]) / np.linalg.norm(B[i]) <= 1e-8
        xstar = sla.solve(D, B[i])
        xo, io = orb.rbicgstab(S, B[i], rec, tol=1e-8)
        assert _rel(res.x[i], xstar) <= max(2.0 * _rel(xo, xstar), 1e-7), (i, _rel(res.x[i], xstar), _rel(xo, xstar))
        if precision == "fp64":
            assert _iters_close(st["iters"], io.iters), (i, st["iters"], io.iters)
            assert _rel(res.x[i], xo) <= XTOL


def _tight_reference(S, b, rec, x_start):
    """x* for the full-size checks: the oracle continued from its own
    tol = 1e-8 answer down to ||b - A x|| <= 1e-12 ||b||."""
    xs, info = orb.rbicgstab(S, b, rec, x_m1=x_start, tol=1e-12)
    assert info.status == orb.OK and info.relres_true <= 2e-12, (info.status, info.relres_true)
    return xs


@pytest.mark.slow
def test_block_mixed_full_size_against_tight_reference():
    """System 1 of the 128^3 shifted sequence at full size (n = 2,097,152):
    its four right-hand sides as one block in the mixed path with a fixed
    k = 20 right-only space, the kernel configuration the benchmark times
    (FP32 passes, 24-column bucket, R = 4).  Every system meets the FP64
    tolerance on its true residual.  The first system's solution is compared
    with a tight reference x* (the oracle continued to 1e-12): it must be as
    close to x* as the oracle's own tol = 1e-8 answer with the same space
    (within 2x), or within 1e-7.  FP32 arithmetic costs iterations: the
    count stays within [0.9, 1.6]x the oracle's (measured ratio ~1.3)."""
    import scipy.sparse as sp
    spec = inputs.config_shifted_3d(N=128, n_shifts=20, n_rhs=4, k=20)
    P = spec.pattern
    vals = spec.values[0]()
    S = sp.csr_matrix((vals, P.col, P.row_ptr), shape=(P.n, P.n))
    B = np.stack([g() for g in spec.rhs[0]])
    U = inputs.random_recycle_basis(P.n, 20, 11)
    s = rb.Solver(precision="mixed", recycle="fixed", k_max=20, tol=1e-8)
    s.set_matrix(P.row_ptr, P.col, vals)
    s.set_recycle(U)
    res = s.solve_block(B)
    for i in range(4):
        assert res.stats[i]["status"] == rb.RB_OK
        assert np.linalg.norm(B[i] - S @ res.x[i]) / np.linalg.norm(B[i]) <= 1e-8
    rec = orb.recycle_setup(S, U)
    xo, io = orb.rbicgstab(S, B[0], rec, tol=1e-8)
    xs = _tight_reference(S, B[0], rec, xo)
    e_gpu, e_ora = _rel(res.x[0], xs), _rel(xo, xs)
    print(f"mixed 128^3: |x-x*|/|x*| gpu {e_gpu:.3e} oracle(1e-8) {e_ora:.3e}; "
          f"iters gpu {res.stats[0]['iters']} oracle {io.iters}")
    assert e_gpu <= max(2.0 * e_ora, 1e-7), (e_gpu, e_ora)
    assert 0.9 * io.iters <= res.stats[0]["iters"] <= 1.6 * io.iters, (res.stats[0]["iters"], io.iters)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs", [1, 4])
def test_27pt_k30_against_dense_lu(precision, nrhs):
    """The large workload's kernels at a size dense LU can check: the noisy
    27-point operator (17 x 15 x 13, n = 3315 = 103 slices + 19 rows), k = 30
    (the 32-column bucket), one right-hand side and a block of four.  Every
    solution is as close to the exact one as the FP64 oracle's with the same
    space (within 2x), or within 1e-7."""
    import scipy.linalg as sla
    A = inputs.stencil27_noisy(17, 15, 13, 10.0)
    S = A.to_scipy()
    D = S.toarray()
    U = inputs.random_recycle_basis(A.n, 30, 31)
    B = _rhs_block(A.n, nrhs, seed0=90)
    s = _solver(A, precision=precision, recycle="fixed", k_max=30, tol=1e-8)
    s.set_recycle(U)
    res = s.solve_block(B) if nrhs > 1 else s.solve(B[0])
    stats = res.stats if nrhs > 1 else [res.stats]
    X = res.x if nrhs > 1 else [res.x]
    rec = orb.recycle_setup(S, U)
    for i in range(nrhs):
        assert stats[i]["status"] == rb.RB_OK, stats[i]
        assert stats[i]["k_used"] == 30
        xstar = sla.solve(D, B[i])
        xo, io = orb.rbicgstab(S, B[i], rec, tol=1e-8)
        assert _rel(X[i], xstar) <= max(2.0 * _rel(xo, xstar), 1e-7), (i, _rel(X[i], xstar), _rel(xo, xstar))
        if precision == "fp64":
            assert _iters_close(stats[i]["iters"], io.iters), (i, stats[i]["iters"], io.iters)
