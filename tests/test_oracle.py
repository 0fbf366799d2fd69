"""Pins for the CPU oracle: each checks it against something other than itself
(a printed value, a published test vector, dense LU, a closed form or an
invariant that Alg. 2 implies).  No GPU needed."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import bicgstab as ob
from oracle import rbicgstab as orb
from oracle import recycle as orc
from oracle.dense import invariant_subspaces, principal_cosines
from oracle.shadow import shadow_vector, splitmix64, splitmix64_scalar
from paper_1406_2831_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return [l.strip() for l in f if l.strip() and not l.startswith("#")]


def _sys2d(N, p, seed=0):
    A = inputs.conv_diff_2d(N, p).to_scipy()
    b = inputs.gaussian_rhs(N * N, seed)
    return A, b


# ---------------------------------------------------------------- shadow vector
def test_splitmix64_published_vector():
    want = [int(v) for v in _golden("splitmix64_seed1234567.txt")]
    assert [splitmix64_scalar(1234567, i) for i in range(5)] == want
    assert [int(v) for v in splitmix64(1234567, 5)] == want


def test_shadow_mapping_exact():
    z = [splitmix64_scalar(0x5EED, i) for i in range(64)]
    want = np.array([2.0 * ((v >> 11) * 2.0 ** -53) - 1.0 for v in z])
    got = shadow_vector(64, 0x5EED)
    assert np.array_equal(got, want)
    big = shadow_vector(200000, 7)
    assert big.min() >= -1.0 and big.max() < 1.0
    assert abs(big.mean()) < 0.01 and abs(big.var() - 1.0 / 3.0) < 0.01


# ---------------------------------------------------------------- dense LU pins
@pytest.mark.parametrize("N,p", [(12, 10.0), (16, 13.0), (20, 17.0)])
def test_plain_bicgstab_matches_dense_lu(N, p):
    A, b = _sys2d(N, p)
    xlu = sla.solve(A.toarray(), b)
    x, info = ob.bicgstab(A, b, tol=1e-13)
    assert info.status == ob.OK
    assert np.linalg.norm(x - xlu) / np.linalg.norm(xlu) <= 1e-9


@pytest.mark.parametrize("N,k,kind", [(12, 1, "random"), (16, 3, "random"), (20, 5, "random"),
                                      (16, 4, "eig"), (20, 6, "eig")])
def test_rbicgstab_matches_dense_lu(N, k, kind):
    A, b = _sys2d(N, 12.0, seed=3)
    Ad = A.toarray()
    xlu = sla.solve(Ad, b)
    if kind == "random":
        U = inputs.random_recycle_basis(N * N, k, seed=11)
        Ut = None
    else:
        U, Ut, _ = invariant_subspaces(Ad, k)
    rec = orb.recycle_setup(A, U, Ut)
    assert rec.k == k
    x, info = orb.rbicgstab(A, b, rec, tol=1e-13)
    assert info.status == orb.OK
    assert np.linalg.norm(x - xlu) / np.linalg.norm(xlu) <= 1e-9
    assert info.relres_true <= 1e-12


def test_rbicgstab_nonzero_initial_guess_matches_lu():
    A, b = _sys2d(14, 11.0, seed=5)
    xlu = sla.solve(A.toarray(), b)
    U = inputs.random_recycle_basis(196, 3, seed=2)
    x0 = inputs.gaussian_rhs(196, 9)
    x, info = orb.rbicgstab(A, b, orb.recycle_setup(A, U), x_m1=x0, tol=1e-13)
    assert np.linalg.norm(x - xlu) / np.linalg.norm(xlu) <= 1e-9


# ---------------------------------------------------------------- k = 0 is BiCGSTAB
def test_k0_reproduces_plain_bicgstab_iterates():
    A, b = _sys2d(32, 14.0, seed=1)
    xp, ip = ob.bicgstab(A, b, tol=1e-10, record=True)
    xr, ir = orb.rbicgstab(A, b, None, tol=1e-10, record=True)
    assert abs(ip.iters - ir.iters) <= 1
    for i in range(min(10, ip.iters)):
        xi_p = ip.iterates[i]
        xi_r = ir.iterates[i][0]
        assert np.linalg.norm(xi_p - xi_r) <= 1e-12 * np.linalg.norm(xi_p)
    assert np.linalg.norm(xp - xr) <= 1e-8 * np.linalg.norm(xp)


# ---------------------------------------------------------------- invariants of Alg. 2
def _recycled_run(N=24, k=4, seed=7):
    A, b = _sys2d(N, 15.0, seed=seed)
    U = inputs.random_recycle_basis(N * N, k, seed=seed + 1)
    Ut = inputs.random_recycle_basis(N * N, k, seed=seed + 2)
    rec = orb.recycle_setup(A, U, Ut)
    x, info = orb.rbicgstab(A, b, rec, tol=1e-10, record=True)
    return A, b, rec, x, info


def test_biorthogonality_and_projector():
    A, b, rec, x, info = _recycled_run()
    M = rec.Ct.T @ rec.C
    off = M - np.diag(np.diag(M))
    assert np.abs(off).max() <= 1e-12 * rec.Dc.max()
    assert np.all(rec.Dc > 0)
    assert np.allclose(np.diag(M), rec.Dc, rtol=1e-12)
    # C-hat^T C = I (eq. (3.4))
    assert np.abs(rec.Chat.T @ rec.C - np.eye(rec.k)).max() <= 1e-12
    # B = (I - C C-hat^T) A annihilates U (Thm 3.2)
    AU = A @ rec.U
    BU = AU - rec.C @ (rec.Chat.T @ AU)
    assert np.linalg.norm(BU) <= 1e-12 * np.linalg.norm(AU)
    # C^T r~_0 = 0 and C~^T r_0 = 0 (condition (c) in the proof of Thm 3.2)
    assert np.linalg.norm(rec.C.T @ info.rt0) <= 1e-12 * np.linalg.norm(rec.C) * np.linalg.norm(info.rt0)
    assert np.linalg.norm(rec.Ct.T @ info.r0) <= 1e-12 * np.linalg.norm(rec.Ct) * np.linalg.norm(info.r0)


@pytest.mark.parametrize("two_sided", [False, True])
def test_projector_is_the_oblique_projector_of_the_raw_spaces(two_sided):
    """C C-hat^T is the projector onto range(A U) along range(A^T U~)^perp:
    C M^+ C~^T with the unrotated C = A U, C~ = A^T U~ and M = C~^T C, whatever
    basis the biorthogonalisation picks; and U C-hat^T, the map the iterate
    correction uses, is U M^+ C~^T."""
    A = inputs.conv_diff_2d(14, 9.0).to_scipy()
    n = A.shape[0]
    U = inputs.random_recycle_basis(n, 5, 21)
    Ut = inputs.random_recycle_basis(n, 5, 22) if two_sided else U
    rec = orb.recycle_setup(A, U, Ut if two_sided else None)
    C, Ct = A @ U, A.T @ Ut
    Mp = np.linalg.pinv(Ct.T @ C)
    want = C @ Mp @ Ct.T
    got = rec.C @ rec.Chat.T
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    assert np.linalg.norm(rec.U @ rec.Chat.T - U @ Mp @ Ct.T) <= 1e-12 * np.linalg.norm(U @ Mp @ Ct.T)
    assert np.linalg.norm(got @ got - got) <= 1e-12 * np.linalg.norm(got)   # a projector


def test_residuals_stay_in_null_space_of_chat():
    A, b, rec, x, info = _recycled_run()
    for (xi, xci, ri) in info.iterates[:40]:
        assert np.linalg.norm(rec.Chat.T @ ri) <= 1e-10 * np.linalg.norm(rec.Chat) * np.linalg.norm(ri)


def test_residual_identity_pins_step8_sign():
    A, b, rec, x, info = _recycled_run()
    nb = np.linalg.norm(b)
    for i, (xi, xci, ri) in enumerate(info.iterates, start=1):
        true_r = b - A @ (xi - rec.U @ xci)
        assert np.linalg.norm(true_r - ri) <= 1e-12 * i * nb * 10


def test_planted_sign_error_in_step8_is_caught():
    """Flip the sign of the final correction x - U x_c in a copy of the result; the identity must fail."""
    A, b, rec, x, info = _recycled_run()
    xi, xci, ri = info.iterates[-1]
    wrong = b - A @ (xi + rec.U @ xci)
    assert np.linalg.norm(wrong - ri) > 1e-6 * np.linalg.norm(b)


# ---------------------------------------------------------------- exact deflation closed form
def test_exact_deflation_spectrum():
    N, k = 14, 4
    A, b = _sys2d(N, 10.0)
    Ad = A.toarray()
    R, L, w = invariant_subspaces(Ad, k)
    rec = orb.recycle_setup(A, R, L)
    B = Ad - rec.C @ (rec.Chat.T @ Ad)
    ev = np.sort_complex(np.linalg.eigvals(B))
    evA = np.linalg.eigvals(Ad)
    order = np.argsort(np.abs(evA))
    rest = np.sort_complex(evA[order[k:]])
    ev_small = ev[np.argsort(np.abs(ev))]
    assert np.abs(ev_small[:k]).max() <= 1e-10
    assert np.abs(np.sort_complex(ev_small[k:]) - rest).max() <= 1e-9
    # deflating the smallest eigenvalues does not slow BiCGSTAB down
    _, ip = ob.bicgstab(A, b, tol=1e-10)
    _, ir = orb.rbicgstab(A, b, rec, tol=1e-10)
    assert ir.iters <= ip.iters


# ---------------------------------------------------------------- harmonic Ritz
def test_harmonic_ritz_recovers_exact_eigenvector():
    N = 14
    A, _ = _sys2d(N, 12.0)
    Ad = A.toarray()
    R, L, w = invariant_subspaces(Ad, 1)
    v = R[:, 0]
    rng = np.random.default_rng(4)
    W = np.column_stack([rng.standard_normal(N * N) for _ in range(5)] + [v])
    W = W @ rng.standard_normal((6, 6))   # hide v inside a mixed basis
    Z = Ad @ W
    y, th = orc.harmonic_ritz_coeffs(Z.T @ Z, Z.T @ W, 1)
    u = W @ y[:, 0]
    u /= np.linalg.norm(u)
    assert abs(abs(u @ v) / np.linalg.norm(v) - 1.0) <= 1e-10
    assert abs(th[0] - w[0]) <= 1e-10 * abs(w[0])


def test_harmonic_ritz_full_space_gives_eigenvalues():
    """When range(W) is the whole space, harmonic Ritz values are eigenvalues."""
    rng = np.random.default_rng(8)
    n = 12
    Ad = rng.standard_normal((n, n)) + 4 * np.eye(n)
    W = rng.standard_normal((n, n))
    Z = Ad @ W
    y, th = orc.harmonic_ritz_coeffs(Z.T @ Z, Z.T @ W, n)
    ev = np.linalg.eigvals(Ad)
    want = np.sort(np.abs(ev))[: len(th)]
    assert np.allclose(np.sort(np.abs(th)), want, rtol=1e-9)


# ---------------------------------------------------------------- Table 1 (Sec. 5)
def test_table1_example1_principal_cosines():
    """Example 1 of Sec. 5: central differences on the 40 x 40 interior grid
    reproduce the printed cosines to the printed 4 digits."""
    want = np.array([float(v) for v in _golden("table1_example1.txt")])
    N, h = 40, 1.0 / 41
    I = sp.identity(N)
    D2 = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(N, N))
    D1 = sp.diags([-1.0, 1.0], [-1, 1], shape=(N, N)) * (h / 2)
    A = (sp.kron(I, D2) + sp.kron(D2, I) + 10.0 * sp.kron(I, D1) - 10.0 * sp.kron(D1, I)).toarray()
    R, L, _ = invariant_subspaces(A, 10)
    got = principal_cosines(R, L)
    assert np.abs(got - want).max() <= 5e-5
    # the generator of the Example 1 system builds the same operator
    E1, _, _ = inputs.example1()
    assert np.array_equal(E1.to_scipy().toarray(), A)


def _example1_runs():
    """The three runs of Sec. 5 on Example 1: no recycling, U = 5 exact right
    eigenvectors with U~ = U, and U, U~ = 5 right and 5 left eigenvectors
    (smallest-magnitude eigenvalues); x_{-1} = ones, tol 1e-10."""
    E1, b, x0 = inputs.example1()
    A = E1.to_scipy()
    R, L, _ = invariant_subspaces(A.toarray(), 5)
    out = {}
    for name, rec in [("none", None), ("right", orb.recycle_setup(A, R)), ("both", orb.recycle_setup(A, R, L))]:
        x, info = orb.rbicgstab(A, b, rec, x_m1=x0, tol=1e-10)
        out[name] = (x, info)
    return A, b, out


def test_example1_left_right_study():
    """Sec. 5, Example 1: recycling the right invariant subspace pays, and
    adding the left one changes little (the paper's finding for this nearly
    normal operator, whose left and right subspaces are close by Table 1).
    Each run meets the tolerance; the discrete solution obeys the maximum
    principle of the M-matrix (values between the boundary values 0 and 1)."""
    A, b, runs = _example1_runs()
    its = {k: v[1].iters for k, v in runs.items()}
    for x, info in runs.values():
        assert info.status == orb.OK
        assert np.linalg.norm(b - A @ x) <= 2e-10 * np.linalg.norm(b)
        assert x.min() > 0.0 and x.max() < 1.0
    assert its["right"] < 0.9 * its["none"] and its["both"] < 0.9 * its["none"]
    assert abs(its["right"] - its["both"]) <= 0.1 * its["none"]


# ---------------------------------------------------------------- recycling pays (Sec. 6.2)
def test_sequence_recycling_reduces_matvecs_small_2d():
    spec = inputs.config_small_2d(N=32)
    mats = [sp.csr_matrix((v, spec.pattern.col, spec.pattern.row_ptr),
                          shape=(spec.pattern.n, spec.pattern.n)) for v in spec.values]
    plain = orc.solve_sequence(mats, spec.rhs, k=spec.k, recycle=False, tol=spec.tol)
    rec = orc.solve_sequence(mats, spec.rhs, k=spec.k, cycle_s=spec.cycle_s, tol=spec.tol)
    assert all(i.relres_true <= 2 * spec.tol for i in rec.info)
    assert all(i.relres_true <= 2 * spec.tol for i in plain.info)
    assert rec.matvecs_iter + rec.matvecs_setup < plain.matvecs_iter
    assert sum(rec.iters[1:]) < sum(plain.iters[1:])


def test_sequence_first_block_order():
    """policy "first_block": the right-hand sides of one matrix all use the
    space in force when the matrix arrives, and the update built during the
    first one's solve is adopted from the next matrix on."""
    import scipy.sparse as sp
    from oracle import rbicgstab as orb2
    spec = inputs.config_small_2d(N=12)
    P = spec.pattern
    mats = [sp.csr_matrix((v, P.col, P.row_ptr), shape=(P.n, P.n)) for v in spec.values[:2]]
    b1 = inputs.gaussian_rhs(P.n, 1)
    rhs = [[spec.rhs[0][0], b1], [spec.rhs[1][0], b1]]
    blk = orc.solve_sequence(mats, rhs, k=4, cycle_s=10, tol=1e-8, policy="first_block")
    seq = orc.solve_sequence(mats, rhs, k=4, cycle_s=10, tol=1e-8, policy="first")
    # the first solve is the same under both orders
    assert np.array_equal(blk.x[0], seq.x[0])
    # the second RHS of matrix 0 runs with no recycle space under first_block
    x_plain, info = orb2.rbicgstab(mats[0], b1, orb2.empty_space(P.n), tol=1e-8)
    assert np.array_equal(blk.x[1], x_plain) and blk.k_used[1] == 0
    # ... and with the update of the first solve under first
    assert seq.k_used[1] == 4
    # matrix 1 starts from the update of matrix 0's first solve in both
    U_after_first = orc.solve_sequence(mats[:1], [rhs[0][:1]], k=4, cycle_s=10, tol=1e-8).U_final
    rec = orb2.recycle_setup(mats[1], U_after_first)
    x_b, _ = orb2.rbicgstab(mats[1], b1, rec, tol=1e-8)
    assert np.allclose(blk.x[3], x_b, rtol=0, atol=1e-12 * np.linalg.norm(x_b))
