"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/rbicgstab.h, its host-only harmonic-Ritz step agrees
with the oracle's (a different algorithm on the same pencil), and its host
SVD (the biorthogonalisation of the recycle setup, Sec. 3) is a valid SVD with the
singular values LAPACK computes."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.dense import principal_cosines
from oracle.recycle import harmonic_ritz_coeffs
from paper_1406_2831_gb300 import build as rbuild
from paper_1406_2831_gb300 import rbicgstab as rb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    rbuild.build()
    return rb.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "rbicgstab.h")).read()
    return sorted(set(re.findall(r"\b(rbicg(?:stab)?_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_error_strings(L):
    for code in range(-10, 2):
        s = rb.error_string(code)
        assert s and s != "unknown status"
    assert rb.error_string(12345) == "unknown status"


def test_header_constants_match_binding():
    assert rb.C["RB_KMAX"] == 64
    assert rb.RB_HOST == 0 and rb.RB_DEVICE == 1


def _pencil(seed, n=300, m=30, rank_drop=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 5 * np.eye(n)
    W = rng.standard_normal((n, m))
    if rank_drop:
        W[:, -rank_drop:] = W[:, :rank_drop] @ rng.standard_normal((rank_drop, rank_drop))
    Z = A @ W
    return W, Z, Z.T @ Z, Z.T @ W


@pytest.mark.parametrize("seed", range(6))
def test_host_harmonic_ritz_matches_oracle(L, seed):
    W, Z, G, H = _pencil(seed)
    k = 8
    y1, t1 = harmonic_ritz_coeffs(G, H, k)
    y2, t2 = rb.harmonic_ritz(G, H, k)
    assert len(t1) == len(t2)
    assert np.abs(np.sort_complex(t1) - np.sort_complex(t2)).max() <= 1e-9 * np.abs(t1).max()
    c = principal_cosines(W @ y1, W @ y2)
    assert 1.0 - c.min() <= 1e-10


def test_host_harmonic_ritz_rank_deficient(L):
    W, Z, G, H = _pencil(7, rank_drop=3)
    y1, t1 = harmonic_ritz_coeffs(G, H, 6)
    y2, t2 = rb.harmonic_ritz(G, H, 6)
    assert len(t1) == len(t2)
    assert np.abs(np.sort_complex(t1) - np.sort_complex(t2)).max() <= 1e-6 * np.abs(t1).max()


def test_host_harmonic_ritz_exact_eigenvector(L):
    """An exact eigenvector inside span W is returned with its eigenvalue."""
    rng = np.random.default_rng(3)
    n = 40
    S = rng.standard_normal((n, n))
    d = np.linspace(0.5, 9.0, n)
    A = S @ np.diag(d) @ np.linalg.inv(S)      # non-normal, real spectrum
    j = 0
    v = S[:, j]
    w = d
    W = np.column_stack([rng.standard_normal((n, 4)), v]) @ rng.standard_normal((5, 5))
    Z = A @ W
    y, th = rb.harmonic_ritz(Z.T @ Z, Z.T @ W, 1)
    u = W @ y[:, 0]
    assert abs(abs(u @ v) / np.linalg.norm(u) / np.linalg.norm(v) - 1) <= 1e-10
    assert abs(th[0] - w[j]) <= 1e-10 * abs(w[j])


def test_harmonic_ritz_rejects_bad_args(L):
    with pytest.raises(rb.RbError):
        rb.harmonic_ritz(np.eye(3), np.eye(3), 5)


def _check_svd(M, P, sig, Q, tol=1e-13):
    k = M.shape[0]
    s1 = np.linalg.svd(M, compute_uv=False)
    assert np.all(np.diff(sig) <= 0)
    assert np.max(np.abs(sig - s1)) <= tol * s1[0]
    assert np.linalg.norm(P @ np.diag(sig) @ Q.T - M) <= tol * np.linalg.norm(M)
    assert np.linalg.norm(Q.T @ Q - np.eye(k)) <= tol * k
    live = sig > 1e-8 * sig[0]
    assert np.linalg.norm(P[:, live].T @ P[:, live] - np.eye(live.sum())) <= tol * k


@pytest.mark.parametrize("k", [1, 5, 20, 40])
def test_host_svd_of_a_biorthogonalisation_gram(L, k):
    """M = C~^T C for random tall C, C~ (the setup's Gram matrix)."""
    rng = np.random.default_rng(k)
    C = rng.standard_normal((300, k))
    Ct = rng.standard_normal((300, k)) + 0.5 * C
    M = Ct.T @ C
    P, sig, Q = rb.svd_small(M)
    _check_svd(M, P, sig, Q)


def test_host_svd_rank_deficient(L):
    rng = np.random.default_rng(3)
    M = rng.standard_normal((10, 3)) @ rng.standard_normal((3, 10))
    P, sig, Q = rb.svd_small(M)
    assert np.all(sig[3:] <= 1e-13 * sig[0])
    _check_svd(M, P, sig, Q)


def test_host_svd_rejects_bad_args(L):
    M = np.eye(3)
    out = [np.zeros(9), np.zeros(3), np.zeros(9)]
    assert L.rbicgstab_svd_small(0, M.ctypes.data, out[0].ctypes.data, out[1].ctypes.data,
                                 out[2].ctypes.data) == rb.C["RB_EINVAL"]
    M[1, 2] = np.nan
    assert L.rbicgstab_svd_small(3, M.ctypes.data, out[0].ctypes.data, out[1].ctypes.data,
                                 out[2].ctypes.data) == rb.C["RB_ENONFINITE"]


def _theta_sorted(t):
    t = np.asarray(t, dtype=complex)
    return t[np.lexsort((t.imag, t.real, np.round(np.abs(t), 12)))]


@pytest.mark.parametrize("seed", range(4))
def test_host_harmonic_ritz_complex_pairs(L, seed):
    """With Z^T Z = I the pencil reduces to H y = (1/theta) y, so the theta are
    the reciprocals of H's eigenvalues (LAPACK through numpy); a random real H
    has complex pairs, each returned as [Re y, Im y] spanning H's invariant
    subspace of the pair."""
    rng = np.random.default_rng(100 + seed)
    m = 14
    H = rng.standard_normal((m, m))
    mu = np.linalg.eigvals(H)
    assert np.any(np.abs(mu.imag) > 1e-3)
    y, th = rb.harmonic_ritz(np.eye(m), H, m)
    assert len(th) == m
    want = _theta_sorted(1.0 / mu)
    got = _theta_sorted(th)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    # each selected column block is invariant under H: H Y = Y M for a small M
    k = 6
    y6, th6 = rb.harmonic_ritz(np.eye(m), H, k)
    Mfit = np.linalg.lstsq(y6, H @ y6, rcond=None)[0]
    assert np.linalg.norm(H @ y6 - y6 @ Mfit) <= 1e-10 * np.linalg.norm(H) * np.linalg.norm(y6)
    ref = _theta_sorted(1.0 / mu)[: len(th6)]
    assert np.abs(_theta_sorted(th6) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_host_harmonic_ritz_defective_block(L):
    """H = S J S^-1 with a 2 x 2 Jordan block for the eigenvalue of largest
    magnitude (2.5): its theta = 0.4 appears twice, accurate to the square
    root of the rounding unit that a defective eigenvalue allows, and the
    first returned direction lies in the block's invariant subspace."""
    rng = np.random.default_rng(11)
    m = 10
    J = np.diag(np.concatenate([[2.5, 2.5], np.linspace(0.3, 1.9, m - 2)]))
    J[0, 1] = 1.0
    S = rng.standard_normal((m, m)) + 3 * np.eye(m)
    H = S @ J @ np.linalg.inv(S)
    y, th = rb.harmonic_ritz(np.eye(m), H, 2)
    assert len(th) == 2
    assert np.abs(np.asarray(th) - 0.4).max() <= 1e-6
    Qb, _ = np.linalg.qr(S[:, :2])
    u = y[:, 0] / np.linalg.norm(y[:, 0])
    assert np.linalg.norm(u - Qb @ (Qb.T @ u)) <= 1e-6
    y_all, th_all = rb.harmonic_ritz(np.eye(m), H, m)
    want = np.sort(1.0 / np.diag(J))
    assert np.abs(np.sort(np.real(th_all)) - want).max() <= 1e-6


def test_noalloc_wrapper_rejects_host_arrays(L):
    """The allocation-free residual wrapper checks its arguments before it
    takes any pointer: host arrays raise RbError(RB_EINVAL)."""
    rp = np.array([0, 1], dtype=np.int32)
    col = np.array([0], dtype=np.int32)
    v = np.ones(1)
    with pytest.raises(rb.RbError) as e:
        rb.residual_noalloc(rp, col, v, v, v, v.copy(), np.zeros(1))
    assert e.value.code == rb.C["RB_EINVAL"]
