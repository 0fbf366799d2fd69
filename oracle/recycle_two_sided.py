"""Two-sided recycle-space update from RBiCG cycles ("mode P"), FP64.

Sec. 6.2 calls RBiCG (Alg. 1) whenever the matrix changes because it yields
approximations to both left and right invariant subspaces; the selection
rule is deferred to the RBiCG paper.  This oracle takes the Petrov-Galerkin
reading on the spaces of a cycle: with W = [U, p_1..p_s] (primary search
directions) and W~ = [U~, p~_1..p~_s] (dual ones),

    right:  W~^T A W y = theta W~^T W y,
    left:   z^T W~^T A W = theta z^T W~^T W,

keep the k pairs of smallest |theta| (a complex pair as its real and
imaginary parts; a pair split at k is dropped), U = W y, U~ = W~ z, columns
scaled to unit norm.  The same eigenvalues serve both sides.

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module; the CUDA library never does.

Measured on the 2D convection-diffusion sequences (see the design notes):
the pairs this produces are nearly orthogonal after biorthogonalisation, so
the space is kept in the oracle and not carried to the GPU.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _real_basis(vals, vecs, order, k):
    """Real basis of the eigenvectors taken in ``order`` up to k columns."""
    cols, taken = [], set()
    for j in order:
        if len(cols) >= k:
            break
        if j in taken:
            continue
        lam, v = vals[j], vecs[:, j]
        if abs(lam.imag) > 1e-13 * max(1.0, abs(lam)):
            if len(cols) + 2 > k:
                break
            cols += [v.real, v.imag]
            mate = int(np.argmin(np.abs(vals - np.conj(lam)) + np.where(np.arange(len(vals)) == j, np.inf, 0.0)))
            taken.add(mate)
        else:
            cols.append(v.real)
        taken.add(j)
    return np.column_stack(cols) if cols else np.zeros((vecs.shape[0], 0))


def petrov_galerkin_update(A, W, Wt, k):
    """(U, U~, theta): the k smallest-|theta| right and left Petrov-Galerkin
    vectors of A on (range W, range W~)."""
    F = Wt.T @ (A @ W)
    E = Wt.T @ W
    vals, vl, vr = sla.eig(F, E, left=True, right=True)
    finite = np.isfinite(vals)
    order = [int(j) for j in np.argsort(np.where(finite, np.abs(vals), np.inf)) if finite[j]]
    Y = _real_basis(vals, vr, order, k)
    Z = _real_basis(vals, vl.conj(), order, k)
    m = min(Y.shape[1], Z.shape[1])
    U, Ut = W @ Y[:, :m], Wt @ Z[:, :m]
    U = U / np.linalg.norm(U, axis=0)
    Ut = Ut / np.linalg.norm(Ut, axis=0)
    sel = []
    for j in order:
        if len(sel) >= m:
            break
        sel.append(vals[j])
    return U, Ut, np.array(sel)
