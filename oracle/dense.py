"""Small dense helpers for the oracle's pins.

``principal_cosines(X, Y)``: cosines of the principal angles between
range(X) and range(Y) (Bjorck and Golub, 1973): orthonormalise both by QR,
then the singular values of Q_X^T Q_Y, in descending order.  Table 1 of Sec. 5
lists such cosines between left and right invariant subspaces.

``invariant_subspaces(A, m)``: right and left invariant subspaces of a dense
matrix for its m eigenvalues of smallest magnitude, as real bases (a complex
pair contributes its real and imaginary parts).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def principal_cosines(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    Qx, _ = np.linalg.qr(X)
    Qy, _ = np.linalg.qr(Y)
    s = np.linalg.svd(Qx.T @ Qy, compute_uv=False)
    return np.clip(s, 0.0, 1.0)


def _real_basis(vals, vecs, order, m):
    cols, used = [], 0
    for j in order:
        if used >= m:
            break
        v = vecs[:, j]
        if vals[j].imag == 0.0:
            cols.append(v.real)
            used += 1
        elif vals[j].imag > 0.0:
            cols += [v.real, v.imag]
            used += 2
    return np.column_stack(cols[:m])


def invariant_subspaces(A: np.ndarray, m: int):
    """(right basis, left basis, eigenvalues) for the m smallest-|lambda| eigenvalues."""
    w, vl, vr = sla.eig(A, left=True, right=True)
    order = np.argsort(np.abs(w), kind="stable")
    R = _real_basis(w, vr, order, m)
    L = _real_basis(w, vl, order, m)
    return R, L, w[order[:m]]
