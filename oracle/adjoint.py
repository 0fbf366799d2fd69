"""Gradient of an output functional of the solution through the dual system.

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module; the CUDA library never does.

For A(p) x = b with A(p) = sum_k p_k A_k and the output functional
L = ||C_out x||^2, the dual system of Sec. 2 (A^* x~ = b~, real here, so
A^* = A^T) with right-hand side b~ = dL/dx = 2 C_out^T C_out x gives the
whole gradient from one extra solve:

    A^T lam = 2 C_out^T C_out x
    dL/db      = lam
    dL/dA_ij   = -lam_i x_j           (on the sparsity pattern of A)
    dL/dp_k    = -lam^T A_k x

(differentiate A x = b: A dx = db - dA x, so dL = (dL/dx)^T dx =
lam^T (db - dA x)).  This is the case Sec. 2 names where the dual system is
of interest rather than auxiliary.

Recycling: the primary system's space is U (C = A U) with left space U~
(C~ = A^T U~), Sec. 3.  For the dual solve A^T is the operator, so the roles
swap: its right space is U~ (A^T U~ = C~) and its left space U ((A^T)^T U =
C); Alg. 2 run on A^T with (U~, U) therefore reuses exactly the products C~
and C of the primary setup.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .rbicgstab import RecycleSpace, SolveInfo, rbicgstab, recycle_setup


@dataclass
class Gradient:
    x: np.ndarray          # primary solution
    lam: np.ndarray        # dual solution (dL/db)
    loss: float            # ||C_out x||^2
    grad_p: np.ndarray     # dL/dp_k
    grad_vals: np.ndarray  # dL/dA_ij on the pattern (CSR order of A)
    info: SolveInfo
    info_dual: SolveInfo


def loss(C_out: np.ndarray, x: np.ndarray) -> float:
    """L = ||C_out x||^2."""
    y = C_out @ x
    return float(y @ y)


def dual_space(A, rec: RecycleSpace | None) -> RecycleSpace | None:
    """The recycle space of the dual operator A^T: right space U~, left U."""
    if rec is None or rec.k == 0:
        return None
    return recycle_setup(sp.csr_matrix(A.T), rec.Ut, rec.U)


def adjoint_gradient(A, b, C_out, basis, rec: RecycleSpace | None = None, tol=1e-8,
                     max_itn=None) -> Gradient:
    """L, x and the gradient of L with respect to b, the entries of A and the
    parameters p (``basis[k]`` = A_k as a sparse matrix, or as values on the
    pattern of ``A``), each solve by Alg. 2."""
    A = sp.csr_matrix(A)
    x, info = rbicgstab(A, b, rec, tol=tol, max_itn=max_itn)
    g = 2.0 * (C_out.T @ (C_out @ x))
    At = sp.csr_matrix(A.T)
    lam, info_t = rbicgstab(At, g, dual_space(A, rec), tol=tol, max_itn=max_itn)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    grad_vals = -lam[rows] * x[A.indices]
    grad_p = np.empty(len(basis))
    for kk, Ak in enumerate(basis):
        if not sp.issparse(Ak):
            Ak = sp.csr_matrix((np.asarray(Ak, dtype=np.float64), A.indices, A.indptr), shape=A.shape)
        grad_p[kk] = -(lam @ (Ak @ x))
    return Gradient(x=x, lam=lam, loss=loss(C_out, x), grad_p=grad_p, grad_vals=grad_vals,
                    info=info, info_dual=info_t)
