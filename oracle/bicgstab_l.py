"""BiCGstab(l) (Sleijpen and Fokkema, 1993), plain and on the recycling
projected operator: the breakdown-robust variant the paper names as future
work next to its remark on the omega = 0 breakdown of BiCGSTAB (Sec. 4,
Sec. 7).  FP64, written from the published method.

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module; the CUDA library never does.

Each outer step takes l BiCG steps (two products each) and then minimises
the residual over the span of r, A r, ..., A^l r (modified Gram-Schmidt on
the residual block), so the stabilising polynomial has degree l instead of
BiCGSTAB's product of degree-1 factors; for l = 1 the method is BiCGSTAB.
With l >= 2 a matrix whose spectrum lies near the imaginary axis (where
BiCGSTAB's omega = (t, s) / (t, t) tends to 0) no longer stalls.

Recycling (Sec. 3): with the recycle space U, C = A U, C-hat = C~ D_c^{-1}
(C-hat^T C = I) the iteration runs on the projected operator
B = (I - C C-hat^T) A from x_0, r_0 of eq. (3.5) and shadow
r~_0 = r~_{-1} - C~ C-check^T r~_{-1} (eq. (3.5)).  If y is the sum of
the Krylov corrections, x = x_0 + y - U C-hat^T A y has the residual
r_0 - B y, the residual the iteration updates; C-hat^T A y is accumulated
from the projection coefficients of every product (Alg. 2's x_c).  With
l = 1 this is Alg. 2.

Readings: convergence ||r|| <= tol ||b|| is tested after every outer step
(the BiCG steps inside one do not test); iteration counts are BiCG steps
(l per outer step); a zero (r~_0, r_j) or (r~_0, u_{j+1}) is the rho
breakdown, a zero residual block norm in the minimisation the omega one.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rbicgstab import BREAKDOWN_OMEGA, BREAKDOWN_RHO, NOTCONV, OK, RecycleSpace, empty_space
from .shadow import DEFAULT_SEED, shadow_vector


@dataclass
class LInfo:
    iters: int = 0          # BiCG steps (l per outer step)
    outer: int = 0
    matvecs: int = 0
    status: int = OK
    relres: float = float("nan")
    iterates: list = field(default_factory=list)   # x after each outer step when record=True


def bicgstab_l(A, b, ell=2, rec: RecycleSpace | None = None, x_m1=None, tol=1e-8, max_itn=None,
               shadow_seed=DEFAULT_SEED, record=False):
    """Solve A x = b by BiCGstab(ell) on B = (I - C C-hat^T) A; returns (x, LInfo)."""
    if ell < 1:
        raise ValueError("ell >= 1")
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    rec = empty_space(n) if rec is None else rec
    if max_itn is None:
        max_itn = min(n, 20000)
    U, C, Ct, Chat, Ccheck = rec.U, rec.C, rec.Ct, rec.Chat, rec.Ccheck
    info = LInfo()
    bnorm = np.linalg.norm(b)
    thresh = tol * bnorm

    def B(v):
        """(I - C C-hat^T) A v and the coefficients C-hat^T A v."""
        w = A @ v
        info.matvecs += 1
        z = Chat.T @ w
        return w - C @ z, z

    # eq. (3.5) and the projected shadow, redrawn while (r~_0, r_0) = 0
    if x_m1 is None or not np.any(x_m1):
        x_m1, r_m1 = np.zeros(n), b.copy()
    else:
        x_m1 = np.asarray(x_m1, dtype=np.float64)
        r_m1 = b - A @ x_m1
        info.matvecs += 1
    x0 = x_m1 + U @ (Chat.T @ r_m1)
    r0 = r_m1 - C @ (Chat.T @ r_m1)
    rt_m1 = shadow_vector(n, shadow_seed)
    rt = rt_m1 - Ct @ (Ccheck.T @ rt_m1)

    # y: the Krylov correction; xc = C-hat^T A y; r[j], u[j] with their
    # coefficient vectors zr[j] = C-hat^T A (the vector whose B-image r[j] is)
    y = np.zeros(n)
    xc = np.zeros(rec.k)
    r = [r0.copy()] + [np.zeros(n) for _ in range(ell)]
    u = [np.zeros(n) for _ in range(ell + 1)]
    zr = [None] + [np.zeros(rec.k) for _ in range(ell)]   # r[j] = B r[j-1]: coefficients of that product
    zu = [None] + [np.zeros(rec.k) for _ in range(ell)]   # u[j] = B u[j-1]
    rho0 = alpha = omega = 1.0

    def done(status):
        info.status = status
        info.relres = np.linalg.norm(r[0]) / bnorm if bnorm > 0 else 0.0
        return x0 + y - U @ xc, info

    if np.linalg.norm(r[0]) <= thresh:
        return done(OK)
    while info.iters + ell <= max_itn:
        rho0 = -omega * rho0
        # BiCG part: l steps
        for j in range(ell):
            rho1 = np.dot(rt, r[j])
            if rho1 == 0.0 or rho0 == 0.0:
                return done(BREAKDOWN_RHO)
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
                if i >= 1:
                    zu[i] = zr[i] - beta * zu[i]
            u[j + 1], zu[j + 1] = B(u[j])
            gamma = np.dot(rt, u[j + 1])
            if gamma == 0.0:
                return done(BREAKDOWN_RHO)
            alpha = rho0 / gamma
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
                if i >= 1:
                    zr[i] = zr[i] - alpha * zu[i + 1]
            r[j + 1], zr[j + 1] = B(r[j])
            y = y + alpha * u[0]
            xc = xc + alpha * zu[1]
            info.iters += 1
        # MR part: minimise ||r[0] - sum_j g_j r[j]|| by modified Gram-Schmidt
        # on r[1..l].  c[j] = C-hat^T A r[j] (j < l) is zr[j + 1], the
        # coefficients of the product r[j + 1] = B r[j]; ch[j] follows the
        # orthogonalised r[j] through the same combinations.
        c = [zr[j + 1].copy() for j in range(ell)]
        tau = np.zeros((ell + 1, ell + 1))
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1)
        ch = [None] * ell
        for j in range(1, ell + 1):
            cj = c[j].copy() if j < ell else None
            for i in range(1, j):
                tau[i, j] = np.dot(r[j], r[i]) / sigma[i]
                r[j] = r[j] - tau[i, j] * r[i]
                if cj is not None:
                    cj = cj - tau[i, j] * ch[i]
            if j < ell:
                ch[j] = cj
            sigma[j] = np.dot(r[j], r[j])
            if sigma[j] == 0.0:
                return done(BREAKDOWN_OMEGA)
            gp[j] = np.dot(r[0], r[j]) / sigma[j]
        g = np.zeros(ell + 1)
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1)
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        if omega == 0.0:
            return done(BREAKDOWN_OMEGA)
        y = y + g[1] * r[0]
        xc = xc + g[1] * c[0]
        r[0] = r[0] - gp[ell] * r[ell]
        u[0] = u[0] - g[ell] * u[ell]
        for j in range(1, ell):
            u[0] = u[0] - g[j] * u[j]
            y = y + gpp[j] * r[j]
            xc = xc + gpp[j] * ch[j]
            r[0] = r[0] - gp[j] * r[j]
        info.outer += 1
        if record:
            info.iterates.append(x0 + y - U @ xc)
        if np.linalg.norm(r[0]) <= thresh:
            return done(OK)
    return done(NOTCONV)
