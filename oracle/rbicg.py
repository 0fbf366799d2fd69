"""Alg. 1 (RBiCG) of Sec. 4 in FP64: BiCG on the projected primary and dual operators.

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module; the CUDA library never does.

RBiCG solves the primary system A x = b and the dual system A^T x~ = b~
together (real arithmetic here, so conj(alpha) = alpha and conj(beta) =
beta).  With a recycle space U, U~ (C = A U, C~ = A^T U~ biorthogonal,
C-hat = C~ D_c^{-1}, C-check = C D_c^{-1}, eq. (3.4)) the primary iteration
runs on the projected operator (I - C C-hat^T) A and the dual on
(I - C~ C-check^T) A^T; the final correction folds the accumulated
coefficients back.

Readings where the paper is silent (each listed in the design notes):

* The dual right-hand side b~ is the caller's; the shadow vector of Alg. 2
  serves when none is given.
* Initial vectors follow eq. (3.5) for both systems:
  x_0 = x_{-1} + U C-hat^T r_{-1},     r_0 = r_{-1} - C C-hat^T r_{-1},
  x~_0 = x~_{-1} + U~ C-check^T r~_{-1}, r~_0 = r~_{-1} - C~ C-check^T r~_{-1}.
* (r_0, r~_0) = 0 at the start: x~_{-1} becomes the shadow vector with seed
  + attempt (at most 3 redraws), and x~_0, r~_0 are formed again.
* Convergence: ||r_i|| <= tol ||b|| and ||r~_i|| <= tol ||b~|| on the
  recursive residuals (relative, as for Alg. 2).  A start that meets both
  returns at once.
* Breakdowns: (p~_i, q_i) = 0 or (r~_i, r_i) = 0 stop the solve with a
  breakdown status (no look-ahead, Sec. 4).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rbicgstab import NOTCONV, OK, RecycleSpace, empty_space
from .shadow import DEFAULT_SEED, shadow_vector

BREAKDOWN_PQ = -8   # (p~_i, q_i) = 0 or (r~_i, r_i) = 0: the library's RB_EBREAKDOWN_RHO


@dataclass
class RBiCGInfo:
    iters: int = 0
    matvecs: int = 0          # A and A^T products of the iteration
    status: int = OK
    relres: float = float("nan")         # ||r_i|| / ||b||
    relres_dual: float = float("nan")    # ||r~_i|| / ||b~||
    seeds_used: int = 0
    iterates: list = field(default_factory=list)   # (x_i, zeta_c, r_i, x~_i, zeta~_c, r~_i) when record=True
    residuals: list = field(default_factory=list)  # (r_i, r~_i) for i = 0.. when record=True
    P: list = field(default_factory=list)          # (p_i, p~_i) when record=True


def rbicg(A, b, bt=None, rec: RecycleSpace | None = None, x_m1=None, xt_m1=None, tol=1e-8,
          max_itn=None, shadow_seed=DEFAULT_SEED, record=False):
    """Alg. 1.  Returns (x, x~, RBiCGInfo)."""
    n = b.shape[0]
    if rec is None:
        rec = empty_space(n)
    if max_itn is None:
        max_itn = min(n, 20000)
    info = RBiCGInfo()
    U, Ut, C, Ct, Chat, Ccheck = rec.U, rec.Ut, rec.C, rec.Ct, rec.Chat, rec.Ccheck
    b = np.asarray(b, dtype=np.float64)
    bt = shadow_vector(n, shadow_seed) if bt is None else np.asarray(bt, dtype=np.float64)
    bnorm, btnorm = np.linalg.norm(b), np.linalg.norm(bt)
    thresh, thresh_t = tol * bnorm, tol * btnorm

    # eq. (3.5) for the primary system
    if x_m1 is None or not np.any(x_m1):
        x_m1, r_m1 = np.zeros(n), b.copy()
    else:
        x_m1 = np.asarray(x_m1, dtype=np.float64)
        r_m1 = b - A @ x_m1
    x = x_m1 + U @ (Chat.T @ r_m1)
    r = r_m1 - C @ (Chat.T @ r_m1)

    def dual_start(xt_start):
        if xt_start is None or not np.any(xt_start):
            xs, rs = np.zeros(n), bt.copy()
        else:
            xs = np.asarray(xt_start, dtype=np.float64)
            rs = bt - A.T @ xs
        return xs + Ut @ (Ccheck.T @ rs), rs - Ct @ (Ccheck.T @ rs)

    # eq. (3.5) for the dual system; redraw x~_{-1} while (r_0, r~_0) = 0
    xt, rt = dual_start(xt_m1)
    rho = np.dot(rt, r)
    for attempt in range(3):
        if rho != 0.0:
            break
        xt, rt = dual_start(shadow_vector(n, shadow_seed + attempt))
        rho = np.dot(rt, r)
        info.seeds_used = attempt + 1
    # first search directions
    p, pt = np.zeros(n), np.zeros(n)
    zc, ztc = np.zeros(rec.k), np.zeros(rec.k)
    beta = 0.0
    if record:
        info.residuals.append((r.copy(), rt.copy()))

    def done(status, i):
        info.status = status
        info.iters = i
        info.relres = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
        info.relres_dual = np.linalg.norm(rt) / btnorm if btnorm > 0 else 0.0
        # final correction of both systems
        return x - U @ zc, xt - Ut @ ztc, info

    if np.linalg.norm(r) <= thresh and np.linalg.norm(rt) <= thresh_t:
        return done(OK, 0)
    if rho == 0.0:
        return done(BREAKDOWN_PQ, 0)
    for i in range(1, max_itn + 1):
        # the iteration; left column: primary; right column: dual
        p = r + beta * p
        pt = rt + beta * pt
        z = A @ p
        zt = A.T @ pt
        info.matvecs += 2
        zeta = Chat.T @ z
        zetat = Ccheck.T @ zt
        q = z - C @ zeta
        qt = zt - Ct @ zetat
        if record:
            info.P.append((p.copy(), pt.copy()))
        ptq = np.dot(pt, q)
        if ptq == 0.0:
            return done(BREAKDOWN_PQ, i - 1)
        alpha = np.dot(rt, r) / ptq
        zc = zc + alpha * zeta
        ztc = ztc + alpha * zetat
        x = x + alpha * p
        xt = xt + alpha * pt
        r = r - alpha * q
        rt = rt - alpha * qt
        if record:
            info.iterates.append((x.copy(), zc.copy(), r.copy(), xt.copy(), ztc.copy(), rt.copy()))
            info.residuals.append((r.copy(), rt.copy()))
        if np.linalg.norm(r) <= thresh and np.linalg.norm(rt) <= thresh_t:
            return done(OK, i)
        rho_new = np.dot(rt, r)
        if rho_new == 0.0:
            return done(BREAKDOWN_PQ, i)
        beta = rho_new / rho
        rho = rho_new
    return done(NOTCONV, max_itn)
