"""Plain BiCGSTAB (van der Vorst, 1992), the no-recycling baseline.

Written separately from ``oracle.rbicgstab`` so that the statement "Alg. 2
with an empty recycle space is BiCGSTAB" (Sec. 4, where U and U~ empty make
C, C-hat empty and every projection vanish) can be checked between two
independent codes.  FP64, scipy.sparse matvec, numpy dots.

Convergence test: ||r_i|| <= tol * ||b|| on the recursively updated residual
(the paper's experiments use a relative tolerance, Sec. 6.2).  A half step
whose s already meets the test ends the solve with x += alpha p.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .shadow import DEFAULT_SEED, shadow_vector

OK, NOTCONV, BREAKDOWN_RHO, BREAKDOWN_OMEGA = 0, -7, -8, -9


@dataclass
class PlainInfo:
    iters: int = 0
    matvecs: int = 0
    status: int = OK
    relres: float = float("nan")
    history: list = field(default_factory=list)   # ||r_i|| / ||b|| per iteration
    iterates: list = field(default_factory=list)  # x_i (only when record=True)


def bicgstab(A, b, x0=None, tol=1e-8, max_itn=None, shadow_seed=DEFAULT_SEED,
             rt=None, record=False):
    """Solve A x = b by BiCGSTAB; returns (x, PlainInfo)."""
    n = b.shape[0]
    if max_itn is None:
        max_itn = min(n, 20000)
    info = PlainInfo()
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if x0 is None or not np.any(x):
        r = b.astype(np.float64).copy()
    else:
        r = b - A @ x
        info.matvecs += 1
    if rt is None:
        rt = shadow_vector(n, shadow_seed)
    bnorm = np.linalg.norm(b)
    thresh = tol * bnorm
    if np.linalg.norm(r) <= thresh:
        info.relres = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
        return x, info
    rho_old = alpha = omega = 1.0
    p = np.zeros(n)
    v = np.zeros(n)
    for it in range(1, max_itn + 1):
        rho = np.dot(rt, r)
        if rho == 0.0:
            info.status = BREAKDOWN_RHO
            break
        if it == 1:
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = A @ p
        info.matvecs += 1
        rtv = np.dot(rt, v)
        if rtv == 0.0:                # (r~, v) = 0: alpha undefined
            info.status = BREAKDOWN_RHO
            break
        alpha = rho / rtv
        s = r - alpha * v
        snorm = np.linalg.norm(s)
        if snorm <= thresh:
            x = x + alpha * p
            r = s
            info.iters = it
            info.history.append(snorm / bnorm)
            if record:
                info.iterates.append(x.copy())
            break
        t = A @ s
        info.matvecs += 1
        tt = np.dot(t, t)
        if tt == 0.0:
            info.status = BREAKDOWN_OMEGA
            break
        omega = np.dot(t, s) / tt
        if omega == 0.0:
            info.status = BREAKDOWN_OMEGA
            break
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        info.iters = it
        rn = np.linalg.norm(r)
        info.history.append(rn / bnorm)
        if record:
            info.iterates.append(x.copy())
        if rn <= thresh:
            break
    else:
        info.status = NOTCONV
    info.relres = np.linalg.norm(r) / bnorm
    if info.status == OK and info.history and info.history[-1] > tol:
        info.status = NOTCONV
    return x, info
