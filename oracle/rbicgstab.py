"""Alg. 2 (RBiCGSTAB) of Sec. 4, in FP64, step by step as the paper states it.

Notation follows the paper: U, U~ (``Ut``) span the recycle space; C = A U,
C~ = A^T U~ (Sec. 3, definition of the recycle space); D_c = C~^T C diagonal
with positive entries; C-hat = C~ D_c^{-1}, C-check = C D_c^{-1}
(eq. (3.4), "CcheckChat"); x_0, r_0, r~_0 from eq. (3.5) ("minusXR").

Readings where the paper is silent (each listed in the design notes):

* Biorthogonalisation (Sec. 3 requires C and C~ biorthogonal but points to a
  thesis for how): SVD of M = C~^T C = P Sigma Q^T, then U <- U Q, C <- C Q,
  U~ <- U~ P, C~ <- C~ P, so C~^T C = Sigma.  Columns with
  sigma_j < 1e-12 sigma_1 are dropped (k_used < k).
* U~ = U when no left space is given (the right-only variant of Sec. 5).
* Convergence: ||r_i|| <= tol ||b|| on the recursive residual; a start with
  ||r_0|| <= tol ||b|| returns immediately.  A half step whose s meets the
  test ends with x += alpha p, x_c += alpha zeta, r = s.
* (r_0, r~_0) = 0 (step 3): redraw r~_{-1} with seed + 1, at most 3 times.
* (r~_0, q_i) = 0 or (r~_0, r_i) = 0 inside the iteration leaves alpha or
  beta undefined: the solve stops with the rho breakdown status (no
  look-ahead, as for step 3); (t, t) = 0 or omega = 0 stop it with the omega
  breakdown status.
* Matvec counting: one per A-product in the iteration, one for r_{-1} when
  x_{-1} != 0, and setup products (C = A U, C~ = A^T U~) counted apart.

Everything here is computed literally: alpha from (r~_0, r_{i-1}) / (r~_0, q_i),
r_i = r_{i-1} - alpha q_i - omega t_i, beta from (r~_0, r_i) / (r~_0, r_{i-1}).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .shadow import DEFAULT_SEED, shadow_vector

OK, NOTCONV, BREAKDOWN_RHO, BREAKDOWN_OMEGA = 0, -7, -8, -9
SVD_DROP = 1e-12


@dataclass
class RecycleSpace:
    """U, U~, C = A U, C~ = A^T U~ (biorthogonal), D_c, C-hat, C-check."""

    U: np.ndarray
    Ut: np.ndarray
    C: np.ndarray
    Ct: np.ndarray
    Dc: np.ndarray
    Chat: np.ndarray
    Ccheck: np.ndarray
    setup_matvecs: int = 0

    @property
    def k(self) -> int:
        return self.U.shape[1]


def empty_space(n: int) -> RecycleSpace:
    z = np.zeros((n, 0))
    return RecycleSpace(z, z, z, z, np.zeros(0), z, z, 0)


def recycle_setup(A, U, Ut=None, drop=SVD_DROP) -> RecycleSpace:
    """Alg. 2 step 1: C = A U, C~ = A^T U~, biorthogonalised; D_c, C-hat, C-check."""
    n = A.shape[0]
    if U is None or U.shape[1] == 0:
        return empty_space(n)
    U = np.asarray(U, dtype=np.float64)
    Ut = U if Ut is None else np.asarray(Ut, dtype=np.float64)
    k = U.shape[1]
    C = np.column_stack([A @ U[:, j] for j in range(k)])
    Ct = np.column_stack([A.T @ Ut[:, j] for j in range(k)])
    M = Ct.T @ C
    P, sig, Qt = np.linalg.svd(M)
    if sig[0] == 0.0:
        return empty_space(n)
    keep = sig >= drop * sig[0]
    Q = Qt.T[:, keep]
    P = P[:, keep]
    Dc = sig[keep]
    U2, C2 = U @ Q, C @ Q
    Ut2, Ct2 = Ut @ P, Ct @ P
    return RecycleSpace(U=U2, Ut=Ut2, C=C2, Ct=Ct2, Dc=Dc,
                        Chat=Ct2 / Dc[None, :], Ccheck=C2 / Dc[None, :],
                        setup_matvecs=2 * k)


@dataclass
class CycleStore:
    """Vectors kept during one cycle of the solve for the recycle update:
    p_i, s_i and their products A p_i, A s_i before projection."""

    P: list = field(default_factory=list)
    S: list = field(default_factory=list)
    AP: list = field(default_factory=list)
    AS: list = field(default_factory=list)

    def __len__(self):
        return len(self.P)

    def W(self):
        return self.P + self.S

    def AW(self):
        return self.AP + self.AS


@dataclass
class SolveInfo:
    iters: int = 0
    matvecs: int = 0
    status: int = OK
    relres_rec: float = float("nan")
    relres_true: float = float("nan")
    history: list = field(default_factory=list)
    iterates: list = field(default_factory=list)   # (x_i, x_c, r_i) when record=True
    seeds_used: int = 1
    rt0: np.ndarray | None = None
    r0: np.ndarray | None = None


def rbicgstab(A, b, rec: RecycleSpace | None = None, x_m1=None, tol=1e-8, max_itn=None,
              shadow_seed=DEFAULT_SEED, record=False, cycle_s=None, on_cycle=None,
              true_residual=True):
    """Alg. 2.  Returns (x, SolveInfo).

    ``cycle_s`` / ``on_cycle``: every ``cycle_s`` iterations (and once more for
    a final partial cycle) ``on_cycle(store)`` is called with the CycleStore
    of that cycle; the recycle-space update (``oracle.recycle``) hooks in here.
    """
    n = b.shape[0]
    if rec is None:
        rec = empty_space(n)
    if max_itn is None:
        max_itn = min(n, 20000)
    info = SolveInfo()
    U, C, Ct, Chat, Ccheck = rec.U, rec.C, rec.Ct, rec.Chat, rec.Ccheck
    b = np.asarray(b, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    thresh = tol * bnorm

    # step 2: x_{-1}, r_{-1}; random r~_{-1}; eq. (3.5)
    if x_m1 is None or not np.any(x_m1):
        x_m1 = np.zeros(n)
        r_m1 = b.copy()
    else:
        x_m1 = np.asarray(x_m1, dtype=np.float64)
        r_m1 = b - A @ x_m1
        info.matvecs += 1
    x = x_m1 + U @ (Chat.T @ r_m1)
    r = r_m1 - C @ (Chat.T @ r_m1)
    # step 3: (r_0, r~_0) = 0 -> redraw r~_{-1}
    for attempt in range(4):
        rt_m1 = shadow_vector(n, shadow_seed + attempt)
        rt0 = rt_m1 - Ct @ (Ccheck.T @ rt_m1)
        rho_prev = np.dot(rt0, r)
        info.seeds_used = attempt + 1
        if rho_prev != 0.0:
            break
    info.rt0, info.r0 = rt0, r.copy()
    # step 4
    beta = omega = 0.0
    p = np.zeros(n)
    q = np.zeros(n)
    xc = np.zeros(rec.k)
    store = CycleStore()

    def flush():
        nonlocal store
        if on_cycle is not None and len(store) > 0:
            on_cycle(store)
        store = CycleStore()

    if np.linalg.norm(r) <= thresh:
        info.relres_rec = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
        info.relres_true = info.relres_rec
        return x - U @ xc, info
    if rho_prev == 0.0:
        info.status = BREAKDOWN_RHO
        info.relres_rec = np.linalg.norm(r) / bnorm
        return x - U @ xc, info

    converged = False
    for i in range(1, max_itn + 1):
        p = r + beta * p - beta * omega * q
        q = A @ p
        info.matvecs += 1
        if cycle_s:
            store.P.append(p.copy())
            store.AP.append(q.copy())
        zeta = Chat.T @ q
        q = q - C @ zeta
        rtq = np.dot(rt0, q)
        if rtq == 0.0:                            # (r~_0, q_i) = 0: no alpha (reading, module doc)
            info.status = BREAKDOWN_RHO
            info.iters = i - 1
            break
        alpha = np.dot(rt0, r) / rtq
        s = r - alpha * q
        if np.linalg.norm(s) <= thresh:          # half step (reading, see module doc)
            x = x + alpha * p
            xc = xc + alpha * zeta
            r = s
            info.iters = i
            info.history.append(np.linalg.norm(r) / bnorm)
            if record:
                info.iterates.append((x.copy(), xc.copy(), r.copy()))
            converged = True
            break
        t = A @ s
        info.matvecs += 1
        if cycle_s:
            store.S.append(s.copy())
            store.AS.append(t.copy())
        gamma = Chat.T @ t
        t = t - C @ gamma
        tt = np.dot(t, t)
        if tt == 0.0:
            info.status = BREAKDOWN_OMEGA
            info.iters = i - 1
            break
        omega = np.dot(s, t) / tt
        if omega == 0.0:
            info.status = BREAKDOWN_OMEGA
            info.iters = i - 1
            break
        x = x + alpha * p + omega * s
        xc = xc + alpha * zeta + omega * gamma
        r_prev = r
        r = r - alpha * q - omega * t
        info.iters = i
        rn = np.linalg.norm(r)
        info.history.append(rn / bnorm)
        if record:
            info.iterates.append((x.copy(), xc.copy(), r.copy()))
        if cycle_s and i % cycle_s == 0:
            flush()
        if rn <= thresh:
            converged = True
            break
        rho = np.dot(rt0, r)
        if rho == 0.0:                            # (r~_0, r_i) = 0: no beta (reading, module doc)
            info.status = BREAKDOWN_RHO
            break
        beta = (rho / np.dot(rt0, r_prev)) * (alpha / omega)
    if cycle_s:
        flush()
    if not converged and info.status == OK:
        info.status = NOTCONV
    # step 8
    x = x - U @ xc
    info.relres_rec = np.linalg.norm(r) / bnorm
    if true_residual:
        info.relres_true = np.linalg.norm(b - A @ x) / bnorm
    return x, info
