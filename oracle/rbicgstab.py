"""RBiCGSTAB (Alg. 2 of Sec. 4) in FP64: BiCGSTAB on the projected operator.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports this module.

The method, restated from its definitions:

* Recycle space (Sec. 3).  U, U~ (``Ut``) span the right and left recycle
  spaces; C = A U and C~ = A^T U~ are made biorthogonal, so that
  D_c = C~^T C is diagonal with positive entries; C-hat = C~ D_c^{-1} and
  C-check = C D_c^{-1} (eq. (3.4)).  C C-hat^T is then the oblique projector
  onto range(C) along the orthogonal complement of range(C~).
* Projected operator (Sec. 3).  B = (I - C C-hat^T) A.  Its products are what
  the iteration needs: for v, the raw product A v, the coefficients
  C-hat^T A v, and B v = A v - C (C-hat^T A v).
* Start (eq. (3.5)).  From x_{-1} and r_{-1} = b - A x_{-1}:
  x_0 = x_{-1} + U C-hat^T r_{-1}, r_0 = (I - C C-hat^T) r_{-1}, and the
  shadow r~_0 = (I - C~ C-check^T) r~_{-1} from a random r~_{-1}.
* Iteration (Sec. 4).  Plain BiCGSTAB (van der Vorst) for B y = r_0 with
  shadow r~_0, written in x directly: every product of B contributes its
  coefficients C-hat^T A v, times the step length it enters x with, to the
  k-vector x_c.
* End (Alg. 2).  x = x_i - U x_c, which turns the approximate solution of the
  projected system into one of A x = b.

Readings where the paper is silent (each listed in the design notes):

* Biorthogonalisation (Sec. 3 requires C and C~ biorthogonal but points to a
  thesis for how): SVD of M = C~^T C = P Sigma Q^T, then U <- U Q, C <- C Q,
  U~ <- U~ P, C~ <- C~ P, so C~^T C = Sigma.  Columns with
  sigma_j < 1e-12 sigma_1 are dropped (k_used < k).
* U~ = U when no left space is given (the right-only variant of Sec. 5).
* Convergence: ||r_i|| <= tol ||b|| on the recursive residual; a start with
  ||r_0|| <= tol ||b|| returns immediately.  A half step whose s meets the
  test ends with x += alpha p, x_c += alpha zeta, r = s.
* (r_0, r~_0) = 0 at the start: redraw r~_{-1} with seed + 1, at most 3
  times.
* (r~_0, q_i) = 0 or (r~_0, r_i) = 0 inside the iteration leaves alpha or
  beta undefined: the solve stops with the rho breakdown status (no
  look-ahead, as at the start); (t, t) = 0 or omega = 0 stop it with the
  omega breakdown status.
* Matvec counting: one per A-product in the iteration, one for r_{-1} when
  x_{-1} != 0, and setup products (C = A U, C~ = A^T U~) counted apart.

The inner products are formed literally: alpha = (r~_0, r_{i-1}) / (r~_0, q_i),
beta = ((r~_0, r_i) / (r~_0, r_{i-1})) (alpha / omega).
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
    """The recycle space of Sec. 3 for matrix A: C = A U, C~ = A^T U~,
    biorthogonalised through the SVD of C~^T C; D_c, C-hat, C-check (eq. (3.4))."""
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


def project_product(A, rec: RecycleSpace, v):
    """Product with B = (I - C C-hat^T) A (Sec. 3): returns (A v, C-hat^T A v, B v)."""
    raw = A @ v
    coef = rec.Chat.T @ raw
    return raw, coef, raw - rec.C @ coef


def initial_projection(A, b, rec: RecycleSpace, x_m1, shadow_seed):
    """Eq. (3.5): x_0, r_0 and the shadow r~_0 from x_{-1} and a random r~_{-1}.

    Returns (x_0, r_0, r~_0, (r~_0, r_0), number of r~_{-1} drawn, matvecs).
    r~_{-1} is drawn again (seed + 1, at most 3 more times) while
    (r~_0, r_0) = 0."""
    n = b.shape[0]
    matvecs = 0
    if x_m1 is None or not np.any(x_m1):
        x_m1 = np.zeros(n)
        r_m1 = b.copy()
    else:
        x_m1 = np.asarray(x_m1, dtype=np.float64)
        r_m1 = b - A @ x_m1
        matvecs = 1
    x0 = x_m1 + rec.U @ (rec.Chat.T @ r_m1)
    r0 = r_m1 - rec.C @ (rec.Chat.T @ r_m1)
    for attempt in range(4):
        rt_m1 = shadow_vector(n, shadow_seed + attempt)
        rt0 = rt_m1 - rec.Ct @ (rec.Ccheck.T @ rt_m1)
        rho0 = np.dot(rt0, r0)
        if rho0 != 0.0:
            break
    return x0, r0, rt0, rho0, attempt + 1, matvecs


def rbicgstab(A, b, rec: RecycleSpace | None = None, x_m1=None, tol=1e-8, max_itn=None,
              shadow_seed=DEFAULT_SEED, record=False, cycle_s=None, on_cycle=None,
              true_residual=True):
    """Alg. 2: BiCGSTAB on B = (I - C C-hat^T) A from the start of eq. (3.5),
    then x = x_i - U x_c.  Returns (x, SolveInfo).

    ``cycle_s`` / ``on_cycle``: every ``cycle_s`` iterations (and once more for
    a final partial cycle) ``on_cycle(store)`` is called with the CycleStore
    of that cycle (p_i, s_i and their raw products A p_i, A s_i); the
    recycle-space update (``oracle.recycle``) hooks in here.
    """
    n = b.shape[0]
    if rec is None:
        rec = empty_space(n)
    if max_itn is None:
        max_itn = min(n, 20000)
    info = SolveInfo()
    b = np.asarray(b, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    thresh = tol * bnorm

    x, r, rt0, rho_prev, info.seeds_used, info.matvecs = initial_projection(A, b, rec, x_m1, shadow_seed)
    info.rt0, info.r0 = rt0, r.copy()
    xc = np.zeros(rec.k)

    def finish(x_i):
        """End of Alg. 2: the solution of A x = b from the projected iterate."""
        x_out = x_i - rec.U @ xc
        info.relres_rec = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
        if true_residual:
            info.relres_true = np.linalg.norm(b - A @ x_out) / bnorm if bnorm > 0 else 0.0
        return x_out

    if np.linalg.norm(r) <= thresh:
        info.relres_rec = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
        info.relres_true = info.relres_rec
        return x - rec.U @ xc, info
    if rho_prev == 0.0:
        info.status = BREAKDOWN_RHO
        info.relres_rec = np.linalg.norm(r) / bnorm
        return x - rec.U @ xc, info

    store = CycleStore()

    def flush():
        nonlocal store
        if on_cycle is not None and len(store) > 0:
            on_cycle(store)
        store = CycleStore()

    # BiCGSTAB recurrences on B; p_1 = r_0 (beta = 0 before the first step)
    beta = omega = 0.0
    p = np.zeros(n)
    q = np.zeros(n)
    converged = False
    for i in range(1, max_itn + 1):
        p = r + beta * p - beta * omega * q
        Ap, zeta, q = project_product(A, rec, p)           # q_i = B p_i
        info.matvecs += 1
        if cycle_s:
            store.P.append(p.copy())
            store.AP.append(Ap.copy())
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
        As, gamma, t = project_product(A, rec, s)         # t_i = B s_i
        info.matvecs += 1
        if cycle_s:
            store.S.append(s.copy())
            store.AS.append(As.copy())
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
        # x moves by alpha p + omega s; its U-component by alpha zeta + omega gamma
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
    return finish(x), info
