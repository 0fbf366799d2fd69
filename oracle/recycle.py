"""Recycle-space update between systems, and the sequence driver (FP64).

Sec. 6.2 builds the recycle space from vectors stored over cycles of s
iterations ("at the end of each cycle ... build or improve the recycle
space"), with s = 25, k = 20, but defers the selection rule to the RBiCG
paper.  For sequences solved with RBiCGSTAB alone ("mode S") this oracle
takes the harmonic-Ritz reading (the GCRO-DR choice the paper compares
against), recycling the eigenvalues of smallest magnitude as in Sec. 5:

* W = [Y, p_1..p_j, s_1..s_j] (Y = the current candidate, initially the
  solve's own U; empty for the first system) and Z = A W =
  [A Y, A p_1.., A s_1..] with the products taken before projection.
* Harmonic Ritz pairs on range(W): Z^T Z y = theta Z^T W y.
  Columns are first scaled to unit ||Z e_j|| (a change of basis); the pencil
  is restricted to the eigenvectors of the scaled Z^T Z with eigenvalue
  > 1e-10 * the largest (numerical rank of W); on that subspace with
  y = V L^{-1/2} z the problem becomes M z = (1/theta) z,
  M = L^{-1/2} V^T H V L^{-1/2}, H = scaled Z^T W.
* The k values of smallest |theta| are kept (ties: Re theta ascending, then
  Im theta >= 0 first).  A complex pair contributes [Re y, Im y]; a pair
  that would be split at position k is dropped.
* Y <- W y, A Y <- Z y, each column scaled to unit 2-norm.
* After the solve U_next = Y and U~_next = U_next (right-only, Sec. 5).

This is the oracle's own algorithm (symmetric eigendecomposition, then
LAPACK's nonsymmetric eigensolver); the CUDA library's host code uses a
different factorisation of the same pencil.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rbicgstab import CycleStore, empty_space, rbicgstab, recycle_setup

RANK_TOL = 1e-10


def harmonic_ritz_coeffs(G: np.ndarray, H: np.ndarray, k: int, rank_tol=RANK_TOL):
    """Coefficients y (m x k_used) of the k harmonic Ritz vectors of smallest |theta|.

    G = Z^T Z, H = Z^T W.  Returns (y, theta_selected)."""
    m = G.shape[0]
    dg = np.diag(G).copy()
    live = dg > 0
    d = np.zeros(m)
    d[live] = 1.0 / np.sqrt(dg[live])
    Gs = d[:, None] * G * d[None, :]
    Hs = d[:, None] * H * d[None, :]
    lam, V = np.linalg.eigh(Gs)
    keep = lam > rank_tol * lam.max()
    V = V[:, keep]
    lam = lam[keep]
    T = V / np.sqrt(lam)[None, :]
    M = T.T @ Hs @ T
    mu, Zv = np.linalg.eig(M)
    with np.errstate(divide="ignore"):
        theta = np.where(mu != 0, 1.0 / np.where(mu != 0, mu, 1.0), np.inf)
    # units: real eigenvalues, or complex pairs represented by the Im > 0 member
    units = []
    for j in range(len(mu)):
        if mu[j].imag == 0.0:
            units.append((abs(theta[j]), theta[j].real, 0, j))
        elif mu[j].imag < 0.0:      # theta = 1/mu has Im > 0
            units.append((abs(theta[j]), theta[j].real, 1, j))
    units.sort(key=lambda u: (u[0], u[1]))
    cols, sel = [], []
    for a, re, cplx, j in units:
        if not np.isfinite(a):
            continue
        need = 2 if cplx else 1
        if len(cols) + need > k:
            break
        y = d * (T @ Zv[:, j])
        if cplx:
            cols += [y.real, y.imag]
            sel += [theta[j], np.conj(theta[j])]
        else:
            cols.append(y.real)
            sel.append(theta[j])
        if len(cols) == k:
            break
    if not cols:
        return np.zeros((m, 0)), np.zeros(0)
    return np.column_stack(cols), np.array(sel)


@dataclass
class Candidate:
    """The evolving candidate recycle space Y and its product A Y."""

    Y: np.ndarray
    AY: np.ndarray
    k: int
    cycles: int = 0
    max_cycles: int = 0          # 0 = every cycle updates
    thetas: list = field(default_factory=list)

    def update(self, store: CycleStore):
        if self.max_cycles and self.cycles >= self.max_cycles:
            return
        W = np.column_stack([self.Y] + store.W()) if self.Y.shape[1] else np.column_stack(store.W())
        Z = np.column_stack([self.AY] + store.AW()) if self.AY.shape[1] else np.column_stack(store.AW())
        G = Z.T @ Z
        H = Z.T @ W
        y, th = harmonic_ritz_coeffs(G, H, self.k)
        Y = W @ y
        AY = Z @ y
        nrm = np.linalg.norm(Y, axis=0)
        self.Y = Y / nrm[None, :]
        self.AY = AY / nrm[None, :]
        self.cycles += 1
        self.thetas.append(th)


@dataclass
class SequenceResult:
    x: list = field(default_factory=list)
    info: list = field(default_factory=list)
    iters: list = field(default_factory=list)
    matvecs_iter: int = 0
    matvecs_setup: int = 0
    U_final: np.ndarray | None = None
    k_used: list = field(default_factory=list)


def solve_sequence(matrices, rhs, k, cycle_s=25, tol=1e-8, policy="first", recycle=True,
                   max_cycles=0, shadow_seed=None, max_itn=None, U0=None):
    """Mode-S sequence: for each matrix A^(i) and each of its right-hand sides,
    run Alg. 2 with the current recycle space; update it with harmonic Ritz
    vectors during the solves selected by ``policy`` ("first": the first RHS
    of every matrix, "all", "none").  ``recycle=False`` runs plain BiCGSTAB
    (Alg. 2 with k = 0) on every system.  Setup (C, C~, D_c) is recomputed
    only when the matrix or U changes (the note under Alg. 2).

    ``policy="first_block"`` is the order of a blocked solve, in which all
    right-hand sides of one matrix iterate together: every RHS of A^(i) uses
    the space in force when A^(i) arrives, and the update built during the
    first RHS's solve takes effect from A^(i+1) on."""
    from .shadow import DEFAULT_SEED
    seed = DEFAULT_SEED if shadow_seed is None else shadow_seed
    res = SequenceResult()
    U = U0
    for A, bs in zip(matrices, rhs):
        rec = None
        pending = None
        for ib, b in enumerate(bs):
            b = b() if callable(b) else b
            if recycle and (rec is None or rec_U_changed):
                rec = recycle_setup(A, U)
                res.matvecs_setup += rec.setup_matvecs
            elif not recycle:
                rec = empty_space(A.shape[0])
            rec_U_changed = False
            upd = recycle and (policy == "all" or (policy in ("first", "first_block") and ib == 0))
            cand = None
            if upd:
                cand = Candidate(Y=rec.U.copy(), AY=rec.C.copy(), k=k, max_cycles=max_cycles)
            x, info = rbicgstab(A, b, rec, tol=tol, shadow_seed=seed, max_itn=max_itn,
                                cycle_s=cycle_s if upd else None,
                                on_cycle=cand.update if upd else None)
            res.x.append(x)
            res.info.append(info)
            res.iters.append(info.iters)
            res.matvecs_iter += info.matvecs
            res.k_used.append(rec.k)
            if upd and cand.Y.shape[1] > 0:
                if policy == "first_block":
                    pending = cand.Y
                else:
                    U = cand.Y
                    rec_U_changed = True
        if pending is not None:
            U = pending
    res.U_final = U
    return res
