"""Seeded synthetic inputs: stencil operators in CSR form and right-hand sides.

This module builds the linear systems A^(iota) x = b^(iota, kappa) (Sec. 1,
eq. (1.1)) that the solver and the CPU oracle are run on.  It holds none of the
solver's arithmetic: only discretisations of convection-diffusion operators,
diagonal mass matrices and Gaussian right-hand sides, all from
``numpy.random.default_rng(seed)``.  The paper's own workloads (the silicon
nitride membrane model of Sec. 6.2 and the coefficient field of Example 2 in
Sec. 5) are not available; these stencil families stand in for them, shaped
like the moment-matching PMOR sequences of Sec. 6.1 (matrix blocks times
right-hand-side blocks, A^(i) = A0 + sigma_i A1).

All operators are scaled by h^2 (the stencil weights are O(1)); a uniform
scaling of a whole system does not change Krylov iterates.  Convection uses
first-order upwind differences with positive velocities, so the upwind
neighbour is the one with the smaller grid index.  Ordering is lexicographic
with x fastest.  Column indices within a row are sorted ascending.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR",
    "conv_diff_2d",
    "conv_diff_3d",
    "stencil27_noisy",
    "mass_diagonal",
    "shifted_values",
    "gaussian_rhs",
    "random_recycle_basis",
    "config_small_2d",
    "config_shifted_3d",
    "ParamSpec",
    "config_param_3d",
    "example1",
    "config_batch_2d",
    "config_large_27pt",
]


@dataclass
class CSR:
    """Compressed sparse row matrix with int32 indices and float64 values."""

    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray      # int32[nnz]
    val: np.ndarray      # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def diag_index(self) -> np.ndarray:
        """Position of the diagonal entry of each row inside ``col``/``val``."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        pos = np.nonzero(self.col == rows)[0]
        if pos.shape[0] != self.n:
            raise ValueError("matrix lacks a full diagonal")
        return pos


def _assemble(n: int, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Build CSR from per-row candidate lists ``cols``/``vals`` of shape (n, w).

    Entries with a negative column are absent.  Candidates must already be in
    ascending column order along axis 1.
    """
    mask = cols >= 0
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return CSR(n=n, row_ptr=row_ptr.astype(np.int32), col=cols[mask].astype(np.int32),
               val=vals[mask].astype(np.float64))


def conv_diff_2d(N: int, p: float, q: float | None = None) -> CSR:
    """5-point -Lap(u) + p u_x + q u_y on an N x N interior grid, h = 1/(N+1).

    h^2-scaled; first-order upwind convection for p, q >= 0 (backward
    differences).  Homogeneous Dirichlet boundary.  Row weights: centre
    4 + (p+q)h, west -1 - ph, south -1 - qh, east -1, north -1.
    """
    if q is None:
        q = p
    h = 1.0 / (N + 1)
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    i = idx % N
    j = idx // N
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5))
    # ascending column order: south, west, centre, east, north
    m = j > 0
    cols[m, 0] = idx[m] - N
    vals[m, 0] = -1.0 - q * h
    m = i > 0
    cols[m, 1] = idx[m] - 1
    vals[m, 1] = -1.0 - p * h
    cols[:, 2] = idx
    vals[:, 2] = 4.0 + (p + q) * h
    m = i < N - 1
    cols[m, 3] = idx[m] + 1
    vals[m, 3] = -1.0
    m = j < N - 1
    cols[m, 4] = idx[m] + N
    vals[m, 4] = -1.0
    return _assemble(n, cols, vals)


def conv_diff_3d(N: int, c, kappa=None) -> CSR:
    """7-point -div(kappa grad u) + c (1,1,1).grad u on an N^3 grid, h = 1/(N+1).

    ``c`` is a scalar or a per-cell array (length N^3) of convection
    magnitudes; ``kappa`` is None (unit diffusion) or a per-cell array of
    diffusion coefficients, with face coefficients the arithmetic mean of the
    two cells (a boundary face takes the cell's own value).  h^2-scaled, upwind
    convection (backward differences), homogeneous Dirichlet boundary.
    """
    h = 1.0 / (N + 1)
    n = N * N * N
    idx = np.arange(n, dtype=np.int64)
    i = idx % N
    j = (idx // N) % N
    l = idx // (N * N)
    cc = np.broadcast_to(np.asarray(c, dtype=np.float64), (n,))
    kc = np.ones(n) if kappa is None else np.asarray(kappa, dtype=np.float64)
    cols = np.full((n, 7), -1, dtype=np.int64)
    vals = np.zeros((n, 7))
    centre = 3.0 * cc * h
    # neighbours in ascending order: -N^2, -N, -1, 0, +1, +N, +N^2
    specs = [(0, -N * N, l > 0, True), (1, -N, j > 0, True), (2, -1, i > 0, True),
             (4, 1, i < N - 1, False), (5, N, j < N - 1, False), (6, N * N, l < N - 1, False)]
    for slot, off, m, upwind in specs:
        nb = np.clip(idx + off, 0, n - 1)
        kf = np.where(m, 0.5 * (kc + kc[nb]), kc)
        centre = centre + kf
        cols[m, slot] = idx[m] + off
        vals[m, slot] = -kf[m] - (cc[m] * h if upwind else 0.0)
    cols[:, 3] = idx
    vals[:, 3] = centre
    return _assemble(n, cols, vals)


def stencil27_noisy(Nx: int, Ny: int, Nz: int, c: float, seed: int = 5,
                    noise: float = 0.1) -> CSR:
    """27-point convection-diffusion operator with noisy coefficients.

    Couplings: -1 to each of the 26 neighbours (diffusion), and -c h more to
    the three upwind face neighbours (first-order upwind convection c(1,1,1)
    with c > 0); every coupling is multiplied by (1 + noise U[-1, 1]), one
    draw per (row, neighbour), so the operator is non-symmetric.  The
    diagonal is the sum of the magnitudes of all 26 couplings of its row,
    those to neighbours outside the grid included (a conservative
    discretisation with homogeneous Dirichlet boundaries): interior row sums
    vanish, boundary rows are strictly dominant, so A is an irreducibly
    diagonally dominant M-matrix for any noise below 1.  Multiplying the
    diagonal by noise of its own as well would leave random row sums of
    order noise * 26 against a smallest eigenvalue of order h^2, which makes
    large grids indefinite.

    h = 1/(max(Nx,Ny,Nz)+1); h^2-scaled.  The noise draw is fixed by ``seed``
    and independent of ``c``, and every entry is linear in ``c``, so a
    drifting ``c`` changes only the centre and the upwind face entries.
    """
    h = 1.0 / (max(Nx, Ny, Nz) + 1)
    n = Nx * Ny * Nz
    idx = np.arange(n, dtype=np.int64)
    i = idx % Nx
    j = (idx // Nx) % Ny
    l = idx // (Nx * Ny)
    rng = np.random.default_rng(seed)
    eta = 1.0 + noise * rng.uniform(-1.0, 1.0, size=(n, 27))
    cols = np.full((n, 27), -1, dtype=np.int64)
    vals = np.zeros((n, 27))
    diag = np.zeros(n)
    centre = -1
    slot = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                off = dx + dy * Nx + dz * Nx * Ny
                if off == 0:
                    centre = slot
                    slot += 1
                    continue
                face = abs(dx) + abs(dy) + abs(dz) == 1
                w = (-1.0 - (c * h if (face and off < 0) else 0.0)) * eta[:, slot]
                diag -= w
                m = ((i + dx >= 0) & (i + dx < Nx) & (j + dy >= 0) & (j + dy < Ny)
                     & (l + dz >= 0) & (l + dz < Nz))
                cols[m, slot] = idx[m] + off
                vals[m, slot] = w[m]
                slot += 1
    cols[:, centre] = idx
    vals[:, centre] = diag
    return _assemble(n, cols, vals)


def mass_diagonal(n: int, seed: int = 1, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    """Diagonal mass matrix entries E_ii ~ U[lo, hi]."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def shifted_values(L: CSR, E: np.ndarray, shift: float) -> np.ndarray:
    """Values of ``shift * diag(E) + L`` on the pattern of L (L has a full diagonal)."""
    v = L.val.copy()
    v[L.diag_index()] += shift * E
    return v


def gaussian_rhs(n: int, seed: int) -> np.ndarray:
    """b ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal(n)


def random_recycle_basis(n: int, k: int, seed: int) -> np.ndarray:
    """Column-major-agnostic n x k Gaussian block (a generic recycle space)."""
    return np.random.default_rng(seed).standard_normal((n, k))


@dataclass
class SequenceSpec:
    """A sequence of systems: matrices share one pattern; ``rhs[i]`` lists the
    right-hand sides solved with matrix i.  ``pattern``, the entries of
    ``values`` and of ``rhs`` may be callables that build them on demand
    (the large workloads)."""

    pattern: CSR
    values: list        # list of float64[nnz] per matrix (lazy callables allowed)
    rhs: list           # list of list of float64[n]
    k: int
    cycle_s: int
    tol: float
    label: str


def config_small_2d(N: int = 64) -> SequenceSpec:
    """2D convection-diffusion, 5-point upwind on an N x N grid (n = N^2),
    A(p) = -Lap + p (1,1).grad, p = 10, 11, ..., 17; one RHS b ~ N(0,1) from
    seed 0 shared by all 8 systems; k = 8, s = 25, tol 1e-8."""
    mats = [conv_diff_2d(N, float(p)) for p in range(10, 18)]
    b = gaussian_rhs(N * N, 0)
    return SequenceSpec(pattern=mats[0], values=[m.val for m in mats],
                        rhs=[[b] for _ in mats], k=8, cycle_s=25, tol=1e-8,
                        label=f"2d-conv-diff-{N}x{N}-p10..17")


def config_shifted_3d(N: int = 128, c: float = 10.0, n_shifts: int = 20, n_rhs: int = 4,
                      k: int = 20, lazy_rhs: bool = True) -> SequenceSpec:
    """3D 7-point upwind convection-diffusion on an N^3 grid with a diagonal
    mass matrix E ~ U[0.5, 1.5] (seed 1): systems (sigma_j E - A_state) with
    A_state = -(-Lap + c(1,1,1).grad), sigma_j = logspace(-2, 2, n_shifts);
    the whole system is h^2-scaled, so matrix j is L_h + h^2 sigma_j E.
    RHS kappa of shift j is N(0,1) from seed 100 + 4 j + kappa."""
    L = conv_diff_3d(N, c)
    h = 1.0 / (N + 1)
    E = mass_diagonal(L.n, seed=1)
    sig = np.logspace(-2, 2, n_shifts)
    diag_pos = L.diag_index()

    def make_vals(s):
        def f():
            v = L.val.copy()
            v[diag_pos] += (h * h * s) * E
            return v
        return f

    values = [make_vals(s) for s in sig]
    if lazy_rhs:
        rhs = [[(lambda seed=100 + 4 * j + kk: gaussian_rhs(L.n, seed)) for kk in range(n_rhs)]
               for j in range(n_shifts)]
    else:
        rhs = [[gaussian_rhs(L.n, 100 + 4 * j + kk) for kk in range(n_rhs)] for j in range(n_shifts)]
    return SequenceSpec(pattern=L, values=values, rhs=rhs, k=k, cycle_s=25, tol=1e-8,
                        label=f"3d-7pt-{N}^3-shifted-{n_shifts}x{n_rhs}")


@dataclass
class ParamSpec:
    """A parametrised operator A(p) = sum_k p_k A_k on one pattern (every A_k
    stored as values on ``pattern``), an output matrix and a right-hand side,
    and the parameter steps of a sequence."""

    pattern: CSR
    basis: list          # float64[nnz] per parameter: the values of dA/dp_k
    names: list          # parameter names
    p0: np.ndarray       # float64[n_params]
    C_out: np.ndarray    # float64[m, n]
    b: np.ndarray        # float64[n]
    steps: list          # parameter vectors of the sequence (steps[0] = p0)
    k: int
    tol: float
    label: str

    def values(self, p) -> np.ndarray:
        """Values of A(p) on the pattern."""
        v = np.zeros_like(self.basis[0])
        for pk, Ak in zip(p, self.basis):
            v += pk * Ak
        return v


def config_param_3d(N: int = 100, kappa: float = 1.0, c: float = 10.0, n_steps: int = 6,
                    step: float = 1.01, m_out: int = 16, k: int = 20) -> ParamSpec:
    """3D 7-point convection-diffusion on an N^3 grid with 8 parameters:
    diffusion kappa_r and convection c_r on 4 regions r = 2[x >= 1/2] +
    [y >= 1/2] (cell centres x = (i+1) h, y = (j+1) h; each region is a pair
    of octants stacked in z).  Face diffusion is the mean of the two cells'
    kappa, convection is upwind c_r (1,1,1).grad (the operator of
    ``conv_diff_3d`` with per-cell coefficients).  A(p) is linear in p, so
    dA/dp_k is the operator with coefficient 1 on region r and 0 elsewhere.
    Steps p_{j+1} = step * p_j; C_out ~ N(0,1) (m_out x n, seed 3); b ~ N(0,1)
    (seed 4)."""
    h = 1.0 / (N + 1)
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    x = (idx % N + 1) * h
    y = ((idx // N) % N + 1) * h
    region = 2 * (x >= 0.5).astype(np.int64) + (y >= 0.5).astype(np.int64)
    basis, names = [], []
    zero = np.zeros(n)
    pattern = None
    for r in range(4):
        A = conv_diff_3d(N, zero, kappa=(region == r).astype(np.float64))
        basis.append(A.val)
        names.append(f"kappa_{r}")
        pattern = A if pattern is None else pattern
    for r in range(4):
        A = conv_diff_3d(N, (region == r).astype(np.float64), kappa=zero)
        basis.append(A.val)
        names.append(f"c_{r}")
    p0 = np.array([kappa] * 4 + [c] * 4, dtype=np.float64)
    steps = [p0 * step ** j for j in range(n_steps)]
    C_out = np.random.default_rng(3).standard_normal((m_out, n))
    b = gaussian_rhs(n, 4)
    pat = CSR(n=n, row_ptr=pattern.row_ptr, col=pattern.col, val=np.zeros_like(pattern.val))
    return ParamSpec(pattern=pat, basis=basis, names=names, p0=p0, C_out=C_out, b=b, steps=steps,
                     k=k, tol=1e-8, label=f"3d-7pt-{N}^3-8-params")


def example1(N: int = 40, a: float = 10.0):
    """Example 1 of Sec. 5: -(u_x)_x - (u_y)_y + a u_x - a u_y = 0 on the unit
    square, an (N+2) x (N+2) vertex grid (N^2 = 1600 unknowns at N = 40),
    u = 1 on the south and west boundaries and 0 on the north and east ones.
    The discretisation is unstated; central differences reproduce the
    paper's Table 1 (first-order upwind does not).  h^2-scaled row weights:
    centre 4, west -1 - a h/2, east -1 + a h/2, south -1 + a h/2, north
    -1 - a h/2; the boundary values move to b.  The paper starts from a
    vector of all ones and stops at relative tolerance 1e-10.
    Returns (A as CSR, b, x_{-1})."""
    h = 1.0 / (N + 1)
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    i = idx % N
    j = idx // N
    w_west, w_east = -1.0 - 0.5 * a * h, -1.0 + 0.5 * a * h
    w_south, w_north = -1.0 + 0.5 * a * h, -1.0 - 0.5 * a * h
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5))
    for slot, off, m, w in [(0, -N, j > 0, w_south), (1, -1, i > 0, w_west),
                            (3, 1, i < N - 1, w_east), (4, N, j < N - 1, w_north)]:
        cols[m, slot] = idx[m] + off
        vals[m, slot] = w
    cols[:, 2] = idx
    vals[:, 2] = 4.0
    b = np.zeros(n)
    b[i == 0] -= w_west * 1.0     # u = 1 on the west boundary
    b[j == 0] -= w_south * 1.0    # u = 1 on the south boundary
    return _assemble(n, cols, vals), b, np.ones(n)


def config_batch_2d(n_systems: int = 256, side_lo: int = 100, side_hi: int = 450,
                    shifts=(0.0, 1e-2, 1e-1, 1.0), k: int = 10, seed: int = 2) -> list:
    """A sweep of independent parameter samples of uneven sizes: system i is
    the 2D operator of ``conv_diff_2d`` on an N_i x N_i grid with
    N_i ~ U{side_lo..side_hi} and p_i ~ U[1, 50] (seed ``seed``), carrying a
    sequence of len(shifts) matrices A_i + sigma I (sigma added to the
    h^2-scaled diagonal, E = I) with one right-hand side N(0,1) (seed
    1000 + i) solved for each.  Returned as one SequenceSpec per system with
    lazy values; k = 10, s = 25, tol 1e-8."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=n_systems)
    ps = rng.uniform(1.0, 50.0, size=n_systems)
    out = []
    for i, (N, p) in enumerate(zip(sides, ps)):
        N = int(N)

        def pattern(N=N, p=float(p)):
            return conv_diff_2d(N, p)

        def make_vals(sig, N=N, p=float(p)):
            def f():
                A = conv_diff_2d(N, p)
                return shifted_values(A, np.ones(A.n), sig)
            return f

        b = (lambda n=N * N, sd=1000 + i: gaussian_rhs(n, sd))
        out.append(SequenceSpec(pattern=pattern, values=[make_vals(sg) for sg in shifts],
                                rhs=[[b] for _ in shifts], k=k, cycle_s=25, tol=1e-8,
                                label=f"2d-{N}x{N}-p{p:.2f}"))
    return out


def config_large_27pt(Nx: int = 256, Ny: int = 256, Nz: int = 128, c0: float = 10.0,
                      drift: float = 1.02, n_systems: int = 10, k: int = 30, seed: int = 5) -> SequenceSpec:
    """The large 27-point sequence: ``stencil27_noisy`` on Nx x Ny x Nz with
    convection c_j = c0 drift^j (j = 0..n_systems-1) and one fixed noise draw
    (seed ``seed``), so only the convection entries change along the
    sequence; one RHS N(0,1) (seed 200 + j) per system; k = 30, s = 25, tol
    1e-8.  Values are generated on demand (224M nonzeros at full size)."""
    cs = [c0 * drift ** j for j in range(n_systems)]

    def make_vals(c):
        return lambda: stencil27_noisy(Nx, Ny, Nz, c, seed=seed).val

    n = Nx * Ny * Nz
    rhs = [[(lambda sd=200 + j: gaussian_rhs(n, sd))] for j in range(n_systems)]
    return SequenceSpec(pattern=lambda: stencil27_noisy(Nx, Ny, Nz, c0, seed=seed),
                        values=[make_vals(c) for c in cs], rhs=rhs, k=k, cycle_s=25, tol=1e-8,
                        label=f"3d-27pt-{Nx}x{Ny}x{Nz}-noisy-drift")
