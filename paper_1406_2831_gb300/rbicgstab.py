"""Python binding of librbicgstab (ctypes).  Argument marshalling only: every
step of the solve runs in the library's CUDA kernels and host code.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA; CUDA
tensors are passed by ``data_ptr()`` with ``where = RB_DEVICE``).  Torch is
used only for device memory and streams.  If the library is missing this
module raises at import of the first handle: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbicgstab.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rbicgstab.h")


def _header_constants() -> dict:
    out = {}
    with open(HEADER) as f:
        for line in f:
            m = re.match(r"#define\s+(RB_\w+)\s+(-?\d+)", line)
            if m:
                out[m.group(1)] = int(m.group(2))
    return out


C = _header_constants()
RB_OK = C["RB_OK"]
RB_HOST, RB_DEVICE = C["RB_HOST"], C["RB_DEVICE"]
PRECISION = {"fp64": C["RB_FP64"], "mixed": C["RB_MIXED"]}
RECYCLE = {"none": C["RB_RECYCLE_NONE"], "fixed": C["RB_RECYCLE_FIXED"],
           "update_first": C["RB_RECYCLE_UPDATE_FIRST"], "update_all": C["RB_RECYCLE_UPDATE_ALL"]}
HARD_ERRORS = {C[k] for k in ("RB_EINVAL", "RB_EDIM", "RB_EBADCSR", "RB_ENONFINITE", "RB_ENOMEM",
                              "RB_ECUDA", "RB_ETIMEOUT")}


class Opts(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("cycle_s", ctypes.c_int32), ("max_itn", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("recycle_mode", ctypes.c_int32),
                ("update_cycles", ctypes.c_int32), ("poll", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("tol", ctypes.c_double), ("shadow_seed", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("k_used", ctypes.c_int32),
                ("seeds_used", ctypes.c_int32), ("matvecs", ctypes.c_int64),
                ("matvecs_setup", ctypes.c_int64), ("matvecs_check", ctypes.c_int64),
                ("cycles", ctypes.c_int32), ("outer", ctypes.c_int32), ("relres_rec", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("bytes_model", ctypes.c_double), ("ms_update", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class RbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} ({code})")


_lib = None


def lib():
    """Load librbicgstab.so (built in-tree by ``paper_1406_2831_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librbicgstab.so not built ({LIB_PATH}); run paper_1406_2831_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    L.rbicgstab_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Opts)]
    L.rbicgstab_destroy.argtypes = [vp]
    L.rbicgstab_set_matrix.argtypes = [vp, i64, i64, dp, dp, dp, ctypes.c_int]
    L.rbicgstab_set_values.argtypes = [vp, dp, ctypes.c_int]
    L.rbicgstab_set_recycle.argtypes = [vp, i32, dp, dp, i64, ctypes.c_int]
    L.rbicgstab_get_recycle.argtypes = [vp, ctypes.POINTER(i32), dp, dp, i64, ctypes.c_int]
    L.rbicgstab_solve.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.POINTER(Stats)]
    L.rbicgstab_apply.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.c_int]
    L.rbicgstab_pattern_outer.argtypes = [vp, dp, dp, ctypes.c_double, dp, ctypes.c_int]
    L.rbicgstab_harmonic_ritz.argtypes = [i32, dp, dp, i32, dp, dp, dp, ctypes.POINTER(i32)]
    L.rbicgstab_svd_small.argtypes = [i32, dp, dp, dp, dp]
    L.rbicgstab_solve_block.argtypes = [vp, i32, dp, dp, i64, ctypes.c_int, ctypes.POINTER(Stats)]
    L.rbicgstab_time_passes.argtypes = [vp, i32, dp, i64, ctypes.c_int, i32, dp]
    L.rbicg_solve.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int, ctypes.POINTER(Stats), ctypes.POINTER(Stats)]
    L.rbicgstab_residual_noalloc.argtypes = [i64, dp, dp, dp, dp, dp, dp, dp, vp]
    L.rbicgstab_residual_noalloc.restype = ctypes.c_int
    L.rbicgstab_update_gram.argtypes = [i64, i64, i32, i32, i32, i32, i32, dp, dp, dp, dp, dp, dp, dp, dp, i32, vp,
                                        ctypes.POINTER(ctypes.c_double)]
    L.rbicgstab_update_gram.restype = ctypes.c_int
    L.rbicgstab_sell_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.rbicgstab_solve_l.argtypes = [vp, i32, dp, dp, ctypes.c_int, ctypes.POINTER(Stats)]
    L.rbicgstab_solve_adjoint.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.POINTER(Stats)]
    L.rbicgstab_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Opts)]
    L.rbicgstab_batch_destroy.argtypes = [vp]
    L.rbicgstab_batch_set_matrices.argtypes = [vp, i32, dp, dp, dp, dp]
    L.rbicgstab_batch_set_values.argtypes = [vp, dp, ctypes.c_int]
    L.rbicgstab_batch_set_recycle.argtypes = [vp, i32, dp, ctypes.c_int]
    L.rbicgstab_batch_solve.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.POINTER(Stats)]
    L.rbicgstab_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                       ctypes.POINTER(ctypes.c_double)]
    for name in ("rbicgstab_batch_create", "rbicgstab_batch_destroy", "rbicgstab_batch_set_matrices",
                 "rbicgstab_batch_set_values", "rbicgstab_batch_set_recycle", "rbicgstab_batch_solve",
                 "rbicgstab_batch_info"):
        getattr(L, name).restype = ctypes.c_int
    L.rbicgstab_solve_adjoint.restype = ctypes.c_int
    L.rbicgstab_solve_l.restype = ctypes.c_int
    L.rbicgstab_sell_stats.restype = ctypes.c_int
    L.rbicgstab_wait_selftest.argtypes = [i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.rbicgstab_wait_selftest.restype = ctypes.c_int
    L.rbicgstab_kernel_launches.argtypes = []
    L.rbicgstab_kernel_launches.restype = ctypes.c_longlong
    L.rbicgstab_error_string.argtypes = [ctypes.c_int]
    L.rbicgstab_error_string.restype = ctypes.c_char_p
    for name in ("rbicgstab_create", "rbicgstab_destroy", "rbicgstab_set_matrix", "rbicgstab_set_values",
                 "rbicgstab_set_recycle", "rbicgstab_get_recycle", "rbicgstab_solve", "rbicgstab_apply",
                 "rbicgstab_harmonic_ritz", "rbicgstab_time_passes", "rbicgstab_solve_block",
                 "rbicg_solve", "rbicgstab_pattern_outer", "rbicgstab_svd_small"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def error_string(code: int) -> str:
    return lib().rbicgstab_error_string(int(code)).decode()


def _check(code: int, where: str) -> int:
    if code in HARD_ERRORS:
        raise RbError(code, where)
    return code


# ---------------------------------------------------------------- array marshalling
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, where, keepalive) for a 1-D/2-D numpy array or torch tensor."""
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        if a.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (RB_DEVICE if a.is_cuda else RB_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, RB_HOST, arr


def _colmajor(U, dtype=np.float64):
    """(pointer, where, ld, keepalive) for an (n, k) block as column-major storage."""
    if _is_torch(U):
        Ut = U.t().contiguous()          # (k, n) row-major == (n, k) column-major
        return Ut.data_ptr(), (RB_DEVICE if U.is_cuda else RB_HOST), U.shape[0], Ut
    arr = np.asfortranarray(U, dtype=dtype)
    return arr.ctypes.data, RB_HOST, arr.shape[0], arr


@dataclass
class SolveResult:
    x: object
    stats: dict


class Solver:
    """One solver handle (``rbicgstab_create``).  Options mirror ``rb_opts``."""

    def __init__(self, k_max=0, cycle_s=25, max_itn=0, precision="fp64", recycle="none",
                 update_cycles=0, poll=0, tol=1e-8, shadow_seed=0x5EED, stream=None):
        L = lib()
        o = Opts()
        o.k_max, o.cycle_s, o.max_itn = k_max, cycle_s, max_itn
        o.precision, o.recycle_mode = PRECISION[precision], RECYCLE[recycle]
        o.update_cycles, o.poll, o.tol, o.shadow_seed = update_cycles, poll, tol, shadow_seed
        if stream is not None:
            o.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
        self._h = ctypes.c_void_p()
        _check(L.rbicgstab_create(ctypes.byref(self._h), ctypes.byref(o)), "rbicgstab_create")
        self.n = 0
        self.nnz = 0
        self.values_version = 0   # counts set_matrix / set_values calls
        self.opts = o

    def close(self):
        if self._h:
            lib().rbicgstab_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_matrix(self, row_ptr, col, val):
        rp, w1, k1 = _ptr(row_ptr, np.int32)
        cp, w2, k2 = _ptr(col, np.int32)
        vp, w3, k3 = _ptr(val, np.float64)
        if len({w1, w2, w3}) != 1:
            raise ValueError("row_ptr, col and val must live in the same memory space")
        n = len(row_ptr) - 1
        nnz = len(val)
        _check(lib().rbicgstab_set_matrix(self._h, n, nnz, rp, cp, vp, w1), "rbicgstab_set_matrix")
        self.n = n
        self.nnz = nnz
        self.values_version += 1

    def set_values(self, val):
        vp, w, keep = _ptr(val, np.float64)
        rc = _check(lib().rbicgstab_set_values(self._h, vp, w), "rbicgstab_set_values")
        self.values_version += 1
        return rc

    def set_recycle(self, U, Ut=None) -> int:
        """Set U (n x k) and U~ (None: U~ = U).  Returns the status (RB_OK or the rank warning)."""
        if U is None or U.shape[1] == 0:
            return _check(lib().rbicgstab_set_recycle(self._h, 0, None, None, max(self.n, 1), RB_HOST),
                          "rbicgstab_set_recycle")
        up, w, ld, k1 = _colmajor(U)
        utp = None
        if Ut is not None:
            utp, w2, ld2, k2 = _colmajor(Ut)
            if w2 != w or ld2 != ld:
                raise ValueError("U and Ut must match")
        return _check(lib().rbicgstab_set_recycle(self._h, U.shape[1], up, utp, ld, w), "rbicgstab_set_recycle")

    def get_recycle(self, device=None):
        """Current (biorthogonalised) U, U~ as (n, k) numpy arrays, or CUDA
        tensors when ``device`` is a torch device."""
        k = ctypes.c_int32()
        _check(lib().rbicgstab_get_recycle(self._h, ctypes.byref(k), None, None, max(self.n, 1), RB_HOST),
               "rbicgstab_get_recycle")
        kk = k.value
        if device is not None:
            import torch
            U = torch.empty((kk, self.n), dtype=torch.float64, device=device)
            Ut = torch.empty_like(U)
            _check(lib().rbicgstab_get_recycle(self._h, ctypes.byref(k), U.data_ptr(), Ut.data_ptr(),
                                               self.n, RB_DEVICE), "rbicgstab_get_recycle")
            return U.t(), Ut.t()
        U = np.zeros((self.n, kk), order="F")
        Ut = np.zeros((self.n, kk), order="F")
        if kk:
            _check(lib().rbicgstab_get_recycle(self._h, ctypes.byref(k), U.ctypes.data, Ut.ctypes.data,
                                               self.n, RB_HOST), "rbicgstab_get_recycle")
        return U, Ut

    def solve(self, b, x=None) -> SolveResult:
        """Solve A x = b; ``x`` (updated in place when given) is x_{-1}."""
        if x is None:
            if _is_torch(b):
                import torch
                x = torch.zeros_like(b)
            else:
                x = np.zeros(len(b))
        bp, wb, kb = _ptr(b, np.float64)
        if _is_torch(x):
            xp, wx, kx = _ptr(x, np.float64)
        else:
            if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
                x = np.ascontiguousarray(x, dtype=np.float64)
            xp, wx, kx = x.ctypes.data, RB_HOST, x
        if wb != wx:
            raise ValueError("b and x must live in the same memory space")
        st = Stats()
        _check(lib().rbicgstab_solve(self._h, bp, xp, wb, ctypes.byref(st)), "rbicgstab_solve")
        return SolveResult(x=x, stats=st.as_dict())

    def solve_block(self, B, X=None):
        """Blocked solve of the nrhs <= RB_MAX_RHS systems A x_i = b_i given
        as the rows of B (shape (nrhs, n); numpy array or CUDA tensor).  X
        (same shape, updated in place when given) holds the initial guesses.
        Returns SolveResult with x = X and stats = one dict per system."""
        if X is None:
            if _is_torch(B):
                import torch
                X = torch.zeros_like(B)
            else:
                X = np.zeros(np.shape(B))
        if len(np.shape(B)) != 2 or tuple(np.shape(B)) != tuple(np.shape(X)):
            raise ValueError("B and X must both have shape (nrhs, n)")
        nrhs, n = int(np.shape(B)[0]), int(np.shape(B)[1])
        bp, wb, kb = _ptr(B, np.float64)
        if _is_torch(X):
            xp, wx, kx = _ptr(X, np.float64)
        else:
            if not (isinstance(X, np.ndarray) and X.dtype == np.float64 and X.flags.c_contiguous):
                X = np.ascontiguousarray(X, dtype=np.float64)
            xp, wx, kx = X.ctypes.data, RB_HOST, X
        if wb != wx:
            raise ValueError("B and X must live in the same memory space")
        st = (Stats * max(nrhs, 1))()
        _check(lib().rbicgstab_solve_block(self._h, nrhs, bp, xp, n, wb, st), "rbicgstab_solve_block")
        return SolveResult(x=X, stats=[st[i].as_dict() for i in range(nrhs)])

    def solve_dual(self, b, bt=None, x=None, xt=None):
        """Alg. 1 (RBiCG): A x = b and A^T x~ = b~ together (rbicg_solve).
        bt None: the shadow vector is b~.  x, xt (updated in place when
        given) hold x_{-1}, x~_{-1}.  Returns (SolveResult for x,
        SolveResult for x~)."""
        def vec(v, like):
            if v is None:
                if _is_torch(like):
                    import torch
                    return torch.zeros_like(like)
                return np.zeros(len(like))
            if _is_torch(v):
                return v
            if not (isinstance(v, np.ndarray) and v.dtype == np.float64 and v.flags.c_contiguous):
                v = np.ascontiguousarray(v, dtype=np.float64)
            return v
        x, xt = vec(x, b), vec(xt, b)
        bp, wb, kb = _ptr(b, np.float64)
        if bt is not None:
            btp, wbt, kbt = _ptr(bt, np.float64)
            if wbt != wb:
                raise ValueError("b and bt must live in the same memory space")
        else:
            btp = None
        xp, wx, kx = _ptr(x, np.float64)
        xtp, wxt, kxt = _ptr(xt, np.float64)
        if not (wb == wx == wxt):
            raise ValueError("b, x and xt must live in the same memory space")
        st, sd = Stats(), Stats()
        _check(lib().rbicg_solve(self._h, bp, btp, xp, xtp, wb, ctypes.byref(st), ctypes.byref(sd)),
               "rbicg_solve")
        return SolveResult(x=x, stats=st.as_dict()), SolveResult(x=xt, stats=sd.as_dict())

    def solve_adjoint(self, g, lam=None) -> SolveResult:
        """The dual system A^T lam = g by Alg. 2 on A^T with the swapped
        recycle space (rbicgstab_solve_adjoint); ``lam`` (updated in place when
        given) is the initial guess."""
        if lam is None:
            if _is_torch(g):
                import torch
                lam = torch.zeros_like(g)
            else:
                lam = np.zeros(len(g))
        gp, wg, kg = _ptr(g, np.float64)
        if _is_torch(lam):
            lp, wl, kl = _ptr(lam, np.float64)
        else:
            if not (isinstance(lam, np.ndarray) and lam.dtype == np.float64 and lam.flags.c_contiguous):
                lam = np.ascontiguousarray(lam, dtype=np.float64)
            lp, wl, kl = lam.ctypes.data, RB_HOST, lam
        if wg != wl:
            raise ValueError("g and lam must live in the same memory space")
        st = Stats()
        _check(lib().rbicgstab_solve_adjoint(self._h, gp, lp, wg, ctypes.byref(st)), "rbicgstab_solve_adjoint")
        return SolveResult(x=lam, stats=st.as_dict())

    def solve_l(self, b, ell: int = 2, x=None) -> SolveResult:
        """Recycled BiCGstab(ell) with the handle's fixed space
        (rbicgstab_solve_l); ``x`` (updated in place when given) is x_{-1}.
        Breakdowns and non-convergence are reported in ``stats['status']``."""
        if x is None:
            if _is_torch(b):
                import torch
                x = torch.zeros_like(b)
            else:
                x = np.zeros(len(b))
        bp, wb, kb = _ptr(b, np.float64)
        if _is_torch(x):
            xp, wx, kx = _ptr(x, np.float64)
        else:
            if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
                x = np.ascontiguousarray(x, dtype=np.float64)
            xp, wx, kx = x.ctypes.data, RB_HOST, x
        if wb != wx:
            raise ValueError("b and x must live in the same memory space")
        st = Stats()
        code = lib().rbicgstab_solve_l(self._h, int(ell), bp, xp, wb, ctypes.byref(st))
        if code in HARD_ERRORS:
            raise RbError(code, "rbicgstab_solve_l")
        return SolveResult(x=x, stats=st.as_dict())

    def sell_stats(self):
        """(slices, stencil slices) of the current matrix's SELL-32 layout
        (rbicgstab_sell_stats)."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().rbicgstab_sell_stats(self._h, ctypes.byref(a), ctypes.byref(b)), "rbicgstab_sell_stats")
        return int(a.value), int(b.value)

    def apply(self, v, transpose=False):
        """y = A v (or A^T v) with the library's SpMV."""
        vp, w, keep = _ptr(v, np.float64)
        if _is_torch(v):
            import torch
            y = torch.empty_like(v)
            yp = y.data_ptr()
        else:
            y = np.empty(len(v))
            yp = y.ctypes.data
        _check(lib().rbicgstab_apply(self._h, vp, yp, int(bool(transpose)), w), "rbicgstab_apply")
        return y

    def pattern_outer(self, u, v, scale=1.0):
        """out_e = scale * u_i * v_j over the entries (i, j) of the matrix's
        pattern in the CSR order of set_matrix (rbicgstab_pattern_outer);
        u, v are CUDA tensors, the result a CUDA tensor of nnz values."""
        import torch
        if not (_is_torch(u) and _is_torch(v) and u.is_cuda and v.is_cuda):
            raise ValueError("pattern_outer takes CUDA tensors")
        up, _, ku = _ptr(u, np.float64)
        vp2, _, kv = _ptr(v, np.float64)
        out = torch.empty(self.nnz, dtype=torch.float64, device=u.device)
        _check(lib().rbicgstab_pattern_outer(self._h, up, vp2, float(scale), out.data_ptr(), RB_DEVICE),
               "rbicgstab_pattern_outer")
        return out


class Batch:
    """Batched solves of many independent systems (rbicgstab_batch_*): one
    launch per pass for all systems.  ``matrices`` is a list of CSR systems
    (objects with n, row_ptr, col, val, e.g. ``inputs.CSR``); right-hand
    sides and solutions are lists of per-system vectors (or one concatenated
    array / CUDA tensor of sum n_i entries)."""

    def __init__(self, matrices, *, k_max=0, tol=1e-8, max_itn=0, precision="fp64", poll=0,
                 shadow_seed=0, stream=None):
        o = Opts()
        o.k_max = int(k_max)
        o.cycle_s = 25
        o.max_itn = int(max_itn)
        o.precision = PRECISION[precision]
        o.recycle_mode = RECYCLE["fixed" if k_max else "none"]
        o.poll = int(poll)
        o.tol = float(tol)
        o.shadow_seed = int(shadow_seed)
        o.cuda_stream = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        h = ctypes.c_void_p()
        _check(lib().rbicgstab_batch_create(ctypes.byref(h), ctypes.byref(o)), "rbicgstab_batch_create")
        self._h = h
        self.sizes = [int(m.n) for m in matrices]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        n = np.asarray(self.sizes, dtype=np.int64)
        rp = np.concatenate([np.asarray(m.row_ptr, dtype=np.int32) for m in matrices])
        col = np.concatenate([np.asarray(m.col, dtype=np.int32) for m in matrices])
        val = np.concatenate([np.asarray(m.val, dtype=np.float64) for m in matrices])
        self.nnz = len(val)
        _check(lib().rbicgstab_batch_set_matrices(self._h, len(self.sizes), n.ctypes.data, rp.ctypes.data,
                                                  col.ctypes.data, val.ctypes.data), "rbicgstab_batch_set_matrices")

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().rbicgstab_batch_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def _cat(self, xs, dtype=np.float64):
        if isinstance(xs, (list, tuple)):
            if any(_is_torch(v) for v in xs):
                import torch
                return torch.cat([v.reshape(-1) for v in xs]).contiguous()
            return np.concatenate([np.asarray(v, dtype=dtype).reshape(-1) for v in xs])
        return xs

    def set_values(self, vals):
        v = self._cat(vals)
        p, w, keep = _ptr(v, np.float64)
        _check(lib().rbicgstab_batch_set_values(self._h, p, w), "rbicgstab_batch_set_values")

    def set_recycle(self, Us):
        """One (n_i, k) block per system (or None to clear)."""
        if Us is None:
            _check(lib().rbicgstab_batch_set_recycle(self._h, 0, None, RB_HOST), "rbicgstab_batch_set_recycle")
            return
        k = int(np.shape(Us[0])[1])
        blocks = np.concatenate([np.asfortranarray(u, dtype=np.float64).ravel(order="F") for u in Us])
        _check(lib().rbicgstab_batch_set_recycle(self._h, k, blocks.ctypes.data, RB_HOST),
               "rbicgstab_batch_set_recycle")

    def solve(self, bs, xs=None):
        """Returns (list of per-system solutions, list of per-system stats)."""
        b = self._cat(bs)
        if xs is None:
            if _is_torch(b):
                import torch
                x = torch.zeros_like(b)
            else:
                x = np.zeros(len(b))
        else:
            x = self._cat(xs)
            if not _is_torch(x):
                x = np.ascontiguousarray(x, dtype=np.float64)
        bp, wb, kb = _ptr(b, np.float64)
        xp, wx, kx = (_ptr(x, np.float64) if _is_torch(x) else (x.ctypes.data, RB_HOST, x))
        if wb != wx:
            raise ValueError("b and x must live in the same memory space")
        st = (Stats * len(self.sizes))()
        code = lib().rbicgstab_batch_solve(self._h, bp, xp, wb, st)
        stats = [s.as_dict() for s in st]
        # a per-system outcome (one system's non-finite iterate, breakdown or
        # non-convergence) is in that system's stats; other codes raise
        if code in HARD_ERRORS and not any(d["status"] == code for d in stats):
            raise RbError(code, "rbicgstab_batch_solve")
        parts = [x[self.offsets[i]:self.offsets[i + 1]] for i in range(len(self.sizes))]
        return parts, stats

    def info(self):
        a, b, c, d = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0)
        _check(lib().rbicgstab_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
               "rbicgstab_batch_info")
        return {"tile_slices": a.value, "ctas_per_sm": b.value, "tiles": c.value, "tuned_p1_ms": d.value}


def wait_selftest(complete: bool, limit_ms: float):
    """Run the library's bounded device wait once (rbicgstab_wait_selftest):
    returns (status, kernel milliseconds); RB_ETIMEOUT when nothing completes
    the barrier, RB_OK when it is completed first."""
    ms = ctypes.c_double(0.0)
    code = lib().rbicgstab_wait_selftest(int(bool(complete)), float(limit_ms), ctypes.byref(ms))
    if code not in (RB_OK, C["RB_ETIMEOUT"]):
        raise RbError(code, "rbicgstab_wait_selftest")
    return code, ms.value


def residual_noalloc(row_ptr, col, val, x, b, r, rnorm2, stream=None, n=None) -> int:
    """r = b - A x and rnorm2[0] = ||r||^2 (rbicgstab_residual_noalloc).

    For callers that cannot allocate device memory: every argument is a CUDA
    tensor the caller owns (int32 row_ptr/col, float64 val/x/b/r, a
    one-element float64 rnorm2); the library allocates nothing.  Ordered on
    ``stream`` (default: the legacy default stream), not synchronised.

    Every argument is checked before a pointer is taken (type, device,
    contiguity, dtype and length); a bad one raises RbError(RB_EINVAL)."""
    tensors = (row_ptr, col, val, x, b, r, rnorm2)
    einval = C["RB_EINVAL"]
    for t in tensors:
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise RbError(einval, "residual_noalloc takes contiguous CUDA tensors")
    import torch
    dev = row_ptr.device
    if any(t.device != dev for t in tensors):
        raise RbError(einval, "residual_noalloc: all tensors on one device")
    for t, dt, name in ((row_ptr, torch.int32, "row_ptr"), (col, torch.int32, "col"),
                        (val, torch.float64, "val"), (x, torch.float64, "x"),
                        (b, torch.float64, "b"), (r, torch.float64, "r"),
                        (rnorm2, torch.float64, "rnorm2")):
        if t.dtype != dt:
            raise RbError(einval, f"residual_noalloc: {name} must be {dt}")
    nn = (row_ptr.numel() - 1) if n is None else int(n)
    if nn < 0 or row_ptr.numel() < nn + 1:
        raise RbError(einval, "residual_noalloc: row_ptr needs n + 1 entries")
    if col.numel() != val.numel():
        raise RbError(einval, "residual_noalloc: col and val differ in length")
    if min(x.numel(), b.numel(), r.numel()) < nn:
        raise RbError(einval, "residual_noalloc: x, b and r need n entries")
    if rnorm2.numel() < 1:
        raise RbError(einval, "residual_noalloc: rnorm2 needs one entry")
    if nn > 0:
        nnz = int(row_ptr[nn].item())
        if nnz > col.numel():
            raise RbError(einval, "residual_noalloc: row_ptr[n] exceeds the length of col and val")
    args = [t.data_ptr() for t in tensors]
    sp = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    return _check(lib().rbicgstab_residual_noalloc(nn, *args, sp), "rbicgstab_residual_noalloc")


GRAM_PATH = {"auto": 0, "cudacore": 1, "tensor": 2}


def update_gram(Y, AY, P, AP, S, AS, kcap: int, scap: int, path: str = "auto", stream=None):
    """Gram step of the recycle update (rbicgstab_update_gram): returns
    (G, H) = (Z^T Z, Z^T W) as float64 numpy arrays for W = [Y, P, S],
    Z = [AY, AP, AS].  Each block is a CUDA float32 tensor of shape
    (columns, ld): the columns stored one after another (column-major with
    leading dimension ld, shared by all blocks); n = ld."""
    blocks = (Y, AY, P, AP, S, AS)
    for t in blocks:
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise RbError(C["RB_EINVAL"], "update_gram takes contiguous CUDA tensors")
    import torch
    if any(t.dtype != torch.float32 or t.dim() != 2 for t in blocks):
        raise RbError(C["RB_EINVAL"], "update_gram takes 2-D float32 tensors (columns, ld)")
    ld = Y.shape[1]
    if any(t.shape[1] != ld for t in blocks):
        raise RbError(C["RB_EINVAL"], "update_gram: blocks differ in ld")
    return update_gram_n(ld, Y, AY, P, AP, S, AS, kcap, scap, path, stream)


def update_gram_n(n: int, Y, AY, P, AP, S, AS, kcap: int, scap: int, path: str = "auto", stream=None,
                  timing: bool = False):
    """update_gram with the vector length n <= ld given explicitly.  With
    ``timing`` returns (G, H, ms) where ms is the Gram kernels' device time."""
    ld = Y.shape[1]
    ky, nit, ns = Y.shape[0], P.shape[0], S.shape[0]
    if AY.shape[0] != ky or AP.shape[0] != nit or AS.shape[0] != ns:
        raise RbError(C["RB_EINVAL"], "update_gram: W and Z blocks differ in columns")
    m = ky + nit + ns
    G = np.zeros((m, m), order="F")
    H = np.zeros((m, m), order="F")
    sp = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    ptr = lambda t: t.data_ptr() if t.numel() else None
    ms = ctypes.c_double(0.0)
    _check(lib().rbicgstab_update_gram(int(n), int(ld), ky, nit, ns, int(kcap), int(scap), ptr(Y), ptr(AY),
                                       ptr(P), ptr(AP), ptr(S), ptr(AS), G.ctypes.data, H.ctypes.data,
                                       GRAM_PATH[path], sp, ctypes.byref(ms) if timing else None),
           "rbicgstab_update_gram")
    return (G, H, ms.value) if timing else (G, H)


def kernel_launches() -> int:
    """Kernels launched by the library in this process (rbicgstab_kernel_launches)."""
    return int(lib().rbicgstab_kernel_launches())


def time_passes(solver: "Solver", b, reps: int = 10):
    """Average ms of passes P1..P5 (rbicgstab_time_passes) for one right-hand
    side (b of shape (n,)) or a block (shape (nrhs, n)); returns (ms[5], status)."""
    shape = tuple(np.shape(b))
    nrhs, n = (1, shape[0]) if len(shape) == 1 else shape
    bp, w, keep = _ptr(b, np.float64)
    ms = np.zeros(5)
    code = lib().rbicgstab_time_passes(solver._h, int(nrhs), bp, int(n), w, int(reps), ms.ctypes.data)
    _check(code, "rbicgstab_time_passes")
    return ms, code


def svd_small(M: np.ndarray):
    """Host SVD of the library's biorthogonalisation (rbicgstab_svd_small):
    M = P diag(sigma) Q^T, sigma descending."""
    k = M.shape[0]
    Mf = np.asfortranarray(M, dtype=np.float64)
    P = np.zeros((k, k), order="F")
    Q = np.zeros((k, k), order="F")
    sig = np.zeros(k)
    _check(lib().rbicgstab_svd_small(k, Mf.ctypes.data, P.ctypes.data, sig.ctypes.data, Q.ctypes.data),
           "rbicgstab_svd_small")
    return P, sig, Q


def harmonic_ritz(G: np.ndarray, H: np.ndarray, k: int):
    """Host harmonic-Ritz step of the library (rbicgstab_harmonic_ritz)."""
    m = G.shape[0]
    Gf = np.asfortranarray(G, dtype=np.float64)
    Hf = np.asfortranarray(H, dtype=np.float64)
    Y = np.zeros((m, k), order="F")
    tr = np.zeros(k)
    ti = np.zeros(k)
    ku = ctypes.c_int32()
    code = lib().rbicgstab_harmonic_ritz(m, Gf.ctypes.data, Hf.ctypes.data, k, Y.ctypes.data,
                                         tr.ctypes.data, ti.ctypes.data, ctypes.byref(ku))
    _check(code, "rbicgstab_harmonic_ritz")
    kk = ku.value
    return Y[:, :kk], tr[:kk] + 1j * ti[:kk]
