"""``torch.autograd.Function`` for x = A^{-1} b on the library's solver.

The values of A (on the pattern given to ``Solver.set_matrix``) and b are the
differentiable inputs.  Forward: ``set_values`` and one solve (Alg. 2, with
the handle's recycle space).  Backward, for an upstream gradient g = dL/dx:
the dual system A^T lam = g (the dual system of Sec. 2, A^* x~ = b~ with
b~ = g) is solved by ``rbicgstab_solve_adjoint`` (Alg. 2 on A^T with the
recycle space's roles swapped: the left space U~ serves as the dual's right
space, reusing the setup's products); then

    dL/db = lam,    dL/dA_ij = -lam_i x_j   (``rbicgstab_pattern_outer``).

A parametrisation A(p) = sum_k p_k A_k written in torch upstream of the
values chains to dL/dp_k = -lam^T A_k x by autograd.  Argument marshalling
only: both solves and the gradient assembly run in the library's kernels.
"""
from __future__ import annotations

import torch

from . import rbicgstab as rb


class RecycledSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, b, solver, checkpoint=False):
        values = values.detach().contiguous()
        b = b.detach().contiguous()
        solver.set_values(values)
        res = solver.solve(b)
        if res.stats["status"] != rb.RB_OK:
            raise RuntimeError(f"forward solve: {rb.error_string(res.stats['status'])}")
        x = res.x
        ctx.solver = solver
        ctx.version = solver.values_version
        ctx.checkpoint = checkpoint
        # checkpointing: x is not kept; backward solves for it again (one
        # more forward solve in exchange for n values of memory per step)
        ctx.save_for_backward(values, b, *(() if checkpoint else (x,)))
        return x

    @staticmethod
    def backward(ctx, gx):
        saved = ctx.saved_tensors
        values, b = saved[0], saved[1]
        s = ctx.solver
        if s.values_version != ctx.version:   # the solver moved on: put this step's matrix back
            s.set_values(values)
        dual = s.solve_adjoint(gx.detach().contiguous())
        if dual.stats["status"] != rb.RB_OK:
            raise RuntimeError(f"dual solve: {rb.error_string(dual.stats['status'])}")
        lam = dual.x
        if ctx.checkpoint:
            res = s.solve(b)
            if res.stats["status"] != rb.RB_OK:
                raise RuntimeError(f"recomputed forward solve: {rb.error_string(res.stats['status'])}")
            x = res.x
        else:
            x = saved[2]
        gvals = s.pattern_outer(lam, x, -1.0) if ctx.needs_input_grad[0] else None
        gb = lam if ctx.needs_input_grad[1] else None
        return gvals, gb, None, None


def solve(solver: rb.Solver, values: torch.Tensor, b: torch.Tensor, checkpoint: bool = False) -> torch.Tensor:
    """x with A(values) x = b, differentiable in values and b (CUDA float64
    tensors; the solver holds the pattern from ``set_matrix``).  With
    ``checkpoint`` the solution is not stored for the backward pass but
    solved for again there (for long sequences of large systems)."""
    return RecycledSolve.apply(values, b, solver, checkpoint)
