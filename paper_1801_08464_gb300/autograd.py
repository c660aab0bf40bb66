"""Adjoint differentiation of x = A(theta)^-1 b through the MGR-preconditioned solve.

Forward: mgr_setup(A, cf_marker) with the transposed operators built too (options.adjoint = 1) and
fgmres_solve(A, b).  Backward, for an upstream gradient g = dL/dx: the same hierarchy solves
A^T lambda = g by fgmres_solve_transpose, preconditioned from the left with M^-T, the transpose of the
forward preconditioner (the operator M^-T A^T = (A M^-1)^T is the transpose of the forward one); then
dL/db = lambda and dL/dA_ij = -lambda_i x_j on the stored block pattern (mgr_bsr3_outer_grad).  The hierarchy lives from
the forward call until the backward call returns (or until the graph is freed).

adjoint="rebuild" instead builds a second hierarchy by mgr_setup on A^T (mgr_bsr3_transpose, same
cf_marker) in the backward pass and solves with it by right-preconditioned FGMRES.
"""
from __future__ import annotations

import ctypes

import torch


def _record(stats, key, m, info):
    if stats is None:
        return
    d = dict(info)
    d["setup_ms"] = m.stats()["setup_ms"]
    d["memory_peak_bytes"] = m.memory_peak_bytes()
    stats[key] = d


def _with_adjoint(opts):
    from . import Options
    o = Options()
    ctypes.memmove(ctypes.byref(o), ctypes.byref(opts), ctypes.sizeof(Options))
    o.adjoint = 1
    return o


class MgrSolve(torch.autograd.Function):
    """x = A^-1 b with A = BSR3(rowptr, colind, values); differentiable in values and b."""

    @staticmethod
    def forward(ctx, values, b, rowptr, colind, cf_marker, opts, rtol, restart, maxit, stats, adjoint):
        from . import BSR3, MGR
        if adjoint not in ("transpose", "rebuild"):
            raise ValueError("adjoint must be 'transpose' or 'rebuild'")
        A = BSR3(rowptr, colind, values.detach().reshape(-1, 3, 3).contiguous())
        m = MGR(_with_adjoint(opts) if adjoint == "transpose" else opts)
        m.setup(A, cf_marker)
        x, info = m.fgmres(A, b.detach().contiguous(), rtol=rtol, restart=restart, maxit=maxit)
        _record(stats, "forward", m, info)
        if adjoint == "rebuild":
            m.close()
            m = None
        ctx.save_for_backward(values, x, rowptr, colind, cf_marker)
        ctx.m, ctx.opts, ctx.adjoint = m, opts, adjoint
        ctx.rtol, ctx.restart, ctx.maxit, ctx.stats = rtol, restart, maxit, stats
        ctx.forward_info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        from . import BSR3, MGR, bsr3_outer_grad, bsr3_transpose
        values, x, rowptr, colind, cf_marker = ctx.saved_tensors
        A = BSR3(rowptr, colind, values.detach().reshape(-1, 3, 3).contiguous())
        if ctx.adjoint == "transpose":
            m = ctx.m
            lam, info = m.fgmres(A, gx.contiguous(), rtol=ctx.rtol, restart=ctx.restart, maxit=ctx.maxit,
                                 transpose=True)
        else:
            At = bsr3_transpose(A)
            m = MGR(ctx.opts)
            m.setup(At, cf_marker)
            lam, info = m.fgmres(At, gx.contiguous(), rtol=ctx.rtol, restart=ctx.restart, maxit=ctx.maxit)
            del At
        _record(ctx.stats, "adjoint", m, info)
        m.close()
        ctx.m = None
        gvals = bsr3_outer_grad(A, lam, x).reshape(values.shape)
        return gvals, lam, None, None, None, None, None, None, None, None, None


def mgr_solve(values, b, rowptr, colind, cf_marker, opts=None, rtol=1e-8, restart=30, maxit=1000, stats=None,
              adjoint="transpose"):
    """Differentiable x = A^-1 b.  adjoint selects the backward solve: "transpose" (the forward
    hierarchy's transposed preconditioner, default) or "rebuild" (a new hierarchy on A^T).  If `stats`
    is a dict, it receives the forward solve's info (and, after backward, the adjoint solve's) with
    the setup time and the handle's peak device bytes."""
    from . import options
    o = opts if opts is not None else options()
    return MgrSolve.apply(values, b, rowptr, colind, cf_marker, o, rtol, restart, maxit, stats, adjoint)
