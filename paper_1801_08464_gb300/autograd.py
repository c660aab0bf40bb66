"""Adjoint differentiation of x = A(theta)^-1 b through the MGR-preconditioned solve.

Forward: mgr_setup(A, cf_marker) and fgmres_solve(A, b).  Backward, for an upstream gradient
g = dL/dx: transpose the blocks of A (mgr_bsr3_transpose), build an MGR hierarchy for A^T with the
same cf_marker, solve A^T lambda = g with FGMRES, then dL/db = lambda and
dL/dA_ij = -lambda_i x_j on the stored block pattern (mgr_bsr3_outer_grad).  Each hierarchy is
released as soon as its solve returns, so the forward and the adjoint never hold device memory at
the same time.
"""
from __future__ import annotations

import torch


def _record(stats, key, m, info):
    if stats is None:
        return
    d = dict(info)
    d["setup_ms"] = m.stats()["setup_ms"]
    d["memory_peak_bytes"] = m.memory_peak_bytes()
    stats[key] = d


class MgrSolve(torch.autograd.Function):
    """x = A^-1 b with A = BSR3(rowptr, colind, values); differentiable in values and b."""

    @staticmethod
    def forward(ctx, values, b, rowptr, colind, cf_marker, opts, rtol, restart, maxit, stats):
        from . import BSR3, MGR
        A = BSR3(rowptr, colind, values.detach().reshape(-1, 3, 3).contiguous())
        m = MGR(opts)
        m.setup(A, cf_marker)
        x, info = m.fgmres(A, b.detach().contiguous(), rtol=rtol, restart=restart, maxit=maxit)
        _record(stats, "forward", m, info)
        m.close()
        ctx.save_for_backward(values, x, rowptr, colind, cf_marker)
        ctx.opts, ctx.rtol, ctx.restart, ctx.maxit, ctx.stats = opts, rtol, restart, maxit, stats
        ctx.forward_info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        from . import BSR3, MGR, bsr3_outer_grad, bsr3_transpose
        values, x, rowptr, colind, cf_marker = ctx.saved_tensors
        A = BSR3(rowptr, colind, values.detach().reshape(-1, 3, 3).contiguous())
        At = bsr3_transpose(A)
        m = MGR(ctx.opts)
        m.setup(At, cf_marker)
        lam, info = m.fgmres(At, gx.contiguous(), rtol=ctx.rtol, restart=ctx.restart, maxit=ctx.maxit)
        _record(ctx.stats, "adjoint", m, info)
        m.close()
        del At
        gvals = bsr3_outer_grad(A, lam, x).reshape(values.shape)
        return gvals, lam, None, None, None, None, None, None, None, None


def mgr_solve(values, b, rowptr, colind, cf_marker, opts=None, rtol=1e-8, restart=30, maxit=1000, stats=None):
    """Differentiable x = A^-1 b.  If `stats` is a dict, it receives the forward solve's info (and,
    after backward, the adjoint solve's) with setup time and the handle's peak device bytes."""
    from . import options
    o = opts if opts is not None else options()
    return MgrSolve.apply(values, b, rowptr, colind, cf_marker, o, rtol, restart, maxit, stats)
