"""Semi-smooth Newton (section 3.1) around the MGR-preconditioned FGMRES solve.

The nonlinear complementarity problem min(F(u), G(u)) = 0 is linearised at each iterate with the
active-set rule of the semi-smooth Newton method: a constraint row takes the derivative of the
branch that attains the minimum (F' where F < G, G' where F >= G).  Each step solves
J(u_k) du = -R(u_k) and sets u_{k+1} = u_k + du; it stops when ||R(u_k)||_2 <= tol (section 6 uses
||F|| <= 1e-5).  The active set fixes which constraint rows are saddle-point rows, so the MGR
cf_marker of the step follows it.

The assembly of R and J belongs to the application (the caller passes `assemble`); this module
holds the outer loop and `MgrLinearSolver`, which keeps the block pattern on the device across steps
(the Jacobian's pattern is fixed by the primary variables, section 3.1) and copies only the values,
the marker and the right-hand side per step.  Every linear solve runs on the GPU.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable

import numpy as np


@dataclasses.dataclass
class NewtonStep:
    step: int
    resnorm: float
    active_changes: int      # constraint rows whose branch differs from the previous step
    lin_iterations: int = 0
    lin_converged: bool = True
    setup_ms: float = 0.0
    solve_ms: float = 0.0
    host_ms: float = 0.0     # assembly and copies


class MgrLinearSolver:
    """J du = rhs on the GPU: MGR setup on the step's Jacobian and cf_marker, then FGMRES(restart)
    to rtol.  The BSR pattern (rowptr, colind) is uploaded once and reused while it is unchanged."""

    def __init__(self, opts=None, rtol: float = 1e-8, restart: int = 30, maxit: int = 1000, device: str = "cuda",
                 **options):
        from . import MGR, options as make_options
        self.m = MGR(opts if opts is not None else make_options(**options))
        self.rtol, self.restart, self.maxit, self.device = rtol, restart, maxit, device
        self._pattern = None
        self.pattern_uploads = 0

    def _upload_pattern(self, rowptr, colind):
        import torch
        if self._pattern is not None:
            rp_h, ci_h, _, _ = self._pattern
            if rp_h.shape == rowptr.shape and ci_h.shape == colind.shape and np.array_equal(rp_h, rowptr) \
                    and np.array_equal(ci_h, colind):
                return self._pattern[2], self._pattern[3]
        rp = torch.as_tensor(np.ascontiguousarray(rowptr, np.int64), device=self.device)
        ci = torch.as_tensor(np.ascontiguousarray(colind, np.int32), device=self.device)
        self._pattern = (np.array(rowptr, copy=True), np.array(colind, copy=True), rp, ci)
        self.pattern_uploads += 1
        return rp, ci

    def __call__(self, rowptr, colind, values, marker, rhs):
        import torch
        from . import BSR3
        rp, ci = self._upload_pattern(rowptr, colind)
        v = torch.as_tensor(np.ascontiguousarray(values, np.float64), device=self.device)
        mk = torch.as_tensor(np.ascontiguousarray(marker, np.int8), device=self.device)
        b = torch.as_tensor(np.ascontiguousarray(rhs, np.float64), device=self.device)
        A = BSR3(rp, ci, v.reshape(-1, 3, 3))
        self.m.setup(A, mk)
        setup_ms = self.m.stats()["setup_ms"]
        x, info = self.m.fgmres(A, b, rtol=self.rtol, restart=self.restart, maxit=self.maxit)
        info = dict(info)
        info["setup_ms"] = setup_ms
        return x.cpu().numpy(), info

    def close(self):
        self.m.close()


def semismooth_newton(assemble: Callable, u0: np.ndarray, solve: Callable, tol: float = 1e-5,
                      max_steps: int = 30):
    """Newton iterations from u0.

    assemble(u) -> (rowptr, colind, values, R, marker, active): the BSR Jacobian at u (values
    [nnzb, 3, 3]), the residual R(u), the MGR cf_marker of the step and the active set (a boolean per
    constraint row, True where the G branch is taken).
    solve(rowptr, colind, values, marker, rhs) -> (du, info) with info["iterations"],
    info["converged"] and optionally info["setup_ms"], info["solve_ms"].

    Returns (u, history, converged)."""
    u = np.array(u0, dtype=np.float64, copy=True).reshape(-1)
    hist = []
    prev = None
    for k in range(max_steps + 1):
        t0 = time.perf_counter()
        rowptr, colind, values, R, marker, active = assemble(u)
        rn = float(np.linalg.norm(R))
        changes = 0 if prev is None else int(np.count_nonzero(prev != active))
        prev = np.array(active, copy=True)
        st = NewtonStep(k, rn, changes)
        hist.append(st)
        if rn <= tol:
            st.host_ms = (time.perf_counter() - t0) * 1e3
            return u, hist, True
        if k == max_steps:
            break
        du, info = solve(rowptr, colind, values, marker, -R)
        st.lin_iterations = int(info.get("iterations", 0))
        st.lin_converged = bool(info.get("converged", True))
        st.setup_ms = float(info.get("setup_ms", 0.0))
        st.solve_ms = float(info.get("solve_ms", 0.0))
        st.host_ms = (time.perf_counter() - t0) * 1e3 - st.setup_ms - st.solve_ms
        if not np.all(np.isfinite(du)):
            break
        u = u + du
    return u, hist, False
