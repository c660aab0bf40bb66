"""The semi-smooth Newton loop (section 3.1) with the GPU linear solver against the same loop with
the oracle's FP64 MGR-FGMRES: same number of Newton steps, same final active set, final states equal
to 1e-7; every GPU solve converges and the block pattern is uploaded once per loop."""
import numpy as np
import pytest

import ncpgen
import oracle
from gpu_common import UNSAT

pytestmark = pytest.mark.gpu

CASES = {
    # two-level unsaturated case, two time steps
    "unsat2d_200x10": (ncpgen.WORKLOADS["unsat2d_200x10"], UNSAT, 2),
    # 3-D NCP case whose active set changes during the step (gas appears), one time step
    "ncp3d_16x16x8": (ncpgen.GridConfig(16, 16, 8, sigma=1.0, absent_frac=0.4, absent_mode=1, seed=3), {}, 1),
}


def _oracle_solve(opts):
    def solve(rowptr, colind, values, marker, rhs):
        o = oracle.OracleMGR(rowptr, colind, values.reshape(-1, 3, 3), marker, **opts)
        x, info = o.fgmres(rhs, rtol=1e-8)
        return x, {"iterations": info["iterations"], "converged": info["converged"]}
    return solve


def _run(cfg, solve, steps):
    from paper_1801_08464_gb300.newton import semismooth_newton
    u = ncpgen.make_problem(cfg).state.reshape(-1).copy()
    hists, acts = [], []
    for _ in range(steps):
        u_old = u.copy()
        u, hist, ok = semismooth_newton(lambda v: ncpgen.newton_system(cfg, v, u_old), u, solve, tol=1e-7)
        assert ok
        hists.append(hist)
        acts.append(ncpgen.newton_system(cfg, u, u_old)[5])
    return u, hists, acts


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_newton_gpu_matches_oracle_loop(name, precision):
    from paper_1801_08464_gb300.newton import MgrLinearSolver
    cfg, opts, steps = CASES[name]
    gsolve = MgrLinearSolver(precision=precision, **opts)
    ug, hg, ag = _run(cfg, gsolve, steps)
    uo, ho, ao = _run(cfg, _oracle_solve(opts), steps)
    assert gsolve.pattern_uploads == 1
    for a, b in zip(hg, ho):
        assert abs(len(a) - len(b)) <= 1, ([h.resnorm for h in a], [h.resnorm for h in b])
        assert all(h.lin_converged for h in a)
    for a, b in zip(ag, ao):
        assert np.array_equal(a, b)
    assert np.linalg.norm(ug - uo) <= 1e-7 * np.linalg.norm(uo)
    if name.startswith("ncp3d"):
        assert sum(h.active_changes for h in hg[0]) > 0
    print(f"{name}/{precision}: Newton steps {[len(h) - 1 for h in hg]}, linear iterations "
          f"{[[h.lin_iterations for h in hh[:-1]] for hh in hg]}")
    gsolve.close()
