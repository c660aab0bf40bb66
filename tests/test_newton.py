"""The semi-smooth Newton loop (section 3.1) on the host: with an exact linear solver it converges
quadratically on the two-level unsaturated case and on a 3-D case whose active set changes (gas
appears), and it reports the active-set changes."""
import numpy as np
import pytest

import ncpgen


def _direct(rowptr, colind, values, marker, rhs):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n = rhs.size
    J = sp.bsr_matrix((values, colind, rowptr), shape=(n, n)).tocsc()
    return spla.spsolve(J, rhs), {"iterations": 1, "converged": True}


@pytest.mark.parametrize("cfg", [
    ncpgen.WORKLOADS["unsat2d_200x10"],
    ncpgen.GridConfig(8, 8, 4, sigma=1.0, absent_frac=0.4, absent_mode=1, seed=3),
])
def test_newton_converges_quadratically(cfg):
    from paper_1801_08464_gb300.newton import semismooth_newton
    p = ncpgen.make_problem(cfg)
    u0 = p.state.reshape(-1).copy()
    u, hist, ok = semismooth_newton(lambda u: ncpgen.newton_system(cfg, u, u0), u0, _direct, tol=1e-9)
    assert ok and len(hist) <= 9
    r = [h.resnorm for h in hist]
    # the last steps contract at least quadratically (r_{k+1} <= C r_k^2 once r_k is small)
    assert r[-1] <= 1e-9 and r[-2] <= 1e-2 * r[-3]
    R = ncpgen.residual(cfg, u, u0)
    assert np.linalg.norm(R) <= 1e-9
    if cfg.absent_frac > 0:
        assert sum(h.active_changes for h in hist) > 0  # phase appearance during the step
        # the final active set is the min-function branch of the converged state
        _, _, _, _, _, act = ncpgen.newton_system(cfg, u, u0)
        s = u[1::3]
        assert np.all(s[~act] == pytest.approx(1.0, abs=1e-8))
