"""The input generator: its Jacobian is the derivative of its residual, and it has the block
structure the paper describes for the NCP linear system (section 3.2)."""
import numpy as np
import pytest

import ncpgen


def _dense(p):
    return p.to_scipy().toarray()


@pytest.mark.parametrize("cfg", [
    ncpgen.GridConfig(8, 8, 1, sigma=1.0, absent_frac=0.3, absent_mode=0, seed=11),
    ncpgen.GridConfig(4, 4, 4, sigma=2.0, absent_frac=0.5, absent_mode=1, seed=12),
    ncpgen.GridConfig(4, 3, 5, sigma=1.0, layer_contrast=1e-4, absent_frac=0.4, absent_mode=1, seed=13),
])
def test_jacobian_matches_central_differences(cfg):
    p = ncpgen.make_problem(cfg)
    u0 = p.state.reshape(-1).copy()
    J = _dense(p)
    Jfd = np.zeros_like(J)
    for j in range(u0.size):
        h = 1e-7 * max(1.0, abs(u0[j]))
        up, um = u0.copy(), u0.copy()
        up[j] += h
        um[j] -= h
        Jfd[:, j] = (ncpgen.residual(cfg, up) - ncpgen.residual(cfg, um)) / (2 * h)
    scale = np.abs(J).max()
    assert np.abs(J - Jfd).max() <= 1e-6 * scale


def _fd_at(cfg, u0):
    rp, ci, v = ncpgen.jacobian(cfg, u0)
    import scipy.sparse as sp
    n = u0.size
    J = sp.bsr_matrix((v, ci, rp), shape=(n, n)).toarray()
    Jfd = np.zeros_like(J)
    for j in range(n):
        h = 1e-7 * max(1.0, abs(u0[j]))
        up, um = u0.copy(), u0.copy()
        up[j] += h
        um[j] -= h
        Jfd[:, j] = (ncpgen.residual(cfg, up) - ncpgen.residual(cfg, um)) / (2 * h)
    return np.abs(J - Jfd).max() / np.abs(J).max()


@pytest.mark.parametrize("cfg,spread", [
    # the unsaturated two-sub-domain state (section 6.1), closed boundary
    (ncpgen.GridConfig(8, 4, 1, sigma=0.0, absent_frac=0.0, closure=1, state_mode=1, closed=1), False),
    # Van Genuchten closures on a seeded heterogeneous state with the outlet, gas present everywhere
    (ncpgen.GridConfig(6, 5, 1, sigma=1.0, absent_frac=0.0, closure=1, seed=5), False),
    # saturations spread over the regularised P_c's linear continuations and its interior
    (ncpgen.GridConfig(5, 4, 1, sigma=0.5, absent_frac=0.0, closure=1, seed=7, closed=1), True),
])
def test_van_genuchten_jacobian_matches_central_differences(cfg, spread):
    """Section 2.3-2.4 closures: the Jacobian at a state off the upwinding ties (P_l perturbed) is
    the derivative of the residual; with `spread`, S_l takes values beyond 1 and below S_lr, where
    the regularised P_c continues linearly, besides interior ones."""
    p = ncpgen.make_problem(cfg)
    u0 = p.state.reshape(-1).copy()
    rng = np.random.default_rng(1)
    u0[0::3] += 1e-3 * rng.standard_normal(p.nb)
    if spread:
        u0[1::3] = np.resize([1.02, 0.005, 0.35, 0.7, 0.9, 0.97], p.nb)
    assert _fd_at(cfg, u0) <= 1e-6


def test_van_genuchten_closures_closed_forms():
    """P_c at the sub-domain states of section 6.1 equals P_g - P_l of its table of initial
    conditions (0.5 and 1.5 in units of P_l = 1e6 Pa; the table's saturations are rounded to 0.1 %
    and the regularisation shifts P_c by P_c(S_le = 1 - eps/2) ~ 1.4e-3, hence 5e-3); S_l = 1 has
    P_c = 0 (the shift), so a state on the Henry line rho = C_h P_l satisfies the constraint rows."""
    cfg = ncpgen.GridConfig(4, 2, 1, sigma=0.0, absent_frac=0.0, closure=1, state_mode=1, closed=1)
    p = ncpgen.make_problem(cfg)
    rho = p.state[:, 2]
    pg = rho / 0.02  # Henry line: rho = C_h P_g with C_h = 0.02
    pc = pg - p.state[:, 0]
    left = p.state[:, 1] == 0.962
    assert np.abs(pc[left] - 0.5).max() <= 5e-3 and np.abs(pc[~left] - 1.5).max() <= 5e-3
    u = p.state.reshape(-1).copy()
    u[1::3] = 1.0
    u[2::3] = 0.02 * u[0::3]  # P_c(1) = 0, so rho = C_h P_l on the Henry line
    R = ncpgen.residual(cfg, u)
    assert np.allclose(R[2::3], 0.0, atol=1e-15)
    # gas present everywhere: every constraint row is rho's (C_h, C_h P_c', -1), never the
    # saturation pin, so the diagonal has no zero (the two-level case of section 6.1)
    rows = np.repeat(np.arange(p.nb), np.diff(p.rowptr))
    d = p.values[rows == p.colind]
    assert np.all(d[:, 2, 2] == -1.0) and np.all(d[:, 2, 0] == 0.02)
    assert np.all(d[:, 0, 0] != 0.0) and np.all(d[:, 1, 1] != 0.0)


def test_two_level_markers_without_absent_gas():
    """Gas present everywhere: two reductions (rho -> 0, S_l -> 1) and P_l -> 2 (section 6.1)."""
    p = ncpgen.make_problem(ncpgen.WORKLOADS["unsat2d_200x10"])
    m = p.cf_marker.reshape(-1, 3)
    assert np.all(m[:, 0] == 2) and np.all(m[:, 1] == 1) and np.all(m[:, 2] == 0)
    assert p.nb == 2000 and np.all(p.gas_present == 1)


def test_constraint_rows_follow_active_set():
    """Section 3.2: gas absent -> A31 = 0, A32 = -1, A33 = 0; gas present -> A33 nonzero; the
    constraint rows are local (diagonal blocks only); A33 is zero exactly on gas-absent rows."""
    p = ncpgen.make_problem(ncpgen.GridConfig(6, 5, 4, sigma=1.5, absent_frac=0.4, absent_mode=1, seed=3))
    rows = np.repeat(np.arange(p.nb), np.diff(p.rowptr))
    diag = rows == p.colind
    assert np.all(p.values[~diag][:, 2, :] == 0.0)
    d = p.values[diag]
    absent = p.gas_present == 0
    assert np.array_equal(d[absent][:, 2, :], np.tile([0.0, -1.0, 0.0], (absent.sum(), 1)))
    assert np.all(d[~absent][:, 2, 2] != 0.0)
    assert np.array_equal(d[:, 2, 2] == 0.0, absent)


def test_markers_and_fractions():
    cfg = ncpgen.GridConfig(16, 16, 16, sigma=2.0, absent_frac=0.5, absent_mode=1, seed=1)
    p = ncpgen.make_problem(cfg)
    assert (p.gas_present == 0).sum() == round(0.5 * p.nb)
    m = p.cf_marker.reshape(-1, 3)
    assert np.all(m[:, 0] == 3) and np.all(m[:, 1] == 1)
    assert np.array_equal(m[:, 2], np.where(p.gas_present == 1, 0, 2))
    assert p.nnzb == p.nb + 2 * 3 * 15 * 16 * 16
    q = ncpgen.make_problem(cfg)
    assert np.array_equal(p.values, q.values) and np.array_equal(p.colind, q.colind)


def test_seeded_normals_are_standard():
    x = ncpgen.normals(200000, seed=2, stream=2)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    assert np.array_equal(x[:10], ncpgen.normals(10, seed=2, stream=2))
