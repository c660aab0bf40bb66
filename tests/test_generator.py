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
