"""The adjoint workloads at full size on the GPU.

64^3 adjoint (786,432 unknowns, FP32 hierarchy / FP64 Krylov): the gradient of L = w . x with respect
to the BSR values, from the MGR-preconditioned A^T solve, against central finite differences of
forward solves on 32 seeded stored entries.
"""
import numpy as np
import pytest

import ncpgen
from gpu_common import to_gpu

pytestmark = pytest.mark.gpu

SOLVER = dict(precision="mixed", amg_theta=0.5, amg_pmax=4, amg_smoother=0, amg_omega=0.8)


def _fd_scale(p):
    """Per stored scalar entry: max(|a_ij|, largest |a_ik| of its scalar row)."""
    rows = np.repeat(np.arange(p.nb), np.diff(p.rowptr))
    rowmax = np.zeros((p.nb, 3))
    np.maximum.at(rowmax, rows, np.abs(p.values).max(axis=2))
    return np.maximum(np.abs(p.values), rowmax[rows][:, :, None]).reshape(-1)


def test_adjoint_64cube_finite_differences():
    """Central differences, step 1e-6 of max(|a_ij|, its row's largest entry), forward solves at
    rtol 1e-13 from the unperturbed solution; relative error <= 1e-5 on 32 seeded nonzero entries
    (relative to max(|g|, 1e-3 max|g|))."""
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.WORKLOADS["ncp3d_64_adjoint"])
    b = torch.as_tensor(ncpgen.normals(p.n, 2), device="cuda")
    w = torch.as_tensor(ncpgen.normals(p.n, 4, stream=4), device="cuda")
    A, mk = to_gpu(p)
    opts = mg.options(**SOLVER)
    vals = A.values.clone().requires_grad_(True)
    bt = b.clone().requires_grad_(True)
    stats = {}
    x = mg.mgr_solve(vals, bt, A.rowptr, A.colind, mk, opts, rtol=1e-12, maxit=3000, stats=stats)
    (x * w).sum().backward()
    assert stats["forward"]["converged"] and stats["adjoint"]["converged"]
    # lambda = dL/db solves A^T lambda = w
    At = mg.bsr3_transpose(A)
    lam = bt.grad.detach()
    r = mg.bsr3_spmv(At, lam, sub=w)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(w)) <= 1e-11
    g = vals.grad.reshape(-1).cpu().numpy()
    gmax = np.abs(g).max()

    m = mg.MGR(opts)
    x0 = x.detach()

    def loss(v):
        Av = A.with_values(v.reshape(-1, 3, 3))
        m.setup(Av, mk)
        xx, info = m.fgmres(Av, b, x=x0.clone(), rtol=1e-13, maxit=3000)
        assert info["converged"]
        return float((xx * w).sum())

    scale = _fd_scale(p)
    flat = p.values.reshape(-1)
    rng = np.random.default_rng(5)
    picks = rng.choice(np.nonzero(flat != 0.0)[0], 32, replace=False)
    worst = 0.0
    for k in picks:
        h = 1e-6 * scale[k]
        vp = A.values.clone().reshape(-1)
        vm = A.values.clone().reshape(-1)
        vp[k] += h
        vm[k] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        err = abs(fd - g[k]) / max(abs(g[k]), 1e-3 * gmax)
        worst = max(worst, err)
    m.close()
    print(f"64^3 adjoint: forward {stats['forward']['iterations']} it, adjoint {stats['adjoint']['iterations']} it, "
          f"worst FD relative error {worst:.2e}")
    assert worst <= 1e-5, worst

