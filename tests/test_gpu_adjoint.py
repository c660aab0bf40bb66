"""Adjoint of x = A(theta)^-1 b through the MGR-preconditioned solve (GPU).

The backward pass solves A^T lambda = dL/dx with an MGR hierarchy built for the transpose and
returns dL/db = lambda, dL/dA_ij = -lambda_i x_j on the pattern.  Checked against the oracle's dense
adjoint gradient on an 8x8x8 instance and against central finite differences of GPU solves on 32
seeded entries (h = 1e-6 relative), for L = w . x with w ~ N(0,1).
"""
import numpy as np
import pytest

import ncpgen
import oracle
from gpu_common import rel, to_gpu

pytestmark = pytest.mark.gpu

CFG8 = ncpgen.GridConfig(8, 8, 8, sigma=2.0, absent_frac=0.5, absent_mode=1, seed=1)


def test_block_transpose_and_outer_grad_kernels():
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.GridConfig(7, 5, 3, absent_frac=0.4, absent_mode=1, seed=2))
    A, _ = to_gpu(p)
    At = mg.bsr3_transpose(A)
    import scipy.sparse as sp
    T = sp.bsr_matrix((At.values.cpu().numpy(), At.colind.cpu().numpy(), At.rowptr.cpu().numpy()),
                      shape=(p.n, p.n)).toarray()
    assert np.array_equal(T, p.to_scipy().toarray().T)
    lam = ncpgen.normals(p.n, 3)
    x = ncpgen.normals(p.n, 4)
    g = mg.bsr3_outer_grad(A, torch.as_tensor(lam, device="cuda"), torch.as_tensor(x, device="cuda")).cpu().numpy()
    rows = np.repeat(np.arange(p.nb), np.diff(p.rowptr))
    ref = -lam.reshape(-1, 3)[rows][:, :, None] * x.reshape(-1, 3)[p.colind][:, None, :]
    assert np.array_equal(g, ref)


@pytest.mark.parametrize("precision,adjoint", [("fp64", "transpose"), ("mixed", "transpose"), ("fp64", "rebuild")])
def test_adjoint_matches_dense_adjoint(precision, adjoint):
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(CFG8)
    b = ncpgen.normals(p.n, 2)
    w = ncpgen.normals(p.n, 4, stream=4)
    xd, lamd, gd = oracle.dense_adjoint(p.rowptr, p.colind, p.values, b, w)
    vals = torch.as_tensor(p.values, device="cuda").requires_grad_(True)
    bt = torch.as_tensor(b, device="cuda").requires_grad_(True)
    rp = torch.as_tensor(p.rowptr, device="cuda")
    ci = torch.as_tensor(p.colind, device="cuda")
    mk = torch.as_tensor(p.cf_marker, device="cuda")
    opts = mg.options(precision=precision)
    x = mg.mgr_solve(vals, bt, rp, ci, mk, opts, rtol=1e-12, maxit=2000, adjoint=adjoint)
    loss = (x * torch.as_tensor(w, device="cuda")).sum()
    loss.backward()
    assert rel(x.detach().cpu().numpy(), xd) <= 1e-9
    assert rel(bt.grad.cpu().numpy(), lamd) <= 1e-9
    assert rel(vals.grad.cpu().numpy().ravel(), gd.ravel()) <= 1e-9


def test_adjoint_matches_finite_differences():
    """Central differences with a step 1e-6 relative to max(|a_ij|, max_k |a_ik|) (the entry, or its
    scalar row's largest magnitude when the entry is tiny: a step 1e-6 |a_ij| on an entry of 1e-6 is
    below the resolution of an FP64 solve), FD solves at rtol 1e-13: relative error <= 1e-5 on 32
    seeded nonzero entries (error relative to max(|g|, 1e-3 max|g|))."""
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(CFG8)
    b = ncpgen.normals(p.n, 2)
    w = torch.as_tensor(ncpgen.normals(p.n, 4, stream=4), device="cuda")
    A, mk = to_gpu(p)
    bt = torch.as_tensor(b, device="cuda")
    vals = A.values.clone().requires_grad_(True)
    x = mg.mgr_solve(vals, bt, A.rowptr, A.colind, mk, mg.options(), rtol=1e-13, maxit=3000)
    (x * w).sum().backward()
    g = vals.grad.cpu().numpy()
    gmax = np.abs(g).max()
    m = mg.MGR()

    def loss(v):
        Av = A.with_values(v)
        m.setup(Av, mk)
        xx, _ = m.fgmres(Av, bt, rtol=1e-13, maxit=3000)
        return float((xx * w).sum())

    rng = np.random.default_rng(5)
    flat = p.values.reshape(-1)
    rows = np.repeat(np.arange(p.nb), np.diff(p.rowptr))
    rowmax = np.zeros((p.nb, 3))
    np.maximum.at(rowmax, rows, np.abs(p.values).max(axis=2))
    scale = np.maximum(np.abs(p.values), rowmax[rows][:, :, None]).reshape(-1)
    cand = np.nonzero(flat != 0.0)[0]
    picks = rng.choice(cand, 32, replace=False)
    worst = 0.0
    for k in picks:
        h = 1e-6 * scale[k]
        vp = A.values.clone().reshape(-1)
        vm = A.values.clone().reshape(-1)
        vp[k] += h
        vm[k] -= h
        fd = (loss(vp.reshape(-1, 3, 3)) - loss(vm.reshape(-1, 3, 3))) / (2 * h)
        gk = g.reshape(-1)[k]
        err = abs(fd - gk) / max(abs(gk), 1e-3 * gmax)
        worst = max(worst, err)
    m.close()
    assert worst <= 1e-5, worst


@pytest.mark.parametrize("precision,frelax", [("fp64", [0, 1, 1]), ("mixed", [0, 1, 1]), ("fp64", [0, 2, 2])])
def test_transposed_preconditioner_is_the_transpose(precision, frelax):
    """mgr_apply_transpose is the transpose of mgr_apply's operator: the dense matrices of both, built
    column by column on a small 3-level problem with a multi-level AMG, agree to rounding."""
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.GridConfig(6, 5, 4, sigma=1.0, layer_contrast=1e-2, absent_frac=0.4, absent_mode=1,
                                              seed=4))
    A, mk = to_gpu(p)
    m = mg.MGR(precision=precision, adjoint=1, amg_max_coarse=8, restrict_type=[1, 1, 0], frelax_type=frelax,
               frelax_sweeps=[1, 2, 2])
    m.setup(A, mk)
    L, na = m.levels()
    assert L == 3 and na >= 3
    eye = torch.eye(p.n, dtype=torch.float64, device="cuda")
    M = torch.stack([m.apply(eye[k].contiguous()) for k in range(p.n)], dim=1)
    MT = torch.stack([m.apply_transpose(eye[k].contiguous()) for k in range(p.n)], dim=1)
    tol = 1e-12 if precision == "fp64" else 1e-5
    err = float(torch.linalg.norm(MT - M.T) / torch.linalg.norm(M))
    assert err <= tol, err
    m.close()


def test_transposed_preconditioner_bilinear_64cube():
    """<M^-T x, y> = <x, M^-1 y> on the 64^3 workload (FP64), where the operators of >= 256K rows run
    in the sliced layouts; and the transposed solve's explicit residual ||w - A^T lambda|| <= 1e-8 ||w||."""
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.WORKLOADS["ncp3d_64_adjoint"])
    A, mk = to_gpu(p)
    m = mg.MGR(precision="fp64", adjoint=1, amg_theta=0.5, amg_pmax=4, amg_smoother=0, amg_omega=0.8)
    m.setup(A, mk)
    xv = torch.as_tensor(ncpgen.normals(p.n, 7), device="cuda")
    yv = torch.as_tensor(ncpgen.normals(p.n, 8), device="cuda")
    lhs = float(torch.dot(m.apply_transpose(xv), yv))
    rhs = float(torch.dot(xv, m.apply(yv)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    w = torch.as_tensor(ncpgen.normals(p.n, 4, stream=4), device="cuda")
    lam, info = m.fgmres(A, w, rtol=1e-8, transpose=True)
    At = mg.bsr3_transpose(A)
    r = mg.bsr3_spmv(At, lam, sub=w)
    assert info["converged"] and float(torch.linalg.norm(r) / torch.linalg.norm(w)) <= 1e-8
    m.close()
