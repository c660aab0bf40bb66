"""The adjoint workloads at full size on the GPU.

64^3 adjoint (786,432 unknowns, FP32 hierarchy / FP64 Krylov): the gradient of L = w . x with respect
to the BSR values, from the MGR-preconditioned A^T solve, against central finite differences of
forward solves on 32 seeded stored entries.

256^3 forward + adjoint (50,331,648 unknowns, 1.05e9 stored scalar entries, FP32 hierarchy / FP64
Krylov, sigma 2 with a 1e-6 layered contrast, half the cells gas-absent): one forward and one adjoint
solve to 1e-8 through the autograd function, each checked by its explicit residual; the gradient on
sampled entries equals -lambda_i x_j; the device footprint (the tensors plus the hierarchy with its
transposed operators and work buffers) stays below 180 GB.  This recipe needs the non-injective
restriction at the second reduction (restrict_type [1, 1, 0]) and the l1-Jacobi AMG smoother; the
lean setup keeps the footprint down.
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


SCALE_SOLVER = dict(precision="mixed", amg_theta=0.5, amg_pmax=4, amg_smoother=1, restrict_type=[1, 1, 0], lean=1)


def test_256cube_forward_and_adjoint():
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.WORKLOADS["ncp3d_256_layered"])
    assert p.n == 50_331_648 and 9 * p.nnzb == 1_053_425_664
    torch.cuda.reset_peak_memory_stats()
    A, mk = to_gpu(p)
    b = torch.as_tensor(ncpgen.normals(p.n, 2), device="cuda")
    w = torch.as_tensor(ncpgen.normals(p.n, 4, stream=4), device="cuda")
    del p
    vals = A.values.requires_grad_(True)
    bt = b.clone().requires_grad_(True)
    stats = {}
    x = mg.mgr_solve(vals, bt, A.rowptr, A.colind, mk, mg.options(**SCALE_SOLVER), rtol=1e-8, maxit=3000,
                     stats=stats)
    (x * w).sum().backward()
    fw, ad = stats["forward"], stats["adjoint"]
    assert fw["converged"] and ad["converged"]
    xd = x.detach()
    Ad = mg.BSR3(A.rowptr, A.colind, vals.detach())
    r = mg.bsr3_spmv(Ad, xd, sub=b)
    relres = float(torch.linalg.norm(r) / torch.linalg.norm(b))
    assert relres <= 1e-8
    del r
    lam = bt.grad.detach()
    At = mg.bsr3_transpose(Ad)
    r = mg.bsr3_spmv(At, lam, sub=w)
    relres_adj = float(torch.linalg.norm(r) / torch.linalg.norm(w))
    assert relres_adj <= 1e-8
    del r, At
    # dL/dA_ij = -lambda_i x_j on sampled stored entries (block k, entry (p, q))
    rng = np.random.default_rng(7)
    ks = torch.as_tensor(rng.integers(0, Ad.nnzb, 4096), device="cuda")
    rows = torch.searchsorted(A.rowptr, ks, right=True) - 1
    cols = A.colind[ks].long()
    ref = -lam.reshape(-1, 3)[rows][:, :, None] * xd.reshape(-1, 3)[cols][:, None, :]
    assert torch.equal(vals.grad[ks], ref)
    torch_peak = torch.cuda.max_memory_allocated()
    lib_peak = max(fw["memory_peak_bytes"], ad["memory_peak_bytes"])
    total = torch_peak + lib_peak
    print(f"256^3: forward {fw['iterations']} it, setup {fw['setup_ms']:.0f} ms, solve {fw['solve_ms']:.0f} ms, "
          f"relres {relres:.2e}; adjoint {ad['iterations']} it, solve {ad['solve_ms']:.0f} ms, relres "
          f"{relres_adj:.2e}; device peak: tensors {torch_peak / 1e9:.1f} GB + hierarchy {lib_peak / 1e9:.1f} GB = "
          f"{total / 1e9:.1f} GB")
    assert total <= 180e9
