"""Full-size workloads on the GPU.

64^3 (786,432 unknowns, FP64, AMG coarse solve): the whole hierarchy against the oracle, splittings
and patterns bit for bit, one preconditioner application against the oracle's, and the solve to
1e-8.
128^3 (6,291,456 unknowns, the benchmark's workload and solver settings): the whole FP64 hierarchy
against the oracle's (splittings, patterns and values bit for bit, every MGR and AMG level), one
FP64 preconditioner application against the oracle's; then the benchmark's configuration (FP32
hierarchy, FP64 Krylov) against the oracle's FP64 solve: residual, iteration count and solution
error; and properties that hold at any size -- level sizes 3N-M, 2N-M, N, the level-1 operator on
sampled rows against its closed form A_cc - A_cf C33^-1 A_fc.
"""
import numpy as np
import pytest

import ncpgen
import oracle
from gpu_common import compare_csr, compare_hierarchy, rel, to_gpu

pytestmark = pytest.mark.gpu

BENCH_SOLVER = dict(amg_theta=0.58, amg_pmax=4, amg_smoother=0, amg_omega=0.8, amg_max_coarse=64,
                    frelax_sweeps=[1, 1, 1])


def test_64cube_full_parity_fp64():
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.WORKLOADS["ncp3d_64"])
    A, mk = to_gpu(p)
    m = mg.MGR(**BENCH_SOLVER)
    m.setup(A, mk)
    o = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, **BENCH_SOLVER)
    L, na = m.levels()
    assert (L, na) == o.info()
    for l in range(L + 1):
        compare_csr(m.scipy(mg.MAT_LEVEL, l), o.scipy(oracle.MAT_LEVEL, l), what=f"A_{l}")
    for l in range(L):
        for kind in (mg.VEC_F, mg.VEC_C):
            assert np.array_equal(m.vector(kind, l).cpu().numpy(), o.vec(kind, l))
    for k in range(na - 1):
        assert np.array_equal(m.vector(mg.VEC_AMG_CF, k).cpu().numpy(), o.vec(oracle.VEC_AMG_CF, k))
        compare_csr(m.scipy(mg.MAT_AMG_P, k), o.scipy(oracle.MAT_AMG_P, k), what=f"AMG P_{k}")
        compare_csr(m.scipy(mg.MAT_AMG_A, k + 1), o.scipy(oracle.MAT_AMG_A, k + 1), what=f"AMG A_{k+1}")
    b = ncpgen.normals(p.n, 2)
    # one preconditioner application (operators of >= 256K rows run in the sliced layouts here)
    z = m.apply(torch.as_tensor(b, device="cuda")).cpu().numpy()
    zo = o.apply(b)
    assert np.linalg.norm(z - zo) <= 1e-9 * np.linalg.norm(zo)
    x, info = m.fgmres(A, torch.as_tensor(b, device="cuda"), rtol=1e-8)
    assert info["converged"]
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - p.to_scipy() @ xg) <= 1e-8 * np.linalg.norm(b)
    m.close()


def test_128cube_mixed_properties():
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.WORKLOADS["ncp3d_128_layered"])
    A, mk = to_gpu(p)
    m = mg.MGR(precision="mixed", **BENCH_SOLVER)
    m.setup(A, mk)
    # every index the apply gathers with is in range, in the sliced layouts of the benchmark's hierarchy
    assert m.audit() == 0
    N, M = p.nb, int(p.gas_present.sum())
    sizes = [m.matrix(mg.MAT_LEVEL, l)[3][0] for l in range(4)]
    assert sizes == [3 * N, 3 * N - M, 2 * N - M, N]
    # level-1 operator on sampled rows: S1 = A_cc - A_cf C33^-1 A_fc (exact: C33 diagonal)
    S1 = m.scipy(mg.MAT_LEVEL, 1)
    Asp = p.to_scipy().tocsr()
    F = np.nonzero(p.cf_marker == 0)[0]
    C = np.nonzero(p.cf_marker > 0)[0]
    d = Asp.diagonal()[F]
    rng = np.random.default_rng(0)
    rows = rng.choice(len(C), 400, replace=False)
    Acf = Asp[C[rows]][:, F]
    Afc = Asp[F]
    ref = (Asp[C[rows]][:, C] - Acf @ (Afc[:, C].multiply(1.0 / d[:, None]))).toarray()
    got = S1[rows].toarray()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    b = ncpgen.normals(p.n, 2)
    x, info = m.fgmres(A, torch.as_tensor(b, device="cuda"), rtol=1e-8)
    assert info["converged"]
    res = np.linalg.norm(b - Asp @ x.cpu().numpy()) / np.linalg.norm(b)
    assert res <= 1e-8
    print(f"128^3 mixed: {info['iterations']} iterations, relres {res:.3e}, setup {m.stats()['setup_ms']:.1f} ms, "
          f"solve {info['solve_ms']:.1f} ms, memory {m.memory_bytes() / 1e9:.2f} GB")
    m.close()


def test_128cube_full_parity_and_mixed_against_oracle():
    """The benchmark's workload at full size against the oracle.  Size-dependent paths of the GPU
    setup run only here (split-row sliced kernels, multi-batch SpGEMM staging)."""
    import paper_1801_08464_gb300 as mg
    import torch
    p = ncpgen.make_problem(ncpgen.WORKLOADS["ncp3d_128_layered"])
    A, mk = to_gpu(p)
    o = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, **BENCH_SOLVER)
    m = mg.MGR(**BENCH_SOLVER)  # FP64 hierarchy
    m.setup(A, mk)
    assert compare_hierarchy(m, o) == 1.0, "setup values are computed by the same IEEE operations as the oracle's"
    b = ncpgen.normals(p.n, 2)
    bt = torch.as_tensor(b, device="cuda")
    z = m.apply(bt).cpu().numpy()
    zo = o.apply(b)
    err_apply = rel(z, zo)
    assert err_apply <= 1e-9, err_apply
    x64, info64 = m.fgmres(A, bt, rtol=1e-8)
    x64 = x64.cpu().numpy()
    m.close()
    mm = mg.MGR(precision="mixed", **BENCH_SOLVER)
    mm.setup(A, mk)
    xm, infom = mm.fgmres(A, bt, rtol=1e-8)
    xm = xm.cpu().numpy()
    mm.close()
    xo, io = o.fgmres(b, rtol=1e-8)
    Asp = p.to_scipy().tocsr()
    nb = np.linalg.norm(b)
    res = {k: np.linalg.norm(b - Asp @ x) / nb for k, x in (("fp64", x64), ("mixed", xm), ("oracle", xo))}
    err = {"fp64": rel(x64, xo), "mixed": rel(xm, xo)}
    print(f"128^3: apply rel. diff {err_apply:.2e}; iterations oracle {io['iterations']} fp64 "
          f"{info64['iterations']} mixed {infom['iterations']}; residuals {res}; rel. error vs the FP64 "
          f"oracle solution: {err}")
    assert infom["converged"] and info64["converged"] and io["converged"]
    assert max(res.values()) <= 1e-8
    assert infom["iterations"] <= 1.2 * io["iterations"]
    assert abs(info64["iterations"] - io["iterations"]) <= 1
    # Both solves follow the same Krylov iteration to within the hierarchy's rounding, so their
    # residual vectors agree to about 1e-6 of their 1e-8 size and the solutions far closer than the
    # tolerance alone would force (measured on a GB300: 3.3e-16 FP64, 1.3e-15 mixed)
    assert err["fp64"] <= 1e-10 and err["mixed"] <= 1e-10, err
