"""Full-size workloads on the GPU.

64^3 (786,432 unknowns, FP64, AMG coarse solve): the whole hierarchy against the oracle, splittings
and patterns bit for bit, one preconditioner application against the oracle's, and the solve to
1e-8.
128^3 (6,291,456 unknowns, FP32 hierarchy / FP64 Krylov, the benchmark's launch configuration):
properties that hold at any size -- level sizes 3N-M, 2N-M, N, the level-1 operator on sampled rows
against its closed form A_cc - A_cf C33^-1 A_fc, the explicit residual of the returned solution.
"""
import numpy as np
import pytest

import ncpgen
import oracle
from gpu_common import compare_csr, to_gpu

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
