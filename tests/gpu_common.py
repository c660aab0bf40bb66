"""Shared helpers of the GPU parity tests: build the same seeded problem for the GPU library (through
the C ABI) and for the CPU oracle, and compare hierarchies."""
import numpy as np

import ncpgen

# Parity workloads: the 32x32 plain workload itself, a 16^3 slice of the 3-D workloads and a ragged
# layered grid (all sizes several tiles, with ragged tails).
PARITY = {
    "ncp2d_32x32": ncpgen.WORKLOADS["ncp2d_32x32"],
    "ncp3d_16": ncpgen.GridConfig(16, 16, 16, sigma=2.0, absent_frac=0.5, absent_mode=1, seed=1),
    "ragged_13x7x9": ncpgen.GridConfig(13, 7, 9, sigma=1.0, layer_contrast=1e-4, absent_frac=0.4, absent_mode=1,
                                       seed=3),
    # the two-level unsaturated case of section 6.1 (Van Genuchten closures, gas present everywhere)
    "unsat2d_200x10": ncpgen.WORKLOADS["unsat2d_200x10"],
}

# Section 6.1's two-level setting: injective R (W_r = 0) at both reductions, three relaxation sweeps
# on the saturation block (l1-Jacobi in place of the paper's Gauss-Seidel), V(2,2) on the pressure.
UNSAT = dict(restrict_type=[0, 0], frelax_type=[1, 1], frelax_sweeps=[1, 3], amg_pre=2, amg_post=2)


def to_gpu(p):
    import torch

    import paper_1801_08464_gb300 as mg
    A = mg.BSR3.from_numpy(p.rowptr, p.colind, p.values)
    mk = torch.as_tensor(p.cf_marker, device="cuda")
    return A, mk


def compare_csr(g, o, rtol=1e-13, what=""):
    """Pattern bit-exact, values within rtol of the largest magnitude; returns the fraction of
    values that agree bit for bit."""
    g = g.tocsr(); o = o.tocsr()
    assert g.shape == o.shape, (what, g.shape, o.shape)
    assert np.array_equal(g.indptr, o.indptr), f"{what}: row pointers differ"
    assert np.array_equal(g.indices, o.indices), f"{what}: columns differ"
    if o.nnz == 0:
        return 1.0
    scale = max(np.abs(o.data).max(), 1e-300)
    d = np.abs(g.data - o.data).max()
    assert d <= rtol * scale, f"{what}: max |diff| {d:.3e} vs scale {scale:.3e}"
    return float(np.mean(g.data == o.data))


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def compare_hierarchy(m, o, binv=True):
    """Every setup object of a GPU hierarchy against the oracle's: level operators, W_p, W_r, P, R,
    F/C splits and relaxation scalings of every MGR level; PMIS splits, strength graphs, P, R, A and
    smoother scalings of every AMG level; the 3x3 block inverses.  Splittings and patterns bit for
    bit; returns the smallest fraction of bit-identical values over the operators."""
    import paper_1801_08464_gb300 as mg
    import oracle
    L, na = m.levels()
    assert (L, na) == o.info()
    same = []
    for l in range(L + 1):
        same.append(compare_csr(m.scipy(mg.MAT_LEVEL, l), o.scipy(oracle.MAT_LEVEL, l), what=f"A_{l}"))
    for l in range(L):
        for kind in (mg.MAT_WP, mg.MAT_WR, mg.MAT_P, mg.MAT_R):
            same.append(compare_csr(m.scipy(kind, l), o.scipy(kind, l), what=f"kind{kind} level {l}"))
        for kind in (mg.VEC_F, mg.VEC_C):
            assert np.array_equal(m.vector(kind, l).cpu().numpy(), o.vec(kind, l)), f"F/C split of level {l}"
        np.testing.assert_allclose(m.vector(mg.VEC_MINV, l).cpu().numpy(), o.vec(oracle.VEC_MINV, l), rtol=1e-14)
    for k in range(na):
        same.append(compare_csr(m.scipy(mg.MAT_AMG_A, k), o.scipy(oracle.MAT_AMG_A, k), what=f"AMG A_{k}"))
        if k < na - 1:
            assert np.array_equal(m.vector(mg.VEC_AMG_CF, k).cpu().numpy(), o.vec(oracle.VEC_AMG_CF, k)), \
                f"PMIS split of AMG level {k}"
            for kind in (mg.MAT_AMG_P, mg.MAT_AMG_R, mg.MAT_AMG_S):
                same.append(compare_csr(m.scipy(kind, k), o.scipy(kind, k), what=f"AMG kind{kind} level {k}"))
            np.testing.assert_allclose(m.vector(mg.VEC_AMG_DINV, k).cpu().numpy(), o.vec(oracle.VEC_AMG_DINV, k),
                                       rtol=1e-14)
    if binv:
        ob = o.vec(oracle.VEC_BINV, 0)
        np.testing.assert_allclose(m.vector(mg.VEC_BINV, 0).cpu().numpy(), ob, rtol=1e-13,
                                   atol=1e-13 * np.abs(ob).max())
    return min(same)
