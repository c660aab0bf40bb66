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
