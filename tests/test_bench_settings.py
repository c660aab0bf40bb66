"""The benchmark's solver settings (bench.py's SOLVER for the 3-D workloads, UNSAT_SOLVER for the
two-level unsaturated ones) are options that both the library and the oracle accept, and the
oracle's MGR-FGMRES reaches the benchmark's tolerance with them on small instances of the same
recipes (no GPU: the library is only asked for its option defaults)."""
import dataclasses
import importlib.util
import os

import numpy as np
import pytest

import ncpgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_settings", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)  # module level: constants only, no GPU work
    return mod


@pytest.mark.parametrize("which", ["SOLVER", "UNSAT_SOLVER"])
def test_settings_are_library_options(which):
    import paper_1801_08464_gb300 as mg
    opts = getattr(_bench(), which)
    o = mg.options(**opts)
    for k, v in opts.items():
        got = getattr(o, k)
        if isinstance(v, (list, tuple)):
            assert [got[i] for i in range(len(v))] == list(v), k
        else:
            assert got == pytest.approx(v), k


@pytest.mark.parametrize("which,cfg", [
    ("SOLVER", dataclasses.replace(ncpgen.WORKLOADS["ncp3d_128_layered"], nx=12, ny=10, nz=8)),
    ("UNSAT_SOLVER", ncpgen.WORKLOADS["unsat2d_200x10"]),
])
def test_oracle_converges_with_the_settings(which, cfg):
    b_mod = _bench()
    opts = getattr(b_mod, which)
    p = ncpgen.make_problem(cfg)
    o = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, **opts)
    b = ncpgen.normals(p.n, 2)
    x, info = o.fgmres(b, rtol=b_mod.RTOL, restart=b_mod.RESTART, maxit=b_mod.MAXIT)
    assert info["converged"]
    assert np.linalg.norm(b - p.to_scipy() @ x) <= b_mod.RTOL * np.linalg.norm(b)
