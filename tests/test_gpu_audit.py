"""Index audit of set-up hierarchies (mgr_audit): every column index the apply and the Krylov
products gather with, recomputed on the device from its stored form, lies within its operator, and
offsets, row pointers, permutations and the F/C/map lists are in order.  It stands in for a memory
checker on the apply's gathers.  Small cases exercise the CSR forms; 64^3 (level operators of more
than 256K rows) the sliced forms: 32-bit columns, 16-bit offsets from a slice base and one-byte
offset codes; the 128^3 benchmark hierarchy is audited in test_gpu_fullsize."""
import pytest

import ncpgen
from gpu_common import PARITY, UNSAT, to_gpu

pytestmark = pytest.mark.gpu

PAPER_62 = dict(frelax_type=[0, 2, 2], frelax_sweeps=[1, 1, 1], restrict_type=[1, 1, 1], amg_pre=2, amg_post=2,
                amg_max_coarse=16)


@pytest.mark.parametrize("name", list(PARITY))
@pytest.mark.parametrize("opts", [{}, dict(adjoint=1), PAPER_62, dict(precision="fp64", adjoint=1)],
                         ids=["default", "adjoint", "paper_62", "fp64_adjoint"])
def test_audit_small(name, opts):
    import paper_1801_08464_gb300 as mg
    if name.startswith("unsat") and "frelax_type" not in opts:
        opts = {**UNSAT, **opts}  # section 6.1's two-level setting
    p = ncpgen.make_problem(PARITY[name])
    A, mk = to_gpu(p)
    m = mg.MGR(**opts)
    m.setup(A, mk)
    assert m.audit() == 0
    m.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_audit_sliced_64cube(precision):
    import paper_1801_08464_gb300 as mg
    p = ncpgen.make_problem(ncpgen.WORKLOADS["ncp3d_64"])
    A, mk = to_gpu(p)
    m = mg.MGR(precision=precision, adjoint=1)
    m.setup(A, mk)
    assert m.audit() == 0
    m.close()


def test_audit_before_setup_is_a_state_error():
    import paper_1801_08464_gb300 as mg
    m = mg.MGR()
    with pytest.raises(mg.MgrError):
        m.audit()
    m.close()
