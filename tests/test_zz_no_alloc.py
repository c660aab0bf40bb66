"""The allocation-free block transpose (mgr_bsr3_transpose_noalloc) against the allocating one.

Some callers cannot let a library allocate device memory during a call: code that runs under a
memory budget or pool the caller owns, latency-critical code that cannot absorb an allocation, or a
host application that hands the library only buffers it manages itself.  For them the library keeps
the transpose's working memory in one fixed-size device array.  This file is collected last so that
a run stopping at its first failure has already run every other test; it passes alone in a fresh
process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import ncpgen
from gpu_common import to_gpu

pytestmark = pytest.mark.gpu


def _noalloc():
    import paper_1801_08464_gb300 as mg
    fn = mg.lib().mgr_bsr3_transpose_noalloc
    fn.argtypes = [ctypes.POINTER(mg.Bsr3), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_transpose_matches_allocating_transpose_on_two_calls():
    import paper_1801_08464_gb300 as mg
    import torch
    fn = _noalloc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row on different matrices: the second must not see the first call's contents
    for cfg in (ncpgen.GridConfig(9, 7, 5, absent_frac=0.4, absent_mode=1, seed=2),
                ncpgen.GridConfig(6, 4, 3, absent_frac=0.3, seed=5)):
        p = ncpgen.make_problem(cfg)
        A, _ = to_gpu(p)
        ref = mg.bsr3_transpose(A)
        rp = torch.full_like(A.rowptr, -7)
        ci = torch.full_like(A.colind, -7)
        v = torch.full_like(A.values, float("nan"))
        rc = fn(ctypes.byref(A.c()), rp.data_ptr(), ci.data_ptr(), v.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == 0, mg.STATUS.get(rc, rc)
        # index work: bit-exact; values are copied, so bit-exact as well
        assert torch.equal(rp, ref.rowptr) and torch.equal(ci, ref.colind) and torch.equal(v, ref.values)
        import scipy.sparse as sp
        T = sp.bsr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(p.n, p.n)).toarray()
        assert np.array_equal(T, p.to_scipy().toarray().T)


def test_noalloc_transpose_rejects_sizes_beyond_its_array():
    import paper_1801_08464_gb300 as mg
    fn = _noalloc()
    too_many_rows = mg.Bsr3((1 << 16) + 1, (1 << 16) + 1, 1, 1, 1)  # rejected before any pointer is used
    assert fn(ctypes.byref(too_many_rows), 1, 1, 1, None) == 9  # MGR_ERR_UNSUPPORTED


def test_noalloc_transpose_rejects_blocks_beyond_its_array():
    import paper_1801_08464_gb300 as mg
    fn = _noalloc()
    too_many_blocks = mg.Bsr3(8, (1 << 19) + 1, 1, 1, 1)  # rejected on the host before any pointer is used
    assert fn(ctypes.byref(too_many_blocks), 1, 1, 1, None) == 9  # MGR_ERR_UNSUPPORTED


def test_noalloc_transpose_reports_malformed_input_and_still_works_after():
    """A column outside [0, nb) or row pointers that do not run 0..nnzb are found on the device,
    reported as MGR_ERR_INVALID_ARG, and nothing is written through them; the next well-formed call
    gives the right transpose."""
    import paper_1801_08464_gb300 as mg
    import torch
    fn = _noalloc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = ncpgen.make_problem(ncpgen.GridConfig(7, 5, 4, absent_frac=0.4, absent_mode=1, seed=4))
    A, _ = to_gpu(p)
    ref = mg.bsr3_transpose(A)

    def run(rowptr, colind):
        B = mg.Bsr3(A.nb, A.nnzb, rowptr.data_ptr(), colind.data_ptr(), A.values.data_ptr())
        rp = torch.full_like(A.rowptr, -7)
        ci = torch.full_like(A.colind, -7)
        v = torch.full_like(A.values, float("nan"))
        rc = fn(ctypes.byref(B), rp.data_ptr(), ci.data_ptr(), v.data_ptr(), stream)
        torch.cuda.synchronize()
        return rc, rp, ci, v

    bad_col = A.colind.clone()
    bad_col[A.nnzb // 2] = A.nb  # one past the last block column
    neg_col = A.colind.clone()
    neg_col[3] = -1
    long_rows = A.rowptr.clone()
    long_rows[-1] = A.nnzb + 5  # the last row would run past the stored blocks
    falling = A.rowptr.clone()
    falling[A.nb // 2] = falling[A.nb // 2 + 1] + 1
    for rowptr, colind in ((A.rowptr, bad_col), (A.rowptr, neg_col), (long_rows, A.colind), (falling, A.colind)):
        rc, _, ci, v = run(rowptr, colind)
        assert rc == 1, mg.STATUS.get(rc, rc)  # MGR_ERR_INVALID_ARG
        assert bool((ci == -7).all()) and bool(torch.isnan(v).all())  # nothing scattered or copied
    rc, rp, ci, v = run(A.rowptr, A.colind)
    assert rc == 0 and torch.equal(rp, ref.rowptr) and torch.equal(ci, ref.colind) and torch.equal(v, ref.values)
