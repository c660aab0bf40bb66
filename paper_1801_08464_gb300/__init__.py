"""MGR-preconditioned flexible GMRES for 3x3-block NCP Jacobians on GB300 (sm_103a).

Thin Python binding of the C ABI in ``include/mgr.h`` (library ``_lib/libmgrgpu.so``): arguments are
marshalled to device pointers of torch CUDA tensors and the current torch stream; every step of the
method runs in the library's CUDA kernels.  There is no CPU path: importing works without a GPU,
but any call raises if the compiled library or a CUDA device is missing.

Method: Bui, Wang & Osei-Kuffuor, "Algebraic multigrid preconditioners for multiphase flow in porous
media with phase transitions" -- the presmoothing MGR Algorithm (section 4) with the three-level
reduction order of section 5, an AMG V-cycle on the pressure system, GMRES outside (section 6).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "libmgrgpu.so")
MAX_LEVELS = 8
_lib = None

STATUS = {0: "MGR_OK", 1: "MGR_ERR_INVALID_ARG", 2: "MGR_ERR_SINGULAR", 3: "MGR_ERR_NOT_CONVERGED",
          4: "MGR_ERR_BREAKDOWN", 5: "MGR_ERR_OOM", 6: "MGR_ERR_CUDA", 7: "MGR_ERR_TIMEOUT", 8: "MGR_ERR_STATE",
          9: "MGR_ERR_UNSUPPORTED"}
PREC_FP64, PREC_MIXED = 0, 1
# introspection kinds (include/mgr.h)
MAT_LEVEL, MAT_WP, MAT_WR, MAT_P, MAT_R, MAT_AMG_A, MAT_AMG_P, MAT_AMG_R, MAT_AMG_S = range(9)
VEC_MINV, VEC_AMG_DINV, VEC_BINV, VEC_F, VEC_C, VEC_AMG_CF = range(6)


class MgrError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("global_relax", ctypes.c_int32),
                ("frelax_type", ctypes.c_int32 * MAX_LEVELS), ("frelax_sweeps", ctypes.c_int32 * MAX_LEVELS),
                ("frelax_omega", ctypes.c_double * MAX_LEVELS), ("restrict_type", ctypes.c_int32 * MAX_LEVELS),
                ("apply_full_R", ctypes.c_int32), ("coarse_solver", ctypes.c_int32), ("amg_theta", ctypes.c_double),
                ("amg_max_levels", ctypes.c_int32), ("amg_max_coarse", ctypes.c_int32),
                ("amg_smoother", ctypes.c_int32), ("amg_pre", ctypes.c_int32), ("amg_post", ctypes.c_int32),
                ("amg_pmax", ctypes.c_int32), ("amg_omega", ctypes.c_double), ("amg_seed", ctypes.c_uint64),
                ("lean", ctypes.c_int32), ("spgemm_stage", ctypes.c_int32),
                ("adjoint", ctypes.c_int32), ("apply_graph", ctypes.c_int32), ("pdl", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class Bsr3(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int64), ("nnzb", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colind", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("relres_true", ctypes.c_double), ("relres_est", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_cap", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


EXPORTS = ["mgr_status_string", "mgr_options_default", "mgr_create", "mgr_setup", "mgr_apply", "fgmres_solve",
           "mgr_apply_transpose", "fgmres_solve_transpose",
           "mgr_destroy", "mgr_get_levels", "mgr_matrix_shape", "mgr_copy_matrix", "mgr_vector_len",
           "mgr_copy_vector", "mgr_memory_bytes", "mgr_memory_peak_bytes", "mgr_get_stats", "mgr_get_host_waits", "mgr_audit", "mgr_bsr3_spmv", "mgr_bsr3_transpose",
           "mgr_bsr3_outer_grad", "mgr_profile", "mgr_profile_select", "mgr_kernel_time",
           "mgr_kernel_bytes", "mgr_kernel_bytes_stored", "mgr_probe_fp64_fma"]


def lib():
    """Load the compiled library (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"CUDA library not built ({LIBPATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIBPATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        P = ctypes.POINTER
        L.mgr_status_string.restype = ctypes.c_char_p
        L.mgr_status_string.argtypes = [i32]
        L.mgr_options_default.argtypes = [P(Options)]
        L.mgr_options_default.restype = None
        L.mgr_create.argtypes = [P(vp), P(Options), vp]
        L.mgr_setup.argtypes = [vp, P(Bsr3), vp]
        L.mgr_apply.argtypes = [vp, vp, vp]
        L.fgmres_solve.argtypes = [vp, P(Bsr3), vp, vp, ctypes.c_double, i32, i32, P(SolveInfo)]
        L.mgr_apply_transpose.argtypes = [vp, vp, vp]
        L.fgmres_solve_transpose.argtypes = [vp, P(Bsr3), vp, vp, ctypes.c_double, i32, i32, P(SolveInfo)]
        L.mgr_destroy.argtypes = [vp]
        L.mgr_get_levels.argtypes = [vp, P(i32), P(i32)]
        L.mgr_matrix_shape.argtypes = [vp, i32, i32, P(i64), P(i64), P(i64)]
        L.mgr_copy_matrix.argtypes = [vp, i32, i32, vp, vp, vp]
        L.mgr_vector_len.argtypes = [vp, i32, i32, P(i64)]
        L.mgr_copy_vector.argtypes = [vp, i32, i32, vp]
        L.mgr_memory_bytes.argtypes = [vp, P(i64)]
        L.mgr_memory_peak_bytes.argtypes = [vp, P(i64)]
        L.mgr_get_stats.argtypes = [vp, P(ctypes.c_double), P(i64), P(i64), P(i64)]
        L.mgr_get_host_waits.argtypes = [P(i64)]
        L.mgr_audit.argtypes = [vp, P(i64)]
        L.mgr_bsr3_spmv.argtypes = [P(Bsr3), vp, vp, vp, vp]
        L.mgr_bsr3_transpose.argtypes = [P(Bsr3), vp, vp, vp, vp]
        L.mgr_bsr3_outer_grad.argtypes = [P(Bsr3), vp, vp, vp, vp]
        L.mgr_profile.argtypes = [vp, i32]
        L.mgr_kernel_time.argtypes = [vp, ctypes.c_char_p, P(i64), P(ctypes.c_double)]
        L.mgr_kernel_bytes.argtypes = [vp, ctypes.c_char_p, P(ctypes.c_double)]
        L.mgr_kernel_bytes_stored.argtypes = [vp, ctypes.c_char_p, P(ctypes.c_double)]
        L.mgr_profile_select.argtypes = [vp, ctypes.c_char_p]
        L.mgr_probe_fp64_fma.argtypes = [i64, i32, vp, P(ctypes.c_double), P(ctypes.c_double)]
        for name in EXPORTS:
            getattr(L, name).restype = ctypes.c_int if name not in ("mgr_status_string", "mgr_options_default") \
                else getattr(L, name).restype
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise MgrError(rc, what)


def options(**kw) -> Options:
    """Library defaults (mgr_options_default) with keyword overrides; per-level lists are padded with
    their last entry.  precision may be 'fp64' / 'mixed'."""
    o = Options()
    lib().mgr_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[v]
        if k == "ideal":
            if v:
                raise ValueError("the ideal (dense exact) mode exists only in the CPU oracle")
            continue
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        if isinstance(v, (list, tuple)):
            arr = getattr(o, k)
            for i in range(MAX_LEVELS):
                arr[i] = v[i] if i < len(v) else v[-1]
        else:
            setattr(o, k, v)
    return o


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@dataclass
class BSR3:
    """3x3 block-CSR matrix on the GPU: rowptr int64 [nb+1], colind int32 [nnzb],
    values float64 [nnzb, 3, 3] (entry (p, q) of block k is A(3I+p, 3J+q))."""
    rowptr: "object"
    colind: "object"
    values: "object"

    @property
    def nb(self) -> int:
        return int(self.rowptr.shape[0]) - 1

    @property
    def nnzb(self) -> int:
        return int(self.colind.shape[0])

    @property
    def n(self) -> int:
        return 3 * self.nb

    def c(self) -> Bsr3:
        return Bsr3(self.nb, self.nnzb, self.rowptr.data_ptr(), self.colind.data_ptr(), self.values.data_ptr())

    @staticmethod
    def from_numpy(rowptr, colind, values, device="cuda"):
        import torch
        return BSR3(torch.as_tensor(rowptr, dtype=torch.int64, device=device).contiguous(),
                    torch.as_tensor(colind, dtype=torch.int32, device=device).contiguous(),
                    torch.as_tensor(values, dtype=torch.float64, device=device).reshape(-1, 3, 3).contiguous())

    def with_values(self, values) -> "BSR3":
        return BSR3(self.rowptr, self.colind, values.reshape(-1, 3, 3).contiguous())


class MGR:
    """An MGR hierarchy (mgr_create / mgr_setup / mgr_apply / fgmres_solve / mgr_destroy)."""

    def __init__(self, opts: Options | None = None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: this library has no CPU path")
        self._h = ctypes.c_void_p()
        o = opts if opts is not None else options(**kw)
        self.opts = o
        _check(lib().mgr_create(ctypes.byref(self._h), ctypes.byref(o), _stream()), "mgr_create")
        self.A = None

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mgr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, A: BSR3, cf_marker):
        import torch
        assert cf_marker.dtype == torch.int8 and cf_marker.is_cuda
        self.A = A
        _check(lib().mgr_setup(self._h, ctypes.byref(A.c()), _ptr(cf_marker.contiguous())), "mgr_setup")
        return self

    def apply(self, r, z=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        _check(lib().mgr_apply(self._h, _ptr(r), _ptr(z)), "mgr_apply")
        return z

    def apply_transpose(self, r, z=None):
        """z = M^-T r (needs options adjoint=1 at setup)."""
        import torch
        if z is None:
            z = torch.empty_like(r)
        _check(lib().mgr_apply_transpose(self._h, _ptr(r), _ptr(z)), "mgr_apply_transpose")
        return z

    def fgmres(self, A: BSR3, b, x=None, rtol=1e-8, restart=30, maxit=1000, history=False, raise_on_fail=True,
               transpose=False):
        """Solve A x = b by FGMRES(restart) right-preconditioned with M^-1, or, with transpose=True on a
        handle set up with adjoint=1, A^T x = b by GMRES(restart) left-preconditioned with M^-T; x is
        the initial guess and the output."""
        import numpy as np
        import torch
        if x is None:
            x = torch.zeros_like(b)
        info = SolveInfo()
        hist = None
        if history:
            hist = np.zeros(maxit + 2)
            info.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            info.history_cap = maxit + 2
        fn = lib().fgmres_solve_transpose if transpose else lib().fgmres_solve
        rc = fn(self._h, ctypes.byref(A.c()), _ptr(b), _ptr(x), rtol, restart, maxit, ctypes.byref(info))
        out = dict(status=rc, iterations=info.iterations, restarts=info.restarts, converged=bool(info.converged),
                   relres_true=info.relres_true, relres_est=info.relres_est, bnorm=info.bnorm,
                   solve_ms=info.solve_ms)
        if history:
            out["history"] = hist[: info.iterations + 1].copy()
        if raise_on_fail and rc not in (0,):
            raise MgrError(rc, "fgmres_solve_transpose" if transpose else "fgmres_solve")
        return x, out

    def audit(self) -> int:
        """Number of out-of-range indices and out-of-order offsets in the hierarchy's apply operators
        (0 for a sound setup); see mgr_audit."""
        t = ctypes.c_int64()
        _check(lib().mgr_audit(self._h, ctypes.byref(t)), "mgr_audit")
        return t.value

    def levels(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().mgr_get_levels(self._h, ctypes.byref(a), ctypes.byref(b)), "mgr_get_levels")
        return a.value, b.value

    def matrix(self, kind: int, level: int):
        """(rowptr, col, val, shape) as torch CUDA tensors (FP64 setup copy)."""
        import torch
        nr, nc, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mgr_matrix_shape(self._h, kind, level, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz)),
               f"mgr_matrix_shape({kind},{level})")
        rp = torch.empty(nr.value + 1, dtype=torch.int64, device="cuda")
        ci = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
        v = torch.empty(max(nnz.value, 1), dtype=torch.float64, device="cuda")
        _check(lib().mgr_copy_matrix(self._h, kind, level, _ptr(rp), _ptr(ci), _ptr(v)), "mgr_copy_matrix")
        return rp, ci[: nnz.value], v[: nnz.value], (nr.value, nc.value)

    def scipy(self, kind: int, level: int):
        import scipy.sparse as sp
        rp, ci, v, shape = self.matrix(kind, level)
        return sp.csr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=shape)

    def vector(self, kind: int, level: int):
        import torch
        n = ctypes.c_int64()
        _check(lib().mgr_vector_len(self._h, kind, level, ctypes.byref(n)), f"mgr_vector_len({kind},{level})")
        out = torch.empty(max(n.value, 1), dtype=torch.float64, device="cuda")
        _check(lib().mgr_copy_vector(self._h, kind, level, _ptr(out)), "mgr_copy_vector")
        return out[: n.value]

    def profile(self, enable: bool = True, only=None):
        """Start (clearing totals) or stop CUDA-event timing of the library's named kernels; `only`
        restricts the recording to the given names."""
        if enable:
            sel = ",".join(only) if only else None
            _check(lib().mgr_profile_select(self._h, sel.encode() if sel else None), "mgr_profile_select")
        _check(lib().mgr_profile(self._h, 1 if enable else 0), "mgr_profile")

    def kernel_time(self, name: str):
        """(launches, total device ms) recorded for a named kernel since profile(True)."""
        n, ms = ctypes.c_int64(), ctypes.c_double()
        _check(lib().mgr_kernel_time(self._h, name.encode(), ctypes.byref(n), ctypes.byref(ms)), "mgr_kernel_time")
        return n.value, ms.value

    def kernel_bytes(self, name: str) -> float:
        """Algorithmic bytes declared by the launches recorded for a named kernel since profile(True)."""
        b = ctypes.c_double()
        _check(lib().mgr_kernel_bytes(self._h, name.encode(), ctypes.byref(b)), "mgr_kernel_bytes")
        return b.value

    def kernel_bytes_stored(self, name: str) -> float:
        """The same bytes with the column indices in the form the sliced layouts store them."""
        b = ctypes.c_double()
        _check(lib().mgr_kernel_bytes_stored(self._h, name.encode(), ctypes.byref(b)), "mgr_kernel_bytes_stored")
        return b.value

    def memory_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(lib().mgr_memory_bytes(self._h, ctypes.byref(b)), "mgr_memory_bytes")
        return b.value

    def memory_peak_bytes(self) -> int:
        """Most device bytes the handle has held at once since it was created."""
        b = ctypes.c_int64()
        _check(lib().mgr_memory_peak_bytes(self._h, ctypes.byref(b)), "mgr_memory_peak_bytes")
        return b.value

    def stats(self):
        s, a, g, t = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mgr_get_stats(self._h, ctypes.byref(s), ctypes.byref(a), ctypes.byref(g), ctypes.byref(t)),
               "mgr_get_stats")
        return dict(setup_ms=s.value, apply_launches=a.value, graph_nodes=g.value, total_launches=t.value)


def host_wait_count() -> int:
    """Process-wide number of host waits on the GPU (read-backs, synchronisations) issued by the library."""
    t = ctypes.c_int64()
    _check(lib().mgr_get_host_waits(ctypes.byref(t)), "mgr_get_host_waits")
    return t.value


def launch_count() -> int:
    """Process-wide number of kernel launches issued by the library since it was loaded."""
    t = ctypes.c_int64()
    _check(lib().mgr_get_stats(None, None, None, None, ctypes.byref(t)), "mgr_get_stats")
    return t.value


def bsr3_spmv(A: BSR3, x, sub=None, out=None):
    """y = A x, or y = sub - A x, FP64."""
    import torch
    y = out if out is not None else torch.empty_like(x)
    _check(lib().mgr_bsr3_spmv(ctypes.byref(A.c()), _ptr(x), _ptr(sub), _ptr(y), _stream()), "mgr_bsr3_spmv")
    return y


def bsr3_transpose(A: BSR3) -> BSR3:
    import torch
    rp = torch.empty_like(A.rowptr)
    ci = torch.empty_like(A.colind)
    v = torch.empty_like(A.values)
    _check(lib().mgr_bsr3_transpose(ctypes.byref(A.c()), _ptr(rp), _ptr(ci), _ptr(v), _stream()),
           "mgr_bsr3_transpose")
    return BSR3(rp, ci, v)


def bsr3_outer_grad(A: BSR3, lam, x):
    """-lambda_i x_j on every stored block entry of A (the adjoint gradient dL/dA on the pattern)."""
    import torch
    g = torch.empty_like(A.values)
    _check(lib().mgr_bsr3_outer_grad(ctypes.byref(A.c()), _ptr(lam), _ptr(x), _ptr(g), _stream()),
           "mgr_bsr3_outer_grad")
    return g


from .autograd import MgrSolve, mgr_solve  # noqa: E402


def probe_fp64_fma(chain_len: int = 4096, launches: int = 20):
    """Measured FP64 FMA rate of the current GPU (mgr_probe_fp64_fma): (G FMA/s, ms per launch)."""
    g, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().mgr_probe_fp64_fma(chain_len, launches, _stream(), ctypes.byref(g), ctypes.byref(ms)),
           "mgr_probe_fp64_fma")
    return g.value, ms.value
