"""TEST INFRASTRUCTURE: ctypes binding of the plain FP64 CPU oracle (mgr_oracle.c).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package.  It shares no code with the GPU library; both are fed the same arrays by ``ncpgen``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgr_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libmgr_oracle.so")
_lib = None
MAXLEV = 8

STATUS = {0: "ok", 1: "invalid argument", 2: "singular", 3: "not converged", 4: "breakdown", 5: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle: single thread, -O2, no fused multiply-add (-ffp-contract=off)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Opts(ctypes.Structure):
    _fields_ = [("global_relax", ctypes.c_int32),
                ("frelax_type", ctypes.c_int32 * MAXLEV),
                ("frelax_sweeps", ctypes.c_int32 * MAXLEV),
                ("frelax_omega", ctypes.c_double * MAXLEV),
                ("restrict_type", ctypes.c_int32 * MAXLEV),
                ("apply_full_R", ctypes.c_int32),
                ("coarse_solver", ctypes.c_int32),
                ("amg_theta", ctypes.c_double),
                ("amg_max_levels", ctypes.c_int32),
                ("amg_max_coarse", ctypes.c_int32),
                ("amg_smoother", ctypes.c_int32),
                ("amg_pre", ctypes.c_int32),
                ("amg_post", ctypes.c_int32),
                ("amg_pmax", ctypes.c_int32),
                ("amg_omega", ctypes.c_double),
                ("amg_seed", ctypes.c_uint64),
                ("ideal", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("relres_true", ctypes.c_double), ("relres_est", ctypes.c_double),
                ("bnorm", ctypes.c_double)]


DEFAULTS = dict(global_relax=1, frelax_type=[0, 1, 1], frelax_sweeps=[1, 2, 2], frelax_omega=[1.0, 1.0, 1.0],
                restrict_type=[1, 0, 0], apply_full_R=0, coarse_solver=0, amg_theta=0.25, amg_max_levels=25,
                amg_max_coarse=256, amg_smoother=1, amg_pre=1, amg_post=1, amg_pmax=0, amg_omega=1.0,
                amg_seed=3, ideal=0)


def _opts(**kw) -> _Opts:
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(f"unknown option {k}")
        d[k] = v
    o = _Opts()
    for k, v in d.items():
        if isinstance(v, (list, tuple)):
            arr = getattr(o, k)
            last = v[-1]
            for i in range(MAXLEV):
                arr[i] = v[i] if i < len(v) else last
        else:
            setattr(o, k, v)
    return o


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        P = ctypes.POINTER
        lib.oracle_mgr_setup.restype = vp
        lib.oracle_mgr_setup.argtypes = [i64, vp, vp, vp, vp, P(_Opts), P(ctypes.c_int)]
        lib.oracle_mgr_free.argtypes = [vp]
        lib.oracle_mgr_apply.argtypes = [vp, vp, vp]
        lib.oracle_fgmres.argtypes = [vp, i64, vp, vp, vp, vp, vp, ctypes.c_double, i32, i32, P(_Info),
                                      vp, vp, vp, vp]
        lib.oracle_get_info.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int)]
        lib.oracle_mat_shape.argtypes = [vp, i32, i32, P(i64), P(i64), P(i64)]
        lib.oracle_mat_copy.argtypes = [vp, i32, i32, vp, vp, vp]
        lib.oracle_vec_len.argtypes = [vp, i32, i32, P(i64)]
        lib.oracle_vec_copy.argtypes = [vp, i32, i32, vp]
        lib.oracle_amg_setup_csr.restype = vp
        lib.oracle_amg_setup_csr.argtypes = [i64, vp, vp, vp, P(_Opts), P(ctypes.c_int)]
        lib.oracle_amg_vcycle.argtypes = [vp, vp, vp]
        lib.oracle_spgemm_csr.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, P(i64), vp, vp, vp]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


# introspection kinds (see mgr_oracle.c)
MAT_LEVEL, MAT_WP, MAT_WR, MAT_P, MAT_R, MAT_AMG_A, MAT_AMG_P, MAT_AMG_R, MAT_AMG_S = range(9)
VEC_MINV, VEC_AMG_DINV, VEC_BINV, VEC_F, VEC_C, VEC_AMG_CF = range(6)


class _Handle:
    def __init__(self, h):
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            _load().oracle_mgr_free(self._h)
            self._h = None

    def info(self):
        L, na = ctypes.c_int(), ctypes.c_int()
        _load().oracle_get_info(self._h, ctypes.byref(L), ctypes.byref(na))
        return L.value, na.value

    def mat(self, kind: int, level: int):
        """(rowptr, col, val, shape) of an operator of the hierarchy."""
        lib = _load()
        nr, nc, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = lib.oracle_mat_shape(self._h, kind, level, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz))
        if rc:
            raise OracleError(rc, f"no matrix kind={kind} level={level}")
        rp = np.empty(nr.value + 1, np.int64)
        ci = np.empty(nnz.value, np.int32)
        v = np.empty(nnz.value, np.float64)
        lib.oracle_mat_copy(self._h, kind, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        return rp, ci, v, (nr.value, nc.value)

    def scipy(self, kind: int, level: int):
        import scipy.sparse as sp
        rp, ci, v, shape = self.mat(kind, level)
        return sp.csr_matrix((v, ci, rp), shape=shape)

    def vec(self, kind: int, level: int) -> np.ndarray:
        lib = _load()
        n = ctypes.c_int64()
        rc = lib.oracle_vec_len(self._h, kind, level, ctypes.byref(n))
        if rc:
            raise OracleError(rc, f"no vector kind={kind} level={level}")
        out = np.empty(n.value, np.float64)
        lib.oracle_vec_copy(self._h, kind, level, out.ctypes.data)
        return out


class OracleMGR(_Handle):
    """MGR hierarchy built by the oracle for a 3x3 BSR matrix and a cf_marker."""

    def __init__(self, rowptr, colind, values, cf_marker, **opts):
        lib = _load()
        self.rowptr = np.ascontiguousarray(rowptr, np.int64)
        self.colind = np.ascontiguousarray(colind, np.int32)
        self.values = np.ascontiguousarray(values, np.float64).reshape(-1, 9)
        self.marker = np.ascontiguousarray(cf_marker, np.int8)
        self.nb = self.rowptr.shape[0] - 1
        o = _opts(**opts)
        st = ctypes.c_int()
        h = lib.oracle_mgr_setup(self.nb, self.rowptr.ctypes.data, self.colind.ctypes.data, self.values.ctypes.data,
                                 self.marker.ctypes.data, ctypes.byref(o), ctypes.byref(st))
        if not h:
            raise OracleError(st.value, "oracle_mgr_setup")
        super().__init__(h)

    def apply(self, r: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(r, np.float64)
        z = np.empty_like(r)
        _load().oracle_mgr_apply(self._h, r.ctypes.data, z.ctypes.data)
        return z

    def global_relax(self, r: np.ndarray) -> np.ndarray:
        """Algorithm step (1) alone: blockdiag(A)^-1 r."""
        r = np.ascontiguousarray(r, np.float64)
        e = np.empty_like(r)
        _load().oracle_global_relax.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _load().oracle_global_relax(self._h, r.ctypes.data, e.ctypes.data)
        return e

    def fgmres(self, b, x0=None, rtol=1e-8, restart=30, maxit=1000, precondition=True, capture=False):
        return fgmres(self.rowptr, self.colind, self.values, b, x0, rtol, restart, maxit,
                      self if precondition else None, capture)


def fgmres(rowptr, colind, values, b, x0=None, rtol=1e-8, restart=30, maxit=1000, prec=None, capture=False):
    """Flexible GMRES(restart) on the BSR matrix; prec = OracleMGR or None.  Returns (x, info dict)."""
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colind = np.ascontiguousarray(colind, np.int32)
    values = np.ascontiguousarray(values, np.float64).reshape(-1, 9)
    nb = rowptr.shape[0] - 1
    n = 3 * nb
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64, copy=True)
    info = _Info()
    hist = np.zeros(maxit + 2)
    V = Z = H = None
    if capture:
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
    ptr = lambda a: a.ctypes.data if a is not None else None
    rc = lib.oracle_fgmres(prec._h if prec is not None else None, nb, rowptr.ctypes.data, colind.ctypes.data,
                           values.ctypes.data, b.ctypes.data, x.ctypes.data, rtol, restart, maxit,
                           ctypes.byref(info), hist.ctypes.data, ptr(V), ptr(Z), ptr(H))
    out = dict(status=rc, iterations=info.iterations, restarts=info.restarts, converged=bool(info.converged),
               relres_true=info.relres_true, relres_est=info.relres_est, bnorm=info.bnorm,
               history=hist[: info.iterations + 1].copy())
    if capture:
        out.update(V=V, Z=Z, H=H)
    return x, out


class OracleAMG(_Handle):
    """AMG hierarchy on a scalar CSR matrix (the pressure-system solver on its own)."""

    def __init__(self, rowptr, col, val, **opts):
        lib = _load()
        self.rowptr = np.ascontiguousarray(rowptr, np.int64)
        self.col = np.ascontiguousarray(col, np.int32)
        self.val = np.ascontiguousarray(val, np.float64)
        o = _opts(**opts)
        st = ctypes.c_int()
        h = lib.oracle_amg_setup_csr(self.rowptr.shape[0] - 1, self.rowptr.ctypes.data, self.col.ctypes.data,
                                     self.val.ctypes.data, ctypes.byref(o), ctypes.byref(st))
        if not h:
            raise OracleError(st.value, "oracle_amg_setup_csr")
        super().__init__(h)

    def vcycle(self, b: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64)
        x = np.empty_like(b)
        _load().oracle_amg_vcycle(self._h, b.ctypes.data, x.ctypes.data)
        return x


def spgemm(A, B):
    """C = A B (scipy CSR inputs) by the oracle's Gustavson product; returns scipy CSR (structural)."""
    import scipy.sparse as sp
    lib = _load()
    A = sp.csr_matrix(A); B = sp.csr_matrix(B)
    A.sort_indices(); B.sort_indices()
    arp, aci, av = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)
    brp, bci, bv = B.indptr.astype(np.int64), B.indices.astype(np.int32), B.data.astype(np.float64)
    nnz = ctypes.c_int64()
    args = (A.shape[0], A.shape[1], B.shape[1], arp.ctypes.data, aci.ctypes.data, av.ctypes.data,
            brp.ctypes.data, bci.ctypes.data, bv.ctypes.data, ctypes.byref(nnz))
    lib.oracle_spgemm_csr(*args, None, None, None)
    crp = np.empty(A.shape[0] + 1, np.int64)
    cci = np.empty(nnz.value, np.int32)
    cv = np.empty(nnz.value, np.float64)
    lib.oracle_spgemm_csr(*args, crp.ctypes.data, cci.ctypes.data, cv.ctypes.data)
    return sp.csr_matrix((cv, cci, crp), shape=(A.shape[0], B.shape[1]))


def dense_adjoint(rowptr, colind, values, b, w):
    """Dense adjoint of L = w . x with A x = b: lambda = A^-T w, dL/db = lambda and
    dL/dA_ij = -lambda_i x_j on every stored block entry (plain definition, numpy LU)."""
    import scipy.sparse as sp
    values = np.asarray(values, np.float64).reshape(-1, 3, 3)
    nb = len(rowptr) - 1
    A = sp.bsr_matrix((values, colind, rowptr), shape=(3 * nb, 3 * nb)).toarray()
    x = np.linalg.solve(A, b)
    lam = np.linalg.solve(A.T, w)
    rows = np.repeat(np.arange(nb), np.diff(rowptr))
    g = -lam.reshape(nb, 3)[rows][:, :, None] * x.reshape(nb, 3)[colind][:, None, :]
    return x, lam, g


def extpi(rowptr, col, val, cf, theta=0.25, pmax=0):
    """Extended+i interpolation (scipy CSR, n x nC) for a given C/F split (1 = C, -1 = F)."""
    import scipy.sparse as sp
    lib = _load()
    lib.oracle_extpi_csr.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    rp = np.ascontiguousarray(rowptr, np.int64); ci = np.ascontiguousarray(col, np.int32)
    v = np.ascontiguousarray(val, np.float64); cf = np.ascontiguousarray(cf, np.int8)
    n = rp.shape[0] - 1
    nnz = ctypes.c_int64()
    args = (n, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, theta, cf.ctypes.data, pmax, ctypes.byref(nnz))
    lib.oracle_extpi_csr(*args, None, None, None)
    prp = np.empty(n + 1, np.int64); pci = np.empty(nnz.value, np.int32); pv = np.empty(nnz.value)
    lib.oracle_extpi_csr(*args, prp.ctypes.data, pci.ctypes.data, pv.ctypes.data)
    return sp.csr_matrix((pv, pci, prp), shape=(n, int((cf == 1).sum())))


def pmis(rowptr, col, val, theta=0.25, seed=3, level=0):
    """Strength graph (scipy CSR pattern, n x n) and PMIS splitting (1 = C, -1 = F) of a scalar matrix,
    with the random numbers of AMG level `level` under `seed`."""
    import scipy.sparse as sp
    lib = _load()
    lib.oracle_pmis_csr.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_void_p]
    rp = np.ascontiguousarray(rowptr, np.int64); ci = np.ascontiguousarray(col, np.int32)
    v = np.ascontiguousarray(val, np.float64)
    n = rp.shape[0] - 1
    nnz = ctypes.c_int64()
    cf = np.zeros(n, np.int8)
    lib.oracle_pmis_csr(n, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, theta, seed, level, None,
                        ctypes.byref(nnz), None, None)
    srp = np.empty(n + 1, np.int64); sci = np.empty(nnz.value, np.int32)
    lib.oracle_pmis_csr(n, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, theta, seed, level, cf.ctypes.data,
                        ctypes.byref(nnz), srp.ctypes.data, sci.ctypes.data)
    S = sp.csr_matrix((np.ones(nnz.value), sci, srp), shape=(n, n))
    return S, cf
