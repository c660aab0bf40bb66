"""Seeded synthetic inputs: 3x3-block NCP Jacobians of two-phase, two-component porous-media flow.

This module manufactures INPUTS only (matrix, phase state, cf_marker, right-hand sides).  It holds
none of the solver's arithmetic; the CPU oracle and the GPU library are both fed from it.  The
physics follows sections 2-3 of Bui, Wang & Osei-Kuffuor (arXiv 1801.08464): water and hydrogen
conservation with Darcy-Muskat velocities and Fick diffusion, Henry's law, the complementarity
constraint min(1 - S_l, C_h P_g - rho) = 0 linearised by the active-set rule of the semi-smooth
Newton algorithm, Corey (n = 2) relative permeabilities and linear capillary pressure, primary
variables (P_l, S_l, rho_l^h) per cell, two-point finite volumes and one backward Euler step.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ncpgen.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libncpgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator (plain C, OpenMP) into ncpgen/_lib/libncpgen.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("sigma", ctypes.c_double), ("layer_contrast", ctypes.c_double),
                ("absent_frac", ctypes.c_double), ("absent_mode", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("seed", ctypes.c_uint64), ("phi", ctypes.c_double),
                ("closure", ctypes.c_int32), ("state_mode", ctypes.c_int32), ("vg_n", ctypes.c_double),
                ("s_lr", ctypes.c_double), ("s_gr", ctypes.c_double), ("p_r", ctypes.c_double),
                ("s_l1", ctypes.c_double), ("s_l2", ctypes.c_double), ("closed", ctypes.c_int32),
                ("pad2_", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.ncp_count.argtypes = [P(_Cfg), P(ctypes.c_int64), P(ctypes.c_int64)]
        lib.ncp_build.argtypes = [P(_Cfg)] + [ctypes.c_void_p] * 6
        lib.ncp_residual.argtypes = [P(_Cfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.ncp_jacobian.argtypes = [P(_Cfg)] + [ctypes.c_void_p] * 6
        lib.ncp_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        lib.ncp_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        lib.ncp_cf_marker.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclasses.dataclass
class GridConfig:
    """Workload recipe: grid, permeability field and phase state."""
    nx: int
    ny: int
    nz: int = 1
    sigma: float = 1.0            # std-dev of log-permeability
    layer_contrast: float = 0.0   # 0 = no layers, else multiplier of the low-permeability layers
    absent_frac: float = 0.3      # fraction of gas-absent cells
    absent_mode: int = 0          # 0 = i.i.d. cells, 1 = seeded blob
    seed: int = 1
    phi: float = 0.3
    closure: int = 0              # 0 = Corey n = 2 + linear P_c, 1 = Van Genuchten (regularised P_c)
    state_mode: int = 0           # 0 = seeded state, 1 = two sub-domains at s_l1 / s_l2 (section 6.1)
    vg_n: float = 1.54
    s_lr: float = 0.01
    s_gr: float = 0.0
    p_r: float = 2.0
    s_l1: float = 0.962
    s_l2: float = 0.842
    closed: int = 0               # 1 = no-flow boundary everywhere

    def _c(self) -> _Cfg:
        return _Cfg(self.nx, self.ny, self.nz, self.sigma, self.layer_contrast, self.absent_frac,
                    self.absent_mode, 0, self.seed, self.phi, self.closure, self.state_mode, self.vg_n,
                    self.s_lr, self.s_gr, self.p_r, self.s_l1, self.s_l2, self.closed, 0)


# The five workloads: 32x32 plain FP64; 64^3 FP64 with AMG; 128^3 mixed precision (headline);
# 64^3 adjoint; 256^3 mixed precision forward + adjoint.  Then the unsaturated two-level family of
# section 6.1 (Van Genuchten closures with n = 1.54, S_lr = 0.01, S_gr = 0, entry pressure 2 in
# units of the 1e6 Pa liquid pressure; homogeneous permeability; closed boundary; gas present
# everywhere; sub-domains at S_l = 0.962 and 0.842) on its four meshes.
WORKLOADS = {
    "ncp2d_32x32": GridConfig(32, 32, 1, sigma=1.0, absent_frac=0.3, absent_mode=0),
    "ncp3d_64": GridConfig(64, 64, 64, sigma=2.0, absent_frac=0.5, absent_mode=1),
    "ncp3d_128_layered": GridConfig(128, 128, 128, sigma=1.0, layer_contrast=1e-4, absent_frac=0.4, absent_mode=1),
    "ncp3d_64_adjoint": GridConfig(64, 64, 64, sigma=2.0, absent_frac=0.5, absent_mode=1),
    "ncp3d_256_layered": GridConfig(256, 256, 256, sigma=2.0, layer_contrast=1e-6, absent_frac=0.5, absent_mode=1),
}
for _nx, _ny in ((200, 10), (400, 20), (800, 40), (1600, 80)):
    WORKLOADS[f"unsat2d_{_nx}x{_ny}"] = GridConfig(_nx, _ny, 1, sigma=0.0, absent_frac=0.0, closure=1, state_mode=1,
                                                  closed=1)


@dataclasses.dataclass
class Problem:
    cfg: GridConfig
    nb: int
    rowptr: np.ndarray      # int64 [nb+1]
    colind: np.ndarray      # int32 [nnzb]
    values: np.ndarray      # float64 [nnzb, 3, 3], entry (p, q) = dR_p(I)/du_q(J)
    gas_present: np.ndarray  # int8 [nb]
    cf_marker: np.ndarray   # int8 [3 nb]
    state: np.ndarray       # float64 [nb, 3] linearisation point (P_l, S_l, rho)
    perm: np.ndarray        # float64 [nb]

    @property
    def n(self) -> int:
        return 3 * self.nb

    @property
    def nnzb(self) -> int:
        return int(self.colind.shape[0])

    def to_scipy(self):
        """The matrix as a scipy BSR matrix (for dense checks in the tests)."""
        import scipy.sparse as sp
        return sp.bsr_matrix((self.values, self.colind, self.rowptr), shape=(self.n, self.n))


def make_problem(cfg: GridConfig) -> Problem:
    lib = _load()
    c = cfg._c()
    nb, nnzb = ctypes.c_int64(), ctypes.c_int64()
    if lib.ncp_count(ctypes.byref(c), ctypes.byref(nb), ctypes.byref(nnzb)) != 0:
        raise ValueError(f"invalid grid config {cfg}")
    nb, nnzb = nb.value, nnzb.value
    rowptr = np.empty(nb + 1, np.int64)
    colind = np.empty(nnzb, np.int32)
    values = np.empty((nnzb, 3, 3), np.float64)
    gp = np.empty(nb, np.int8)
    state = np.empty((nb, 3), np.float64)
    perm = np.empty(nb, np.float64)
    rc = lib.ncp_build(ctypes.byref(c), rowptr.ctypes.data, colind.ctypes.data, values.ctypes.data,
                       gp.ctypes.data, state.ctypes.data, perm.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"ncp_build failed ({rc})")
    marker = np.empty(3 * nb, np.int8)
    lib.ncp_cf_marker(nb, gp.ctypes.data, marker.ctypes.data)
    return Problem(cfg, nb, rowptr, colind, values, gp, marker, state, perm)


def residual(cfg: GridConfig, u: np.ndarray, u_old: np.ndarray | None = None) -> np.ndarray:
    """Nonlinear residual R(u) of one backward Euler step; u_old (optional) is the previous time
    level, whose mass is subtracted."""
    lib = _load()
    u = np.ascontiguousarray(u, np.float64).reshape(-1)
    uo = None if u_old is None else np.ascontiguousarray(u_old, np.float64).reshape(-1)
    R = np.empty_like(u)
    if lib.ncp_residual(ctypes.byref(cfg._c()), u.ctypes.data, None if uo is None else uo.ctypes.data,
                        R.ctypes.data) != 0:
        raise RuntimeError("ncp_residual failed")
    return R


def jacobian(cfg: GridConfig, u: np.ndarray, want_residual: bool = False, u_old: np.ndarray | None = None):
    """BSR Jacobian (rowptr, colind, values) at an arbitrary state u, with the configuration's
    permeability and the active-set rule of the constraint rows; also R(u) when asked (u_old: the
    previous time level, as in `residual`)."""
    lib = _load()
    c = cfg._c()
    nb, nnzb = ctypes.c_int64(), ctypes.c_int64()
    if lib.ncp_count(ctypes.byref(c), ctypes.byref(nb), ctypes.byref(nnzb)) != 0:
        raise ValueError(f"invalid grid config {cfg}")
    nb, nnzb = nb.value, nnzb.value
    u = np.ascontiguousarray(u, np.float64).reshape(-1)
    if u.size != 3 * nb:
        raise ValueError("state size does not match the grid")
    rowptr = np.empty(nb + 1, np.int64)
    colind = np.empty(nnzb, np.int32)
    values = np.empty((nnzb, 3, 3), np.float64)
    R = np.empty(3 * nb, np.float64) if want_residual else None
    uo = None if u_old is None else np.ascontiguousarray(u_old, np.float64).reshape(-1)
    rc = lib.ncp_jacobian(ctypes.byref(c), u.ctypes.data, None if uo is None else uo.ctypes.data,
                          rowptr.ctypes.data, colind.ctypes.data, values.ctypes.data,
                          R.ctypes.data if R is not None else None)
    if rc != 0:
        raise RuntimeError(f"ncp_jacobian failed ({rc})")
    return (rowptr, colind, values, R) if want_residual else (rowptr, colind, values)


def newton_system(cfg: GridConfig, u: np.ndarray, u_old: np.ndarray | None = None):
    """The linear system of one semi-smooth Newton step at u (section 3.1): the BSR Jacobian, R(u),
    the cf_marker of the step's active set and the active set itself (True where a constraint row
    takes the G branch, i.e. the gas phase is present)."""
    rowptr, colind, values, R = jacobian(cfg, u, want_residual=True, u_old=u_old)
    rows = np.repeat(np.arange(rowptr.shape[0] - 1), np.diff(rowptr))
    d = values[rows == colind]
    active = d[:, 2, 2] == -1.0  # G' = (C_h, C_h P_c', -1); F' = (0, -1, 0)
    marker = cf_marker(active.astype(np.int8))
    return rowptr, colind, values, R, marker, active


def normals(n: int, seed: int, stream: int = 2) -> np.ndarray:
    """Seeded N(0,1) vector (splitmix64 counters + Box-Muller); stream 2 = rhs, 4 = adjoint w."""
    out = np.empty(n, np.float64)
    _load().ncp_normals(seed, stream, n, out.ctypes.data)
    return out


def uniforms(n: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().ncp_uniforms(seed, stream, n, out.ctypes.data)
    return out


def cf_marker(gas_present: np.ndarray) -> np.ndarray:
    gp = np.ascontiguousarray(gas_present, np.int8)
    out = np.empty(3 * gp.shape[0], np.int8)
    _load().ncp_cf_marker(gp.shape[0], gp.ctypes.data, out.ctypes.data)
    return out


def poisson(nx: int, ny: int, nz: int = 1, neumann: bool = False):
    """Scalar 5/7-point Laplacian as CSR arrays (rowptr int64, col int32, val float64): Dirichlet
    (diagonal 2d) or pure Neumann rows with zero row sum when neumann=True."""
    n = nx * ny * nz
    rows, cols, vals = [], [], []
    idx = np.arange(n).reshape(nz, ny, nx)
    diag = np.zeros(n)
    for axis, m in ((2, nx), (1, ny), (0, nz)):
        if m == 1:
            continue
        a = np.take(idx, np.arange(m - 1), axis=axis).ravel()
        b = np.take(idx, np.arange(1, m), axis=axis).ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [-np.ones(a.size), -np.ones(a.size)]
        np.add.at(diag, a, 1.0)
        np.add.at(diag, b, 1.0)
    if not neumann:
        dim = sum(1 for m in (nx, ny, nz) if m > 1)
        diag[:] = 2.0 * dim
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    import scipy.sparse as sp
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)
