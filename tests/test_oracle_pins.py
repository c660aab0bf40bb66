"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU).

Each test states the passage it pins.  None of them compares the oracle with itself: the
references are dense numpy linear algebra, scipy's sparse product, closed forms from the paper,
hand-computed interpolation weights and invariants of the published AMG components.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import ncpgen
import oracle

TINY = [
    ncpgen.GridConfig(6, 6, 1, sigma=1.0, absent_frac=0.3, absent_mode=0, seed=5),
    ncpgen.GridConfig(4, 4, 4, sigma=2.0, absent_frac=0.5, absent_mode=1, seed=6),
    ncpgen.GridConfig(5, 4, 3, sigma=1.0, layer_contrast=1e-4, absent_frac=0.4, absent_mode=1, seed=7),
]


def _level_sets(marker):
    """Level-l dof lists (ascending original index) and the F/C splits of section 5."""
    L = int(marker.max())
    dofs = [np.nonzero(marker >= l)[0] for l in range(L + 1)]
    return L, dofs


def _schur(A, F, C):
    Aff, Afc, Acf, Acc = A[np.ix_(F, F)], A[np.ix_(F, C)], A[np.ix_(C, F)], A[np.ix_(C, C)]
    return Acc - Acf @ np.linalg.solve(Aff, Afc) if len(F) else Acc


def _split(marker_l, l):
    return np.nonzero(marker_l == l)[0], np.nonzero(marker_l > l)[0]


@pytest.mark.parametrize("cfg", TINY)
@pytest.mark.parametrize("rtype", [0, 1])
def test_ideal_RAP_is_schur_complement(cfg, rtype):
    """Section 4: with ideal P = [-A_ff^-1 A_fc; I], R A P equals S = A_cc - A_cf A_ff^-1 A_fc for
    injective and non-injective R (RAQ = 0 in the MGR identities)."""
    p = ncpgen.make_problem(cfg)
    m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, ideal=1, restrict_type=[rtype] * 3)
    L, dofs = _level_sets(p.cf_marker)
    A = p.to_scipy().toarray()
    for l in range(L):
        mk = p.cf_marker[dofs[l]]
        F, C = _split(mk, l)
        A = _schur(A, F, C)
        got = m.scipy(oracle.MAT_LEVEL, l + 1).toarray()
        assert np.abs(got - A).max() <= 1e-11 * np.abs(A).max()


@pytest.mark.parametrize("cfg", TINY)
def test_ideal_preconditioner_is_exact_inverse(cfg):
    """MGR identities (section 4): exact F-solves, ideal P and an exact coarse solve make the
    two-level error propagator zero, so M^-1 A = I and FGMRES converges in one iteration."""
    p = ncpgen.make_problem(cfg)
    m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, ideal=1)
    A = p.to_scipy()
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(p.n)
        z = m.apply(A @ x)
        assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x)
    b = ncpgen.normals(p.n, 2)
    x, info = m.fgmres(b, rtol=1e-9)
    assert info["converged"] and info["iterations"] == 1


@pytest.mark.parametrize("cfg", TINY)
def test_level1_is_exact_and_matches_closed_form(cfg):
    """Section 5: the first reduction is exact because C33 is diagonal, so with
    W_p = -D_ff^-1 A_fc the coarse operator equals the closed form
    [[A11 - A13 C33^-1 C31, A12 - A13 C33^-1 C32, A14], [...], [C41, C42, 0]] (the Schur complement)."""
    p = ncpgen.make_problem(cfg)
    m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker)
    A = p.to_scipy().toarray()
    F, C = _split(p.cf_marker, 0)
    Aff = A[np.ix_(F, F)]
    assert np.count_nonzero(Aff - np.diag(np.diag(Aff))) == 0
    S1 = A[np.ix_(C, C)] - A[np.ix_(C, F)] @ np.diag(1.0 / np.diag(Aff)) @ A[np.ix_(F, C)]
    got = m.scipy(oracle.MAT_LEVEL, 1).toarray()
    assert np.abs(got - S1).max() <= 1e-13 * np.abs(S1).max()
    # gas-absent constraint rows keep their 0 diagonal: the paper's C41 C42 0 block
    mk1 = p.cf_marker[C]
    absent_rows = np.nonzero(mk1 == 2)[0]
    assert np.all(np.diag(got)[absent_rows] == 0.0)


@pytest.mark.parametrize("cfg", TINY)
def test_levels_2_and_3_match_paper_formulas(cfg):
    """Section 5: with injective R and S~_22 = diag(S_22),
    S^2 = S^1_cc - S^1_cf diag(S^1_ff)^-1 S^1_fc (the displayed 2x2 block formula) and
    S^3 = S^2_11 - S^2_12 diag(S^2_22)^-1 S^2_21; after level 2 the diagonal has no zeros."""
    p = ncpgen.make_problem(cfg)
    m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker)
    L, dofs = _level_sets(p.cf_marker)
    for l in (1, 2):
        Sl = m.scipy(oracle.MAT_LEVEL, l).toarray()
        F, C = _split(p.cf_marker[dofs[l]], l)
        D = np.diag(Sl[np.ix_(F, F)])
        ref = Sl[np.ix_(C, C)] - Sl[np.ix_(C, F)] @ (Sl[np.ix_(F, C)] / D[:, None])
        got = m.scipy(oracle.MAT_LEVEL, l + 1).toarray()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        if l == 2:
            assert np.all(np.diag(Sl) != 0.0)


@pytest.mark.parametrize("cfg", TINY + [ncpgen.GridConfig(12, 10, 1, absent_frac=0.25, seed=9)])
def test_level_sizes(cfg):
    """Sections 3.2 and 5: level sizes 3N - M, 2N - M and N (M gas-present cells)."""
    p = ncpgen.make_problem(cfg)
    m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker)
    N, M = p.nb, int(p.gas_present.sum())
    sizes = [m.mat(oracle.MAT_LEVEL, l)[3][0] for l in range(4)]
    assert sizes == [3 * N, 3 * N - M, 2 * N - M, N]


@pytest.mark.parametrize("cfg", [
    ncpgen.GridConfig(4, 4, 1, sigma=0.5, absent_frac=0.3, seed=21),
    ncpgen.GridConfig(8, 8, 1, sigma=1.0, absent_frac=0.3, seed=22),
    ncpgen.GridConfig(4, 4, 4, sigma=1.0, absent_frac=0.5, absent_mode=1, seed=23),
])
def test_fgmres_mgr_matches_dense_solve(cfg):
    """x = A^-1 b by dense LU (numpy) versus MGR-FGMRES run to 1e-12."""
    p = ncpgen.make_problem(cfg)
    A = p.to_scipy().toarray()
    b = ncpgen.normals(p.n, 2)
    xd = np.linalg.solve(A, b)
    m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, amg_max_coarse=8)
    x, info = m.fgmres(b, rtol=1e-12, restart=30, maxit=500)
    assert info["converged"]
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.0001
    err = np.linalg.norm(x - xd) / np.linalg.norm(xd)
    assert err <= 1e-12 * np.linalg.cond(A)
    assert err <= 1e-9


def test_gmres_exact_in_n_steps_and_arnoldi_relation():
    """GMRES(m >= n) on n = 48 unknowns terminates within n steps; A Z_j = V_{j+1} Hbar_j holds;
    the implicit residual estimate agrees with the explicit one."""
    p = ncpgen.make_problem(ncpgen.GridConfig(4, 4, 1, sigma=0.5, absent_frac=0.3, seed=31))
    A = p.to_scipy().toarray()
    b = ncpgen.normals(p.n, 2)
    x, info = oracle.fgmres(p.rowptr, p.colind, p.values, b, rtol=1e-10, restart=p.n, maxit=p.n, capture=True)
    assert info["converged"] and info["iterations"] <= p.n
    k = info["iterations"]
    V, Z, H = info["V"], info["Z"], info["H"]
    lhs = A @ Z[:k].T
    rhs = V[: k + 1].T @ H[: k + 1, :k]
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()
    # the leading basis vectors are orthonormal (MGS loses orthogonality only as the basis grows)
    G = V[:8] @ V[:8].T
    assert np.abs(G - np.eye(8)).max() < 1e-12
    assert abs(info["relres_est"] - info["relres_true"]) <= 1e-9


def test_flexible_arnoldi_relation_with_mgr():
    """With the MGR preconditioner (Z != V) the flexible relation A Z_j = V_{j+1} Hbar_j holds."""
    p = ncpgen.make_problem(ncpgen.GridConfig(6, 6, 1, sigma=1.0, absent_frac=0.3, seed=32))
    A = p.to_scipy().toarray()
    b = ncpgen.normals(p.n, 2)
    m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, amg_max_coarse=8)
    x, info = m.fgmres(b, rtol=1e-10, restart=20, capture=True)
    k = min(info["iterations"], 20)
    V, Z, H = info["V"], info["Z"], info["H"]
    lhs = A @ Z[:k].T
    rhs = V[: k + 1].T @ H[: k + 1, :k]
    assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(lhs).max()


def test_spgemm_matches_scipy():
    rng = np.random.default_rng(3)
    for m_, k_, n_, d in [(50, 40, 60, 0.1), (200, 150, 120, 0.03), (7, 9, 5, 0.5)]:
        A = sp.random(m_, k_, density=d, random_state=rng, format="csr")
        B = sp.random(k_, n_, density=d, random_state=rng, format="csr")
        C = oracle.spgemm(A, B)
        ref = (A @ B).toarray()
        assert np.allclose(C.toarray(), ref, rtol=1e-14, atol=1e-15)
        # structural pattern: every position of every product is present
        patt = ((abs(A) > 0).astype(int) @ (abs(B) > 0).astype(int)).toarray() > 0
        assert np.array_equal(C.toarray() != 0, (C.toarray() != 0) & patt)
        assert C.nnz == patt.sum()


def test_extpi_linear_interpolation_1d():
    """Extended+i on the 1-D Laplacian with the split C F F C F F C: the distance-two formula gives
    linear interpolation, weights (2/3, 1/3) and (1/3, 2/3); C points inject."""
    n = 10
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    A.sort_indices()
    cf = np.array([1 if i % 3 == 0 else -1 for i in range(n)], np.int8)
    P = oracle.extpi(A.indptr, A.indices, A.data, cf).toarray()
    expect = np.zeros((n, 4))
    for i in range(n):
        c, r = divmod(i, 3)
        if r == 0:
            expect[i, c] = 1.0
        else:
            expect[i, c] = (3 - r) / 3.0
            if c + 1 < 4:
                expect[i, c + 1] = r / 3.0
    # the last F pair (i = 10 would be C) does not occur: n = 10 ends on a C point
    assert np.abs(P - expect).max() <= 1e-15


def test_extpi_reproduces_constants_on_zero_row_sum_rows():
    """Extended+i interpolation preserves constants on rows of a zero-row-sum M-matrix."""
    rp, ci, v = ncpgen.poisson(12, 12, 1, neumann=True)
    A = sp.csr_matrix((v, ci, rp))
    amg = oracle.OracleAMG(rp, ci, v, amg_max_coarse=4)
    cf = amg.vec(oracle.VEC_AMG_CF, 0).astype(np.int8)
    P = oracle.extpi(rp, ci, v, cf)
    s = np.asarray(P.sum(axis=1)).ravel()
    nonempty = np.diff(P.indptr) > 0
    assert nonempty.sum() > 0.9 * A.shape[0]
    assert np.abs(s[nonempty] - 1.0).max() < 1e-13


def test_strength_anisotropic():
    """Classical strength with theta = 0.25 on the Laplacian with couplings -1 (x) and -0.1 (y):
    only x-neighbours are strong."""
    nx, ny = 10, 8
    n = nx * ny
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            diag = 0.0
            for di, dj, w in ((-1, 0, 1.0), (1, 0, 1.0), (0, -1, 0.1), (0, 1, 0.1)):
                a, b = i + di, j + dj
                if 0 <= a < nx and 0 <= b < ny:
                    rows.append(r); cols.append(b * nx + a); vals.append(-w)
                diag += w
            rows.append(r); cols.append(r); vals.append(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    amg = oracle.OracleAMG(A.indptr, A.indices, A.data, amg_max_coarse=4, amg_theta=0.25)
    S = amg.scipy(oracle.MAT_AMG_S, 0).tocoo()
    assert S.nnz > 0
    assert np.all(np.abs(S.row - S.col) == 1)
    assert S.nnz == 2 * (nx - 1) * ny


@pytest.mark.parametrize("shape", [(16, 16, 1), (8, 8, 8)])
def test_pmis_is_maximal_independent_set_on_symmetric_graph(shape):
    """PMIS (De Sterck, Yang & Heys 2006) on a symmetric strength graph yields C points that are
    pairwise non-adjacent, and every F point with a strong connection has a strong C neighbour."""
    rp, ci, v = ncpgen.poisson(*shape)
    amg = oracle.OracleAMG(rp, ci, v, amg_max_coarse=4)
    cf = amg.vec(oracle.VEC_AMG_CF, 0)
    S = amg.scipy(oracle.MAT_AMG_S, 0)
    assert (S != S.T).nnz == 0
    C = cf == 1
    S = S.tocsr()
    for i in range(S.shape[0]):
        nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
        if C[i]:
            assert not C[nb].any()
        elif len(nb):
            assert C[nb].any()


@pytest.mark.parametrize("shape,bound", [((64, 64, 1), 0.5), ((20, 20, 20), 0.5)])
def test_amg_vcycle_converges_on_poisson(shape, bound):
    """Textbook multigrid behaviour: the V(1,1) cycle as a stationary iteration on the Dirichlet
    Poisson problem contracts the error by a mesh-independent factor well below one."""
    rp, ci, v = ncpgen.poisson(*shape)
    A = sp.csr_matrix((v, ci, rp))
    amg = oracle.OracleAMG(rp, ci, v, amg_max_coarse=50)
    rng = np.random.default_rng(1)
    xs = rng.standard_normal(A.shape[0])
    b = A @ xs
    x = np.zeros_like(b)
    errs = []
    for _ in range(12):
        x = x + amg.vcycle(b - A @ x)
        errs.append(np.sqrt((x - xs) @ (A @ (x - xs))))
    rho = (errs[-1] / errs[1]) ** (1.0 / 10)
    assert rho < bound, rho


def test_edge_cases_all_present_and_all_absent():
    """M = N (no gas-absent cell: the third reduction has no F point) and M = 0 (no gas-present
    cell: the first reduction has no F point) still give a convergent preconditioner."""
    for frac in (0.0, 1.0):
        p = ncpgen.make_problem(ncpgen.GridConfig(8, 8, 1, absent_frac=frac, seed=41))
        m = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker)
        b = ncpgen.normals(p.n, 2)
        x, info = m.fgmres(b, rtol=1e-8)
        assert info["converged"]
        A = p.to_scipy()
        assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001


def test_singular_diagonal_block_is_reported():
    p = ncpgen.make_problem(ncpgen.GridConfig(4, 4, 1, seed=2))
    vals = p.values.copy()
    rows = np.repeat(np.arange(p.nb), np.diff(p.rowptr))
    k = np.nonzero((rows == 3) & (p.colind == 3))[0][0]
    vals[k] = 0.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.OracleMGR(p.rowptr, p.colind, vals, p.cf_marker)
    assert e.value.code == 2


def test_dense_adjoint_matches_finite_differences():
    """dL/db = lambda and dL/dA_ij = -lambda_i x_j for L = w . A^-1 b, by central differences."""
    p = ncpgen.make_problem(ncpgen.GridConfig(3, 3, 1, seed=4))
    b = ncpgen.normals(p.n, 2)
    w = ncpgen.normals(p.n, 4, stream=4)
    x, lam, g = oracle.dense_adjoint(p.rowptr, p.colind, p.values, b, w)

    def loss(vals, bb):
        A = sp.bsr_matrix((vals, p.colind, p.rowptr), shape=(p.n, p.n)).toarray()
        return w @ np.linalg.solve(A, bb)

    rng = np.random.default_rng(0)
    for _ in range(8):
        k, a, c = rng.integers(p.nnzb), rng.integers(3), rng.integers(3)
        if p.values[k, a, c] == 0.0:
            continue
        h = 1e-6 * abs(p.values[k, a, c])
        vp, vm = p.values.copy(), p.values.copy()
        vp[k, a, c] += h
        vm[k, a, c] -= h
        fd = (loss(vp, b) - loss(vm, b)) / (2 * h)
        assert abs(fd - g[k, a, c]) <= 1e-6 * max(abs(g[k, a, c]), 1e-3 * np.abs(g).max())
    for i in rng.integers(p.n, size=5):
        e = np.zeros(p.n); e[i] = 1e-6
        fd = (loss(p.values, b + e) - loss(p.values, b - e)) / 2e-6
        assert abs(fd - lam[i]) <= 1e-7 * max(1.0, abs(lam[i]))


def test_global_relaxation_is_blockdiag_inverse():
    """Algorithm step (1): e_1 = blockdiag(A)^-1 r.  On a block-diagonal matrix this is already
    A^-1 r, the later steps add nothing, and M^-1 = A^-1."""
    p = ncpgen.make_problem(ncpgen.GridConfig(5, 4, 1, absent_frac=0.4, seed=51))
    rows = np.repeat(np.arange(p.nb), np.diff(p.rowptr))
    vals = p.values.copy()
    vals[rows != p.colind] = 0.0
    m = oracle.OracleMGR(p.rowptr, p.colind, vals, p.cf_marker, amg_max_coarse=4)
    A = sp.bsr_matrix((vals, p.colind, p.rowptr), shape=(p.n, p.n)).toarray()
    r = ncpgen.normals(p.n, 2)
    z = m.apply(r)
    assert np.linalg.norm(z - np.linalg.solve(A, r)) <= 1e-12 * np.linalg.norm(z)
    full = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker)
    e1 = full.global_relax(r).reshape(-1, 3)
    diag_blocks = p.values[rows == p.colind]
    ref = np.linalg.solve(diag_blocks, r.reshape(-1, 3)[:, :, None])[:, :, 0]
    assert np.abs(e1 - ref).max() <= 1e-12 * np.abs(ref).max()
    binv = m.vec(oracle.VEC_BINV, 0).reshape(-1, 3, 3)
    blocks = vals[rows == p.colind]
    assert np.abs(np.einsum("kij,kjl->kil", binv, blocks) - np.eye(3)).max() < 1e-12


@pytest.mark.parametrize("wy,strong", [(0.3, True), (0.2, False), (0.25, True), (0.26, True), (0.24, False)])
def test_strength_threshold(wy, strong):
    """Classical strength: j is strong for i iff -a_ij >= theta max_k(-a_ik); theta = 0.25 and the
    x-couplings are -1, so a y-coupling -wy is strong exactly when wy >= 0.25."""
    nx, ny = 6, 5
    n = nx * ny
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            diag = 0.0
            for di, dj, w in ((-1, 0, 1.0), (1, 0, 1.0), (0, -1, wy), (0, 1, wy)):
                a, b = i + di, j + dj
                if 0 <= a < nx and 0 <= b < ny:
                    rows.append(r); cols.append(b * nx + a); vals.append(-w)
                diag += w
            rows.append(r); cols.append(r); vals.append(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    amg = oracle.OracleAMG(A.indptr, A.indices, A.data, amg_max_coarse=4, amg_theta=0.25)
    S = amg.scipy(oracle.MAT_AMG_S, 0).tocoo()
    ny_links = int((np.abs(S.row - S.col) == nx).sum())
    assert ny_links == (2 * nx * (ny - 1) if strong else 0)
    assert int((np.abs(S.row - S.col) == 1).sum()) == 2 * (nx - 1) * ny


@pytest.mark.parametrize("cfg", TINY)
@pytest.mark.parametrize("rtype", [0, 1])
def test_amg_frelaxation_exact_limit_is_two_level_formula(cfg, rtype):
    """F-relaxation by AMG (frelax_type 2, section 6.2): when the AMG on A_ff is a single dense level
    (amg_max_coarse >= nF) the F-solve is exact, and with an exact coarse solve and no global
    relaxation one apply of the one-level MGR (markers 0 and 1 only) is the two-level multiplicative
    formula z_F = A_ff^-1 r_F + W_p e_c, z_C = e_c, e_c = A_c^-1 (r_C - A_cf A_ff^-1 r_F),
    with A_c = R A P the oracle's own coarse operator (checked separately by P2-P4)."""
    p = ncpgen.make_problem(cfg)
    marker = np.where(p.cf_marker == 0, 0, 1).astype(np.int8)  # one reduction: the Henry rows
    o = oracle.OracleMGR(p.rowptr, p.colind, p.values, marker, frelax_type=[2], frelax_sweeps=[1],
                         restrict_type=[rtype], global_relax=0, coarse_solver=1, amg_max_coarse=100000)
    assert o.info()[0] == 1
    A = p.to_scipy().toarray()
    F, C = np.nonzero(marker == 0)[0], np.nonzero(marker == 1)[0]
    Ac = o.scipy(oracle.MAT_LEVEL, 1).toarray()
    Wp = o.scipy(oracle.MAT_WP, 0).toarray()
    r = ncpgen.normals(p.n, 3)
    eF = np.linalg.solve(A[np.ix_(F, F)], r[F])
    ec = np.linalg.solve(Ac, r[C] - A[np.ix_(C, F)] @ eF)
    z = np.empty(p.n)
    z[C] = ec
    z[F] = eF + Wp @ ec
    zo = o.apply(r)
    assert np.linalg.norm(zo - z) <= 1e-10 * np.linalg.norm(z)


# ---- Pins of the AMG components the paper leaves to BoomerAMG: interpolation truncation, PMIS on
# ---- non-symmetric strength graphs, and the relaxation scalings (section 4 F-relaxation, section 6
# ---- AMG coarse solve).  The expected values below are worked out by hand from the published
# ---- definitions (extended+i: De Sterck, Falgout, Nolting & Yang 2008; PMIS: De Sterck, Yang &
# ---- Heys 2006; l1-Jacobi: Baker, Falgout, Kolev & Yang 2011).

def _csr(n, entries):
    rows, cols, vals = zip(*entries)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)


# Two F points (0, 1) and four C points (2..5).  Row 0 is strongly connected to F point 1 and to C
# points 2 and 3, and weakly (positive entry) to C point 4, which enters Chat_0 at distance two
# through point 1; C point 5 enters the same way with no direct coupling.  theta = 0.25.
EXTPI_ROWS = [(0, 0, 4.0), (0, 1, -2.0), (0, 2, -1.0), (0, 3, -1.5), (0, 4, 1.5),
              (1, 0, -1.0), (1, 1, 5.0), (1, 4, -2.0), (1, 5, -1.0)] + [(i, i, 1.0) for i in range(2, 6)]
EXTPI_CF = np.array([-1, -1, 1, 1, 1, 1], np.int8)
# Hand computation, row 0: S_0 = {1, 2, 3} (threshold 0.25 * 2 = 0.5; the +1.5 entry is weak),
# F_0^s = {1}, Chat_0 = {2, 3} + C_1^s = {2, 3, 4, 5}.  den_1 = abar_10 + abar_14 + abar_15 =
# -1 - 2 - 1 = -4 (the negative entries of row 1 over Chat_0 + {0}), q_1 = a_01 / den_1 = 1/2.
# Diagonal: a_00 + q_1 abar_10 = 4 - 1/2 = 7/2 (the weak neighbour 4 lies in Chat_0: not lumped).
# Numerators a_0j + q_1 abar_1j: j = 2: -1; j = 3: -3/2; j = 4: 3/2 - 1 = 1/2; j = 5: -1/2.
# Weights -(num / (7/2)): 2/7, 3/7, -1/7, 1/7 (row sum 5/7).
# Row 1: S_1 = {0, 4, 5}, Chat_1 = {4, 5} + C_0^s = {2, 3, 4, 5}; den_0 over Chat_1 + {1} keeps the
# negative entries of row 0: -2 - 1 - 3/2 = -9/2 (the +3/2 at column 4 has the diagonal's sign),
# q_0 = -1 / (-9/2) = 2/9; diagonal 5 + (2/9)(-2) = 41/9; numerators: j = 2: (2/9)(-1) = -2/9;
# j = 3: (2/9)(-3/2) = -1/3; j = 4: -2; j = 5: -1.  Weights 2/41, 3/41, 18/41, 9/41 (sum 32/41).
EXTPI_FULL = {0: [2 / 7, 3 / 7, -1 / 7, 1 / 7], 1: [2 / 41, 3 / 41, 18 / 41, 9 / 41]}
# Truncation to pmax entries keeps the largest |w| (equal |w|: the smaller column) and scales the
# kept ones by (sum of all w) / (sum of kept w), so the row sum is unchanged.
#   row 0, pmax 2: keeps 3/7, 2/7; factor (5/7)/(5/7) = 1.
#   row 0, pmax 3: keeps 3/7, 2/7 and, of the tie |-1/7| = |1/7|, column 2 (w = -1/7); kept sum
#     4/7, factor 5/4: 5/14, 15/28, -5/28.
#   row 1, pmax 2: keeps 18/41, 9/41; factor (32/41)/(27/41) = 32/27: 64/123, 32/123.
#   row 1, pmax 3: keeps 18/41, 9/41, 3/41; factor 32/30: 16/205, 96/205, 48/205.
EXTPI_TRUNC = {2: {0: [2 / 7, 3 / 7, 0, 0], 1: [0, 0, 64 / 123, 32 / 123]},
               3: {0: [5 / 14, 15 / 28, -5 / 28, 0], 1: [0, 16 / 205, 96 / 205, 48 / 205]}}


def test_extpi_hand_computed_distance_two_row():
    """Extended+i weights of two F rows with a distance-two C point, a weak positive coupling to a
    point of Chat_i and a strong F-F coupling, against the hand computation above."""
    rp, ci, v = _csr(6, EXTPI_ROWS)
    P = oracle.extpi(rp, ci, v, EXTPI_CF, theta=0.25).toarray()
    for i, w in EXTPI_FULL.items():
        assert np.abs(P[i] - np.array(w)).max() <= 1e-15, (i, P[i], w)
    assert np.array_equal(P[2:], np.eye(4))  # C points inject


@pytest.mark.parametrize("pmax", [2, 3])
def test_extpi_truncation_hand_computed(pmax):
    """Interpolation truncation (amg_pmax): which entries survive (largest |w|, ties to the smaller
    column), and the rescaling that keeps the row sum, against the hand computation above."""
    rp, ci, v = _csr(6, EXTPI_ROWS)
    P = oracle.extpi(rp, ci, v, EXTPI_CF, theta=0.25, pmax=pmax)
    D = P.toarray()
    for i, w in EXTPI_TRUNC[pmax].items():
        assert np.abs(D[i] - np.array(w)).max() <= 1e-15, (i, D[i], w)
        assert P.indptr[i + 1] - P.indptr[i] == pmax
        assert abs(D[i].sum() - sum(EXTPI_FULL[i])) <= 1e-15
    assert np.array_equal(D[2:], np.eye(4))


def _random_graph_laplacian(nx, ny, seed):
    """Periodic 5-point graph Laplacian with random positive conductances: a zero-row-sum M-matrix."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    ent = {}
    for j in range(ny):
        for i in range(nx):
            a = j * nx + i
            for b in (j * nx + (i + 1) % nx, ((j + 1) % ny) * nx + i):
                g = float(rng.uniform(0.2, 2.0))
                ent[(a, b)] = ent.get((a, b), 0.0) - g
                ent[(b, a)] = ent.get((b, a), 0.0) - g
                ent[(a, a)] = ent.get((a, a), 0.0) + g
                ent[(b, b)] = ent.get((b, b), 0.0) + g
    return _csr(n, [(r, c, x) for (r, c), x in ent.items()])


@pytest.mark.parametrize("pmax", [1, 2, 3])
def test_truncated_extpi_rows_sum_to_one_on_zero_row_sum_matrix(pmax):
    """On a zero-row-sum M-matrix extended+i interpolates constants exactly (every row sums to 1);
    truncation keeps that sum, keeps at most pmax entries, and leaves shorter rows unchanged."""
    rp, ci, v = _random_graph_laplacian(10, 9, seed=pmax)
    _, cf = oracle.pmis(rp, ci, v, theta=0.25, seed=11)
    assert 0 < (cf == 1).sum() < len(cf)
    full = oracle.extpi(rp, ci, v, cf, theta=0.25)
    tr = oracle.extpi(rp, ci, v, cf, theta=0.25, pmax=pmax)
    lf, lt = np.diff(full.indptr), np.diff(tr.indptr)
    assert (lf > pmax).sum() > 10  # truncation is exercised
    assert np.all(lt == np.minimum(lf, pmax))
    s = np.asarray(tr.sum(axis=1)).ravel()
    assert np.abs(s - 1.0).max() <= 1e-13
    short = lf <= pmax
    assert np.abs((full - tr).toarray()[short]).max() == 0.0
    # the kept entries are the largest |w| of the full row
    F = full.toarray()
    T = tr.toarray()
    for i in np.nonzero(~short)[0]:
        kept = np.nonzero(T[i])[0]
        dropped = np.setdiff1d(np.nonzero(F[i])[0], kept)
        assert np.abs(F[i, kept]).min() >= np.abs(F[i, dropped]).max()


def _directed(n, edges, weak=()):
    """A scalar matrix whose strength graph (theta = 0.25) is exactly `edges` (i strongly depends
    on j for (i, j) in edges): strong entries -1, weak entries -0.01, diagonal = row length + 1."""
    ent = {(i, j): -1.0 for i, j in edges}
    for i, j in weak:
        ent.setdefault((i, j), -0.01)
    for i in range(n):
        ent[(i, i)] = 1.0 + sum(1 for (a, _b) in ent if a == i)
    return _csr(n, [(r, c, x) for (r, c), x in ent.items()])


@pytest.mark.parametrize("seed", range(12))
def test_pmis_measure_counts_dependants(seed):
    """PMIS's measure is lambda_i = |S^T_i|, the number of points that strongly depend on i.  Points
    1..5 depend on 0 and 0 depends on 1: lambda = (5, 1, 0, 0, 0, 0) whatever the random part, so
    2..5 (which influence nobody) start as F, 0 beats 1 and becomes C, and 1, depending on 0,
    becomes F.  With the measure taken from S instead, every point has measure 1 and the random
    part decides."""
    rp, ci, v = _directed(6, [(0, 1)] + [(i, 0) for i in range(1, 6)])
    S, cf = oracle.pmis(rp, ci, v, theta=0.25, seed=seed)
    assert set(zip(*S.nonzero())) == {(0, 1)} | {(i, 0) for i in range(1, 6)}
    assert cf.tolist() == [1, -1, -1, -1, -1, -1]


@pytest.mark.parametrize("seed", range(12))
def test_pmis_f_rule_follows_dependence(seed):
    """An undecided point becomes F when it strongly depends on a new C point, not when it
    influences one.  0 depends on 1, and 1 (depended on by 0, 3, 4, 5: lambda 4) beats 0 (lambda 1,
    from 2) and becomes C; 0 depends on it and becomes F.  Were the rule taken the other way round,
    nothing would turn 0 into F (1 depends on nobody) and 0 would become C next to 1."""
    rp, ci, v = _directed(6, [(0, 1), (2, 0), (3, 1), (4, 1), (5, 1)])
    _, cf = oracle.pmis(rp, ci, v, theta=0.25, seed=seed)
    assert cf.tolist() == [-1, 1, -1, -1, -1, -1]


@pytest.mark.parametrize("seed", range(12))
def test_pmis_selection_looks_both_ways(seed):
    """A point joins the independent set of a round only when it beats every undecided neighbour in
    S + S^T, the points it depends on and the points that depend on it.  Here
    lambda = (1, 1, 1, 0, 3, 2, 4), so the outcome does not depend on the random part: round 1
    selects 6 (it beats 1, 2, 4); 1, 2, 4 depend on 6 and become F (3 influences nobody: F from the
    start); round 2 selects 5 over 0; round 3 selects 0, whose only neighbour 5 is now C.  Were the
    selection to look only at S_i, 0 (which depends on nobody) would be selected in round 1 and 5,
    depending on it, would become F."""
    edges = [(1, 5), (1, 6), (2, 5), (2, 6), (3, 1), (3, 2), (3, 4), (3, 6), (4, 6), (5, 0), (5, 4), (6, 4)]
    rp, ci, v = _directed(7, edges)
    _, cf = oracle.pmis(rp, ci, v, theta=0.25, seed=seed)
    assert cf.tolist() == [1, -1, -1, -1, -1, 1, 1]


@pytest.mark.parametrize("seed", range(40))
def test_pmis_brute_force_on_random_nonsymmetric_graphs(seed):
    """On random directed strength graphs of 12 points (S != S^T), checked point by point: every
    point is decided; a C point is strongly depended on by someone; an F point either influences
    nobody or strongly depends on a C point; and strong dependence among C points has no cycle.
    (A C point i that depends on a C point j was selected in an earlier round than j: had j been
    selected first, i would have become F in that round, and the two cannot be selected together,
    being neighbours.  So, unlike on symmetric graphs, C points need not be independent in S + S^T,
    but their dependences order them.)"""
    rng = np.random.default_rng(1000 + seed)
    n = 12
    edges = {(i, j) for i in range(n) for j in range(n) if i != j and rng.random() < 0.18}
    has_strong = {i for i, _ in edges}
    # weak entries only in rows that also hold a strong one (a row's threshold is relative to its
    # own largest entry)
    weak = {(i, j) for i in range(n) for j in range(n) if i != j and i in has_strong and rng.random() < 0.1}
    rp, ci, v = _directed(n, sorted(edges), sorted(weak))
    S, cf = oracle.pmis(rp, ci, v, theta=0.25, seed=seed)
    got = set(zip(*(x.tolist() for x in S.nonzero())))
    assert got == edges
    assert set(np.unique(cf).tolist()) <= {-1, 1}
    dep = {i: {j for (a, j) in edges if a == i} for i in range(n)}      # S_i: what i depends on
    infl = {i: {a for (a, j) in edges if j == i} for i in range(n)}     # S^T_i: who depends on i
    C = {i for i in range(n) if cf[i] == 1}
    for i in range(n):
        if cf[i] == 1:
            assert infl[i], i
        else:
            assert not infl[i] or dep[i] & C, (i, C)
    # no cycle of strong dependence among C points (repeatedly remove C points that depend on no
    # remaining C point)
    left = set(C)
    while left:
        sinks = {i for i in left if not dep[i] & left}
        assert sinks, ("dependence cycle among C points", left)
        left -= sinks
    if any(infl[i] for i in range(n)):
        assert C


# Two gas-present cells, markers (P, S, rho) = (2, 1, 0): the first reduction's F points are the two
# rho dofs 2 and 5.  Their rows couple to each other (an F-F entry) and to P and S dofs (off-F
# entries, which do not belong to A_ff).  Diagonal of dof 2 is negative to exercise the sign.
MGR_BLOCKS = np.array([
    # block (0, 0): rows dof 0..2, columns dof 0..2
    [[6.0, 0.5, 0.25], [0.5, 5.0, 0.4], [0.7, -0.9, -3.0]],
    # block (0, 1): rows dof 0..2, columns dof 3..5
    [[-1.0, 0.1, 0.0], [0.2, -0.5, 0.0], [0.3, 0.0, 0.5]],
    # block (1, 0)
    [[-1.2, 0.0, 0.0], [0.0, -0.4, 0.0], [0.0, 0.6, -1.0]],
    # block (1, 1)
    [[7.0, 0.3, -0.2], [0.1, 4.0, 0.0], [0.2, -1.1, 4.0]],
])
MGR_RP = np.array([0, 2, 4], np.int64)
MGR_CI = np.array([0, 1, 0, 1], np.int32)
MGR_MARKER = np.array([2, 1, 0, 2, 1, 0], np.int8)


@pytest.mark.parametrize("ftype,omega,expect", [
    # l1-Jacobi over A_ff's row: dof 2: a_22 = -3, the F-F entry a_25 = 0.5 -> 1/(-3 - 0.5) = -2/7;
    # dof 5: a_55 = 4, a_52 = -1 -> 1/(4 + 1) = 1/5.  The off-F entries (0.7, -0.9, 0.3 and 0.6,
    # -1.1) are not part of A_ff and do not enter.
    (1, 1.0, [-2 / 7, 1 / 5]),
    # omega-Jacobi: omega / a_ii
    (0, 0.7, [0.7 / -3.0, 0.7 / 4.0]),
])
def test_frelaxation_scaling_hand_computed(ftype, omega, expect):
    """F-relaxation scaling of the Algorithm's step (2) on the first reduction: l1-Jacobi sums the
    off-diagonal magnitudes of A_ff's row only, with the diagonal's sign; omega-Jacobi is
    omega / a_ii."""
    o = oracle.OracleMGR(MGR_RP, MGR_CI, MGR_BLOCKS.reshape(-1), MGR_MARKER, frelax_type=[ftype, 1, 1],
                         frelax_omega=[omega, 1.0, 1.0], amg_max_coarse=4)
    assert o.vec(oracle.VEC_F, 0).tolist() == [2, 5]
    minv = o.vec(oracle.VEC_MINV, 0)
    assert np.abs(minv - np.array(expect)).max() <= 1e-16, (minv, expect)


@pytest.mark.parametrize("smoother,omega,expect", [
    # l1-Jacobi over the whole row of the AMG level matrix, with the diagonal's sign:
    # row 3: 2.5 + (1 + 0.5 + 0.25) = 4.25; row 4: -2 - (0.5 + 1) = -3.5
    (1, 1.0, {3: 1 / 4.25, 4: 1 / -3.5}),
    # omega-Jacobi: omega / a_ii
    (0, 0.8, {3: 0.8 / 2.5, 4: 0.8 / -2.0}),
])
def test_amg_smoother_scaling_hand_computed(smoother, omega, expect):
    """AMG smoother scaling (section 6's coarse solve): l1-Jacobi 1 / (a_ii + sign(a_ii) sum_{j != i}
    |a_ij|) over the full row, omega-Jacobi omega / a_ii."""
    n = 10
    ent = []
    for i in range(n):
        ent.append((i, i, 3.0 + 0.1 * i))
        if i > 0:
            ent.append((i, i - 1, -1.0))
        if i < n - 1:
            ent.append((i, i + 1, -0.5))
    ent = [e for e in ent if e[0] not in (3, 4)]
    ent += [(3, 3, 2.5), (3, 2, -1.0), (3, 4, -0.5), (3, 7, 0.25),
            (4, 4, -2.0), (4, 3, 0.5), (4, 5, 1.0)]
    rp, ci, v = _csr(n, ent)
    amg = oracle.OracleAMG(rp, ci, v, amg_max_coarse=2, amg_max_levels=2, amg_smoother=smoother,
                           amg_omega=omega)
    dinv = amg.vec(oracle.VEC_AMG_DINV, 0)
    for i, x in expect.items():
        assert abs(dinv[i] - x) <= 1e-16, (i, dinv[i], x)
