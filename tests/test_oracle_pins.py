"""Pins of the FP64 oracle against what mathematics fixes independently of
its code: dense products and LAPACK solves, the defining property of ILU(0)
((L U)_ij = A_ij on the pattern), exactness of ILU(0) on block-tridiagonal
matrices, the paper's form of the Quasi-IMPES operator multiplied back,
Galerkin coarse operators against explicit P^T A P, symmetry of a symmetric
V-cycle, and GMRES and BiCGSTAB identities."""
import numpy as np
import pytest

import bogen
import oracle
from oracle import BsrMatrix


def _random_bsr(nx, ny, nz, seed, diag_boost=6.0):
    rng = np.random.default_rng(seed)
    rowptr, col = bogen.pattern(nx, ny, nz)
    val = rng.standard_normal((col.size, 3, 3))
    for i in range(rowptr.size - 1):
        for e in range(rowptr[i], rowptr[i + 1]):
            if col[e] == i:
                val[e] += diag_boost * np.eye(3)
    return BsrMatrix(rowptr, col, val)


def _tiny_system(seed=0, dims=(20, 20, 5)):
    c = bogen.tiny_case(seed, *dims)
    a = bogen.assemble(c)
    return BsrMatrix(a["rowptr"], a["col"], a["val"]), a["b"]


def _pattern_set(A):
    s = set()
    for i in range(A.nb):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            s.add((i, int(A.col[e])))
    return s


def test_spmv_matches_dense_product():
    A = _random_bsr(5, 4, 3, 1)
    x = np.random.default_rng(2).standard_normal(A.n)
    assert np.allclose(oracle.spmv(A, x), A.to_dense() @ x, rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("nthreads", [1, 3, 7])
def test_threaded_spmv_matches_dense_product(nthreads):
    # the CPU bandwidth baseline: the dense product, and bitwise the serial
    # SpMV (same sums per row, rows split over threads)
    A = _random_bsr(6, 5, 3, 4)
    x = np.random.default_rng(3).standard_normal(A.n)
    y = oracle.spmv_threads(A, x, nthreads)
    assert np.allclose(y, A.to_dense() @ x, rtol=1e-14, atol=1e-13)
    assert np.array_equal(y, oracle.spmv(A, x))


def test_qi_operator_multiplied_back_gives_A():
    # paper Sec. 3.2: D_QI = [[I, D_ps D_ss^-1, 0], [0, I, 0], [0, 0, I]] with
    # D_ps = diag(A_ps), D_ss = diag(A_ss); built here as a dense matrix in
    # the cell-interleaved ordering, D_QI (D_QI^{-1} A) must give A back
    A, _ = _tiny_system(0, (6, 5, 3))
    At, w = oracle.qi_decouple(A)
    Ad = A.to_dense()
    D = np.eye(A.n)
    for i in range(A.nb):
        blk = Ad[3 * i:3 * i + 3, 3 * i:3 * i + 3]
        D[3 * i, 3 * i + 1] = blk[0, 1] / blk[1, 1]
        D[3 * i, 3 * i + 2] = blk[0, 2] / blk[2, 2]
        # the tiny case's pressure pivots stay positive: pure Quasi-IMPES
        assert blk[0, 0] - D[3 * i, 3 * i + 1] * blk[1, 0] - D[3 * i, 3 * i + 2] * blk[2, 0] > 0
    assert np.allclose(D @ At.to_dense(), Ad, rtol=1e-13, atol=1e-10 * np.abs(Ad).max())
    assert np.allclose(w[:, 0], 1.0) and np.allclose(-w[:, 1], np.diag(D, 1)[0::3])


def test_flooded_injector_cells_take_exact_local_decoupling():
    # an injector cell swept to residual oil (So = s_orw): the oil row barely
    # depends on pressure and the water pivot turns negative, so Quasi-IMPES
    # would give a negative pressure pivot; there the decoupled row is row 0
    # of A_ii^{-1} A, whose diagonal block row is exactly e_0
    case = bogen.waterflood_case(12, 12, 4, seed=3, day=0, corr=(2, 2, 1), front0=4.0)
    a = bogen.assemble(case)
    A = BsrMatrix(a["rowptr"], a["col"], a["val"])
    At, g = oracle.qi_decouple(A)
    n_fallback = 0
    for i in range(A.nb):
        e = [e for e in range(A.rowptr[i], A.rowptr[i + 1]) if A.col[e] == i][0]
        blk = A.val[e]
        qi = blk[0, 0] - blk[0, 1] / blk[1, 1] * blk[1, 0] - blk[0, 2] / blk[2, 2] * blk[2, 0]
        if qi > 0:
            assert np.allclose(g[i], [1.0, -blk[0, 1] / blk[1, 1], -blk[0, 2] / blk[2, 2]])
        else:
            n_fallback += 1
            assert np.allclose(g[i], np.linalg.inv(blk)[0], rtol=1e-12)
            assert np.allclose(At.val[e][0], [1.0, 0.0, 0.0], atol=1e-12)
        assert At.val[e][0, 0] > 0
    assert n_fallback > 0


def test_qi_removes_local_saturation_coupling_of_pressure_row():
    # D_ss = diag(A_ss) is exact when the cell's saturation block is diagonal:
    # then the decoupled pressure row no longer sees the cell's own saturations
    A, _ = _tiny_system(1)
    for i in range(A.nb):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            if A.col[e] == i:
                A.val[e][1, 2] = 0.0
                A.val[e][2, 1] = 0.0
    At, _ = oracle.qi_decouple(A)
    for i in range(A.nb):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            if At.col[e] == i:
                scale = np.abs(A.val[e]).max()
                assert abs(At.val[e][0, 1]) <= 1e-12 * scale
                assert abs(At.val[e][0, 2]) <= 1e-12 * scale
                # saturation rows are left as they were
                assert np.array_equal(At.val[e][1:], A.val[e][1:])


def _lu_dense(LU: BsrMatrix):
    bs = LU.bs
    L = np.eye(LU.n)
    U = np.zeros((LU.n, LU.n))
    for i in range(LU.nb):
        for e in range(LU.rowptr[i], LU.rowptr[i + 1]):
            j = LU.col[e]
            blk = LU.val[e]
            if j < i:
                L[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = blk
            else:
                U[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = blk
    return L, U


@pytest.mark.parametrize("order", ["natural", "red_black"])
def test_ilu0_defining_property(order):
    # ILU(0) is characterised by (L U)_ij = A_ij for every (i, j) of the pattern
    A = _random_bsr(4, 4, 3, 5)
    if order == "red_black":
        A = oracle.permute(A, oracle.red_black_perm(4, 4, 3))
    LU = oracle.ilu0(A)
    L, U = _lu_dense(LU)
    P = L @ U
    Ad = A.to_dense()
    for (i, j) in _pattern_set(A):
        assert np.allclose(P[3 * i:3 * i + 3, 3 * j:3 * j + 3], Ad[3 * i:3 * i + 3, 3 * j:3 * j + 3], atol=1e-12)
    # and the solve applies (L U)^{-1}
    r = np.random.default_rng(0).standard_normal(A.n)
    assert np.allclose(oracle.ilu0_solve(LU, r), np.linalg.solve(P, r), rtol=1e-10, atol=1e-12)


def test_ilu0_exact_on_block_tridiagonal_column():
    # a 1x1xnz column gives a block tridiagonal matrix: ILU(0) drops no fill
    A = _random_bsr(1, 1, 9, 7, diag_boost=1.0)
    LU = oracle.ilu0(A)
    r = np.random.default_rng(1).standard_normal(A.n)
    assert np.allclose(oracle.ilu0_solve(LU, r), np.linalg.solve(A.to_dense(), r), rtol=1e-11, atol=1e-12)


def test_red_black_black_diagonal_update_is_schur_complement():
    # in red-black order red rows have no lower part, and every black pivot
    # block equals D_b - sum_r A_br D_r^{-1} A_rb over its red neighbours
    nx, ny, nz = 4, 3, 2
    A = _random_bsr(nx, ny, nz, 11)
    perm = oracle.red_black_perm(nx, ny, nz)
    B = oracle.permute(A, perm)
    LU = oracle.ilu0(B)
    nred = int(np.sum([((c % nx) + (c // nx) % ny + c // (nx * ny)) % 2 == 0 for c in range(nx * ny * nz)]))
    Bd = B.to_dense()
    blk = lambda M, i, j: M[3 * i:3 * i + 3, 3 * j:3 * j + 3]
    for b in range(nred, B.nb):
        S = blk(Bd, b, b).copy()
        for r in range(nred):
            if np.any(blk(Bd, b, r)):
                S -= blk(Bd, b, r) @ np.linalg.solve(blk(Bd, r, r), blk(Bd, r, b))
        e = [e for e in range(LU.rowptr[b], LU.rowptr[b + 1]) if LU.col[e] == b][0]
        assert np.allclose(LU.val[e], S, rtol=1e-12, atol=1e-12)


def test_permute_matches_dense_permutation():
    A = _random_bsr(4, 3, 2, 3)
    perm = oracle.red_black_perm(4, 3, 2)
    B = oracle.permute(A, perm)
    P = np.zeros((A.n, A.n))
    for new, old in enumerate(perm):
        P[3 * new:3 * new + 3, 3 * old:3 * old + 3] = np.eye(3)
    assert np.allclose(B.to_dense(), P @ A.to_dense() @ P.T)
    for i in range(B.nb):
        assert np.all(np.diff(B.col[B.rowptr[i]:B.rowptr[i + 1]]) > 0)


def test_dense_solve_matches_lapack():
    rng = np.random.default_rng(4)
    M = rng.standard_normal((50, 50))
    b = rng.standard_normal(50)
    assert np.allclose(oracle.dense_solve(M, b), np.linalg.solve(M, b), rtol=1e-11)
    with pytest.raises(ArithmeticError):
        oracle.dense_solve(np.zeros((3, 3)), np.ones(3))


def test_rel_residual_matches_numpy():
    A = _random_bsr(4, 4, 2, 9)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(A.n)
    b = rng.standard_normal(A.n)
    ref = np.linalg.norm(b - A.to_dense() @ x) / np.linalg.norm(b)
    assert oracle.rel_residual(A, b, x) == pytest.approx(ref, rel=1e-13)


# ----------------------------------------------------------------- GMRES
def test_gmres_identity_one_iteration():
    nb = 10
    rowptr = np.arange(nb + 1, dtype=np.int32)
    col = np.arange(nb, dtype=np.int32)
    val = np.tile(np.eye(3), (nb, 1, 1))
    I = BsrMatrix(rowptr, col, val)
    b = np.random.default_rng(0).standard_normal(3 * nb)
    x, info = oracle.gmres(I, b, tol=1e-12)
    assert info["iters"] == 1 and np.allclose(x, b, rtol=1e-15)


def test_gmres_zero_budget_returns_initial_guess():
    A, b = _tiny_system(0, (4, 4, 2))
    x0 = np.random.default_rng(1).standard_normal(A.n)
    x, info = oracle.gmres(A, b, x0=x0, maxit=0)
    assert np.array_equal(x, x0) and info["iters"] == 0 and not info["converged"]


@pytest.mark.parametrize("prec", ["none", "ilu0", "cpr"])
def test_gmres_matches_lapack_on_small_black_oil(prec):
    dims = (6, 5, 4)
    A, b = _tiny_system(2, dims)
    if prec == "none":  # unpreconditioned: a well-conditioned random system
        A = _random_bsr(*dims, 2)
    P = None
    if prec == "ilu0":
        P = oracle.ilu0_prec(A)
    elif prec == "cpr":
        P = oracle.cpr_prec(A, dims)
    x, info = oracle.gmres(A, b, tol=1e-13, maxit=2000, prec=P)
    ref = np.linalg.solve(A.to_dense(), b)
    assert info["converged"]
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-10


def test_gmres_tiny_case_true_residual():
    A, b = _tiny_system(0)
    P = oracle.ilu0_prec(A)
    x, info = oracle.gmres(A, b, tol=1e-8, prec=P)
    assert info["converged"] and oracle.rel_residual(A, b, x) <= 1e-8


# ----------------------------------------------------------------- BiCGSTAB
def test_bicgstab_identity_one_iteration():
    nb = 10
    rowptr = np.arange(nb + 1, dtype=np.int32)
    col = np.arange(nb, dtype=np.int32)
    I = BsrMatrix(rowptr, col, np.tile(np.eye(3), (nb, 1, 1)))
    b = np.random.default_rng(0).standard_normal(3 * nb)
    x, info = oracle.bicgstab(I, b, tol=1e-12)
    assert info["converged"] and info["iters"] == 1 and np.allclose(x, b, rtol=1e-15)


def test_bicgstab_exact_preconditioner_one_iteration():
    # ILU(0) of a block-tridiagonal column is its exact LU: with M = A the
    # first BiCG half step gives alpha = 1 and s = 0
    A = _random_bsr(1, 1, 9, 7, diag_boost=1.0)
    b = np.random.default_rng(2).standard_normal(A.n)
    x, info = oracle.bicgstab(A, b, tol=1e-12, prec=oracle.ilu0_prec(A))
    assert info["converged"] and info["iters"] == 1
    assert np.allclose(x, np.linalg.solve(A.to_dense(), b), rtol=1e-11, atol=1e-12)


def test_bicgstab_zero_budget_and_zero_rhs():
    A, b = _tiny_system(0, (4, 4, 2))
    x0 = np.random.default_rng(1).standard_normal(A.n)
    x, info = oracle.bicgstab(A, b, x0=x0, maxit=0)
    assert np.array_equal(x, x0) and info["iters"] == 0 and not info["converged"]
    x, info = oracle.bicgstab(A, np.zeros(A.n))
    assert info["converged"] and info["iters"] == 0 and not x.any()


@pytest.mark.parametrize("prec", ["none", "ilu0", "cpr"])
def test_bicgstab_matches_lapack_on_small_black_oil(prec):
    dims = (6, 5, 4)
    A, b = _tiny_system(2, dims)
    if prec == "none":
        A = _random_bsr(*dims, 2)
    P = None
    if prec == "ilu0":
        P = oracle.ilu0_prec(A)
    elif prec == "cpr":
        P = oracle.cpr_prec(A, dims)
    x, info = oracle.bicgstab(A, b, tol=1e-13, maxit=2000, prec=P)
    ref = np.linalg.solve(A.to_dense(), b)
    assert info["converged"]
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-10


def test_bicgstab_skew_matrix_reports_breakdown():
    # for a skew-symmetric A and shadow vector r0, (r0, A r0) = 0: the BiCG
    # step cannot be taken, and a restart cannot change that
    S = np.array([[0.0, 1.0, 2.0, 0.5, 0.0, 1.0], [-1.0, 0.0, 1.0, 0.0, 2.0, 0.0],
                  [-2.0, -1.0, 0.0, 1.0, 0.0, 3.0], [-0.5, 0.0, -1.0, 0.0, 1.0, 0.0],
                  [0.0, -2.0, 0.0, -1.0, 0.0, 1.0], [-1.0, 0.0, -3.0, 0.0, -1.0, 0.0]])
    assert abs(np.linalg.det(S)) > 1e-3
    rowptr = np.array([0, 2, 4], dtype=np.int32)
    col = np.array([0, 1, 0, 1], dtype=np.int32)
    val = np.stack([S[0:3, 0:3], S[0:3, 3:6], S[3:6, 0:3], S[3:6, 3:6]])
    A = BsrMatrix(rowptr, col, val)
    x, info = oracle.bicgstab(A, np.arange(1.0, 7.0), maxit=50)
    assert info["breakdown"] and not info["converged"] and info["iters"] == 0


def test_cpr_bicgstab_reaches_paper_tolerance_tiny_case():
    A, b = _tiny_system(0)
    x, info = oracle.bicgstab(A, b, tol=1e-8, prec=oracle.cpr_prec(A, (20, 20, 5)))
    assert info["converged"] and oracle.rel_residual(A, b, x) <= 1e-8


# ----------------------------------------------------------------- AMG
def _laplacian(nx, ny, nz, coef=None, shift=0.0):
    """Scalar 7-point matrix with face weights coef(c, d) (symmetric)."""
    rowptr, col = bogen.pattern(nx, ny, nz)
    val = np.zeros(col.size)
    N = nx * ny * nz
    rng = np.random.default_rng(0)
    wts = {}
    for i in range(N):
        for e in range(rowptr[i], rowptr[i + 1]):
            j = col[e]
            if j != i:
                key = (min(i, j), max(i, j))
                if key not in wts:
                    wts[key] = 1.0 if coef is None else coef(rng)
                val[e] = -wts[key]
    for i in range(N):
        s = 0.0
        for e in range(rowptr[i], rowptr[i + 1]):
            if col[e] != i:
                s -= val[e]
        for e in range(rowptr[i], rowptr[i + 1]):
            if col[e] == i:
                val[e] = s + shift
    return rowptr, col, val


def _csr_dense(rp, c, v):
    n = rp.size - 1
    M = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            M[i, c[e]] += v[e]
    return M


def _aggregation_P(nx, ny, nz):
    cx, cy, cz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    P = np.zeros((nx * ny * nz, cx * cy * cz))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                P[i + nx * (j + ny * k), i // 2 + cx * (j // 2 + cy * (k // 2))] = 1.0
    return P


def test_amg_galerkin_equals_explicit_triple_product():
    dims = (7, 6, 5)  # odd sizes: aggregates of 1 cell at the far faces
    rp, c, v = _laplacian(*dims, coef=lambda r: np.exp(r.normal(0, 1)), shift=0.3)
    amg = oracle.Amg(rp, c, v, dims, oracle.AmgParams(coarse_max=8))
    assert amg.nlevels >= 2
    A0 = _csr_dense(rp, c, v)
    P = _aggregation_P(*dims)
    A1 = _csr_dense(*amg.level_matrix(1))
    assert amg.dims(1) == (4, 3, 3)
    assert np.allclose(A1, P.T @ A0 @ P, rtol=1e-13, atol=1e-13)


def test_amg_galerkin_on_a_nonsymmetric_matrix():
    # the decoupled pressure matrix is not symmetric (upwinded mobilities and
    # the Quasi-IMPES weights), so P^T A P must not come out as P^T A^T P
    dims = (6, 5, 3)
    rp, c, v = _laplacian(*dims)
    rng = np.random.default_rng(11)
    v = v.copy()
    for i in range(rp.size - 1):
        off = [e for e in range(rp[i], rp[i + 1]) if c[e] != i]
        v[off] *= np.exp(rng.normal(0.0, 0.5, len(off)))
        for e in range(rp[i], rp[i + 1]):
            if c[e] == i:
                v[e] = -v[off].sum() + 0.2
    A0 = _csr_dense(rp, c, v)
    assert not np.allclose(A0, A0.T)
    amg = oracle.Amg(rp, c, v, dims, oracle.AmgParams(coarse_max=8))
    P = _aggregation_P(*dims)
    A1 = _csr_dense(*amg.level_matrix(1))
    assert np.allclose(A1, P.T @ A0 @ P, rtol=1e-13, atol=1e-13)


def test_amg_coarse_laplacian_keeps_zero_row_sums_and_symmetry():
    dims = (8, 8, 4)
    rp, c, v = _laplacian(*dims)
    amg = oracle.Amg(rp, c, v, dims, oracle.AmgParams(coarse_max=4))
    for l in range(1, amg.nlevels):
        M = _csr_dense(*amg.level_matrix(l))
        assert np.abs(M.sum(axis=1)).max() <= 1e-12
        assert np.allclose(M, M.T)
        # still a 7-point stencil on the coarse grid
        assert max(np.count_nonzero(M[i]) for i in range(M.shape[0])) <= 7


def test_amg_single_level_is_exact_solve():
    dims = (5, 4, 3)
    rp, c, v = _laplacian(*dims, shift=0.5)
    amg = oracle.Amg(rp, c, v, dims, oracle.AmgParams(coarse_max=1000))
    assert amg.nlevels == 1
    f = np.random.default_rng(3).standard_normal(60)
    assert np.allclose(amg.vcycle(f), np.linalg.solve(_csr_dense(rp, c, v), f), rtol=1e-12)


@pytest.mark.parametrize("overcorr", [1.0, 1.6])
def test_amg_symmetric_vcycle_is_symmetric_operator(overcorr):
    # red-black pre-smoothing mirrored by black-red post-smoothing makes the
    # V-cycle a symmetric linear operator for a symmetric matrix
    dims = (6, 6, 4)
    rp, c, v = _laplacian(*dims, coef=lambda r: np.exp(r.normal(0, 1)), shift=0.1)
    amg = oracle.Amg(rp, c, v, dims, oracle.AmgParams(coarse_max=10, overcorr=overcorr))
    n = 144
    M = np.stack([amg.vcycle(np.eye(n)[i]) for i in range(n)], axis=1)
    assert np.allclose(M, M.T, rtol=1e-11, atol=1e-13)


def _two_level(dims, nu1, nu2, smoother, overcorr):
    rp, c, v = _laplacian(*dims, coef=lambda r: np.exp(r.normal(0, 1)), shift=0.2)
    ncoarse = np.prod([(d + 1) // 2 for d in dims])
    prm = oracle.AmgParams(smoother=smoother, nu1=nu1, nu2=nu2, overcorr=overcorr, coarse_max=int(ncoarse))
    amg = oracle.Amg(rp, c, v, dims, prm)
    assert amg.nlevels == 2
    A = _csr_dense(rp, c, v)
    P = _aggregation_P(*dims)
    return amg, A, P, prm


def test_amg_two_level_without_smoothing_is_scaled_coarse_correction():
    # with no sweeps a two-level cycle is x = s P (P^T A P)^{-1} P^T f
    dims = (6, 5, 4)
    amg, A, P, prm = _two_level(dims, 0, 0, oracle.SMOOTHER_RBGS, 1.6)
    f = np.random.default_rng(8).standard_normal(A.shape[0])
    ref = prm.overcorr * P @ np.linalg.solve(P.T @ A @ P, P.T @ f)
    assert np.allclose(amg.vcycle(f), ref, rtol=1e-12, atol=1e-14)


def test_amg_two_level_jacobi_cycle_closed_form():
    # one damped-Jacobi pre-sweep from zero, then the coarse correction:
    # x1 = w D^{-1} f;  x = x1 + s P A_c^{-1} P^T (f - A x1)
    dims = (5, 4, 4)
    amg, A, P, prm = _two_level(dims, 1, 0, oracle.SMOOTHER_JACOBI, 1.3)
    f = np.random.default_rng(9).standard_normal(A.shape[0])
    x1 = prm.omega * f / np.diag(A)
    ref = x1 + prm.overcorr * P @ np.linalg.solve(P.T @ A @ P, P.T @ (f - A @ x1))
    assert np.allclose(amg.vcycle(f), ref, rtol=1e-12, atol=1e-14)


def test_amg_two_level_gauss_seidel_cycle_closed_form():
    # one red-black Gauss-Seidel pre-sweep and one black-red post-sweep: each
    # half sweep solves its colour's rows exactly with the other colour fixed
    dims = (4, 4, 3)
    amg, A, P, prm = _two_level(dims, 1, 1, oracle.SMOOTHER_RBGS, 1.3)
    n = A.shape[0]
    red = np.array([((c % 4) + (c // 4) % 4 + c // 16) % 2 == 0 for c in range(n)])

    def half(x, f, colour):
        x = x.copy()
        S = colour
        O = ~colour
        x[S] = (f[S] - A[np.ix_(S, O)] @ x[O]) / np.diag(A)[S]
        return x

    f = np.random.default_rng(10).standard_normal(n)
    x = half(half(np.zeros(n), f, red), f, ~red)
    x = x + prm.overcorr * P @ np.linalg.solve(P.T @ A @ P, P.T @ (f - A @ x))
    x = half(half(x, f, ~red), f, red)
    assert np.allclose(amg.vcycle(f), x, rtol=1e-12, atol=1e-14)


def test_amg_vcycle_iteration_converges_to_solution():
    dims = (16, 16, 8)
    rp, c, v = _laplacian(*dims, coef=lambda r: np.exp(r.normal(0, 1.5)), shift=1e-3)
    amg = oracle.Amg(rp, c, v, dims, oracle.AmgParams(coarse_max=64))
    A = _csr_dense(rp, c, v)
    f = np.random.default_rng(1).standard_normal(A.shape[0])
    ref = np.linalg.solve(A, f)
    x = np.zeros_like(f)
    for _ in range(250):
        x = x + amg.vcycle(f - A @ x)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8


# ----------------------------------------------------------------- CPR
def test_cpr_exact_when_local_solver_is_exact():
    # on a 1x1xnz column natural-order ILU(0) is an exact factorisation, so
    # Alg. 2 returns A^{-1} v regardless of the AMG stage
    dims = (1, 1, 12)
    rng = np.random.default_rng(0)
    c = bogen.uniform_case(*dims)
    c.x = c.xn * rng.uniform(0.95, 1.05, 3 * c.N)
    a = bogen.assemble(c)
    A = BsrMatrix(a["rowptr"], a["col"], a["val"])
    P = oracle.cpr_prec(A, dims, ordering=oracle.ORDER_NATURAL)
    v = rng.standard_normal(A.n)
    assert np.allclose(P.apply(v), np.linalg.solve(A.to_dense(), v), rtol=1e-9)


def test_cpr_stages_compose_as_alg2():
    # the full preconditioner equals the composition of its stages:
    # x1 = R f; x2 = x1 + Pi_p AMG Pi_r (f - At x1); x3 = x2 + R (f - At x2)
    dims = (4, 4, 3)
    A, _ = _tiny_system(3, dims)
    At, w = oracle.qi_decouple(A)
    Rp = oracle.cpr_prec(A, dims, stage=oracle.STAGE_ILU)
    Mp = oracle.cpr_prec(A, dims, stage=oracle.STAGE_AMG)
    Cp = oracle.cpr_prec(A, dims, stage=oracle.STAGE_CPR_DECOUPLED)
    Full = oracle.cpr_prec(A, dims, stage=oracle.STAGE_CPR)
    f = np.random.default_rng(2).standard_normal(A.n)
    Atd = At.to_dense()
    x1 = Rp.apply(f)
    x2 = x1 + Mp.apply(f - Atd @ x1)
    x3 = x2 + Rp.apply(f - Atd @ x2)
    assert np.allclose(Cp.apply(f), x3, rtol=1e-12, atol=1e-14)
    # the full form decouples its input first: z = CPR(D_QI^{-1} v)
    fd = f.copy()
    fd[0::3] = w[:, 0] * f[0::3] + w[:, 1] * f[1::3] + w[:, 2] * f[2::3]
    assert np.allclose(Full.apply(f), Cp.apply(fd), rtol=1e-12, atol=1e-14)


def test_cpr_gmres_reaches_paper_tolerance_tiny_case():
    A, b = _tiny_system(0)
    P = oracle.cpr_prec(A, (20, 20, 5))
    x, info = oracle.gmres(A, b, tol=1e-8, prec=P)
    assert info["converged"] and oracle.rel_residual(A, b, x) <= 1e-8
