"""GPU parity of the learned coarse space and the learned initial guess
against the FP64 oracle, through the C ABI.

Tolerances as for the other preconditioner stages: FP64 applications agree
to 1e-9 in norm (triangular and coarse solves amplify rounding by the
conditioning of the factors); solves reach the true relative residual 1e-8
and the oracle's solution to 1e-6."""
import numpy as np
import pytest

import bogen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AMG = dict(nu1=2, nu2=2, overcorr=1.3)


@pytest.fixture(scope="module")
def bo():
    import paper_1606_00556_gb300 as m
    m.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


@pytest.fixture(scope="module")
def ctx(bo):
    return bo.Context(0)


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _pair(bo, ctx, case, dims, precision=0):
    a = bogen.assemble(case)
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], a["val"])
    P = bo.Preconditioner(A, precision=precision, **AMG)
    return a, Ao, A, P


def _zc(n, seed, zero_tile=None, dims=None, tile=None):
    rng = np.random.default_rng(seed)
    z = rng.uniform(0.5, 2.0, n) * np.sign(rng.standard_normal(n))
    if zero_tile is not None:
        nx, ny, nz = dims
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        t = (i // tile[0] + (-(-nx // tile[0])) * (j // tile[1] + (-(-ny // tile[1])) * (k // tile[2]))).ravel()
        z[t == zero_tile] = 0.0
    return z


CASES = [((20, 20, 5), (8, 8, 3)), ((32, 7, 9), (16, 4, 4)), ((6, 5, 3), (6, 5, 3))]


@pytest.mark.parametrize("dims,tile", CASES)
@pytest.mark.parametrize("stage", ["amg", "cpr"])
def test_coarse_space_stage_matches_oracle(bo, ctx, dims, tile, stage):
    case = bogen.tiny_case(21, *dims)
    a, Ao, A, P = _pair(bo, ctx, case, dims)
    zc = _zc(Ao.nb, 3, zero_tile=1 if np.prod(dims) > 100 else None, dims=dims, tile=tile)
    P.set_coarse_space(_dev(zc), tile)
    so = {"amg": oracle.STAGE_AMG, "cpr": oracle.STAGE_CPR}[stage]
    sg = {"amg": bo.BO_STAGE_AMG, "cpr": bo.BO_STAGE_CPR}[stage]
    Po = oracle.cpr_prec(Ao, dims, amg=oracle.AmgParams(coarse_max=128, **AMG), stage=so)
    oracle.cpr_set_coarse(Po, zc, dims, tile)
    r = np.random.default_rng(9).standard_normal(Ao.n)
    z = P.apply(sg, _dev(r), torch.zeros(Ao.n, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = Po.apply(r)
    assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref)
    # removing the space gives back the plain stage
    P.set_coarse_space(None)
    Po2 = oracle.cpr_prec(Ao, dims, amg=oracle.AmgParams(coarse_max=128, **AMG), stage=so)
    z2 = P.apply(sg, _dev(r), torch.zeros(Ao.n, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.linalg.norm(z2 - Po2.apply(r)) <= 1e-9 * np.linalg.norm(ref)


def test_coarse_space_follows_matrix_update(bo, ctx):
    dims, tile = (20, 20, 5), (10, 10, 5)
    a0 = bogen.assemble(bogen.tiny_case(0))
    a1 = bogen.assemble(bogen.tiny_case(1))
    Ao1 = oracle.BsrMatrix(a1["rowptr"], a1["col"], a1["val"])
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a0["rowptr"], a0["col"], a0["val"])
    P = bo.Preconditioner(A, **AMG)
    zc = _zc(Ao1.nb, 5)
    P.set_coarse_space(_dev(zc), tile)
    A.update_values(a1["val"])
    P.update()
    Po = oracle.cpr_prec(Ao1, dims, amg=oracle.AmgParams(coarse_max=128, **AMG), stage=oracle.STAGE_AMG)
    oracle.cpr_set_coarse(Po, zc, dims, tile)
    r = np.random.default_rng(1).standard_normal(Ao1.n)
    z = P.apply(bo.BO_STAGE_AMG, _dev(r), torch.zeros(Ao1.n, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = Po.apply(r)
    assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref)


def test_coarse_space_rejects_bad_tiles(bo, ctx):
    dims = (20, 20, 5)
    a, Ao, A, P = _pair(bo, ctx, bogen.tiny_case(2, *dims), dims)
    zc = _dev(np.ones(Ao.nb))
    with pytest.raises(bo.BoError):
        P.set_coarse_space(zc, (0, 4, 4))
    with pytest.raises(bo.BoError):
        P.set_coarse_space(zc, (1, 1, 5))  # 400 tiles > 128
    # the failed calls leave no space behind
    r = _dev(np.random.default_rng(0).standard_normal(Ao.n))
    z = P.apply(bo.BO_STAGE_AMG, r, torch.zeros_like(r)).cpu().numpy()
    Po = oracle.cpr_prec(Ao, dims, amg=oracle.AmgParams(coarse_max=128, **AMG), stage=oracle.STAGE_AMG)
    ref = Po.apply(r.cpu().numpy())
    assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_with_coarse_space_matches_oracle(bo, ctx, precision):
    dims, tile = (20, 20, 5), (8, 8, 3)
    a, Ao, A, P = _pair(bo, ctx, bogen.tiny_case(7), dims, precision)
    x_ref, info = oracle.gmres(Ao, a["b"], tol=1e-13, maxit=5000, prec=oracle.ilu0_prec(Ao))
    assert info["converged"]
    P.set_coarse_space(_dev(x_ref[0::3]), tile)
    b = _dev(a["b"])
    x = torch.zeros_like(b)
    out = P.solve(b, x, tol=1e-8)
    xg = x.cpu().numpy()
    assert out["status"] == bo.BO_OK
    assert oracle.rel_residual(Ao, a["b"], xg) <= 1e-8
    assert np.linalg.norm(xg - x_ref) <= 1e-6 * np.linalg.norm(x_ref)


def test_learned_guess_keeps_good_and_drops_bad_guesses(bo, ctx):
    dims = (20, 20, 5)
    a, Ao, A, P = _pair(bo, ctx, bogen.tiny_case(8), dims)
    x_ref, _ = oracle.gmres(Ao, a["b"], tol=1e-13, maxit=5000, prec=oracle.ilu0_prec(Ao))
    V = Ao.nb
    scale = (100.0, 0.01, 0.01)
    pred = np.zeros((V, 4), np.float32)
    for k in range(3):
        pred[:, k] = x_ref[k::3] / scale[k]
    b = _dev(a["b"])
    x0 = torch.full_like(b, float("nan"))
    predg = torch.tensor(pred, device="cuda")
    assert P.learned_guess(b, predg, scale, 3, x0)
    want = np.zeros(3 * V)
    for k in range(3):
        want[k::3] = scale[k] * pred[:, k].astype(np.float64)
    np.testing.assert_array_equal(x0.cpu().numpy(), want)
    # the pressure-only guess keeps the saturations at zero
    assert P.learned_guess(b, predg, scale, 1, x0) in (True, False)
    got = x0.cpu().numpy()
    assert np.all(got[1::3] == 0.0) and np.all(got[2::3] == 0.0)
    # a guess further from the solution than zero is replaced by zero
    bad = torch.tensor(np.random.default_rng(0).standard_normal((V, 4)).astype(np.float32) * 1e4, device="cuda")
    x0.fill_(float("nan"))
    assert not P.learned_guess(b, bad, scale, 3, x0)
    assert torch.count_nonzero(x0).item() == 0
    # a solve from the (near-exact, FP32-rounded) kept guess needs fewer
    # iterations than one from zero, and reaches the same tolerance
    xz = torch.zeros_like(b)
    it0 = P.solve(b, xz, tol=1e-8)["iters"]
    assert P.learned_guess(b, predg, scale, 3, x0)
    info = P.solve(b, x0, tol=1e-8, x0_is_zero=False)
    assert info["status"] == bo.BO_OK and info["iters"] < it0
    assert oracle.rel_residual(Ao, a["b"], x0.cpu().numpy()) <= 1e-8
