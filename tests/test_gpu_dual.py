"""GPU parity of the dual-porosity solve against the FP64 oracle (plain
GMRES + ILU(0) on the full 2N-block-row system, or dense LU), through the C
ABI.  At tol 1e-8 the full system's true FP64 residual must be <= 1e-8
(checked by the oracle's compensated residual).  The error bound that
residual gives is kappa * 1e-8, and these systems are worse conditioned than
the single-porosity ones (the matrix continuum stores fluid that moves
through the far more conductive fractures), so the solution is compared
with the oracle's to 1e-6 after a solve to 1e-11."""
import numpy as np
import pytest

import oracle
from bogen import dual as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def _oracle_solution(a):
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    if Ao.n <= 3000:
        return Ao, oracle.dense_solve(Ao.to_dense(), a["b"])
    x, info = oracle.gmres(Ao, a["b"], tol=1e-13, maxit=20000, prec=oracle.ilu0_prec(Ao))
    assert info["converged"]
    return Ao, x


@pytest.mark.parametrize("dims", [(8, 6, 4), (20, 20, 5), (32, 7, 9)])
@pytest.mark.parametrize("precision", [0, 1])
def test_dual_solve_matches_oracle(bo, ctx, dims, precision):
    case = D.dual_case(sum(dims), *dims)
    a = D.assemble_dual(case)
    Ao, x_ref = _oracle_solution(a)
    dp = bo.DualPorosity(ctx, *dims, a["rowptr"], a["col"], a["val"])
    P = bo.Preconditioner(dp.fracture_matrix, precision=precision)
    b = torch.tensor(a["b"], device="cuda")
    x = torch.zeros_like(b)
    info = dp.solve(P, b, x, tol=1e-8)
    xg = x.cpu().numpy()
    assert info["status"] == bo.BO_OK and info["iters"] > 0
    assert oracle.rel_residual(Ao, a["b"], xg) <= 1e-8
    assert info["true_rel_res"] <= 1e-8
    x.zero_()
    info = dp.solve(P, b, x, tol=1e-11)
    xg = x.cpu().numpy()
    assert info["status"] == bo.BO_OK
    assert oracle.rel_residual(Ao, a["b"], xg) <= 1e-11
    assert np.linalg.norm(xg - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    # the matrix continuum is recovered, not left at zero
    N = int(np.prod(dims))
    assert np.linalg.norm(xg[3 * N:]) > 0


def test_dual_update_values(bo, ctx):
    dims = (8, 6, 4)
    a0 = D.assemble_dual(D.dual_case(1, *dims))
    a1 = D.assemble_dual(D.dual_case(2, *dims))
    dp = bo.DualPorosity(ctx, *dims, a0["rowptr"], a0["col"], a0["val"])
    P = bo.Preconditioner(dp.fracture_matrix)
    dp.update_values(torch.tensor(a1["val"].reshape(-1), device="cuda"))
    P.update()
    b = torch.tensor(a1["b"], device="cuda")
    x = torch.zeros_like(b)
    info = dp.solve(P, b, x, tol=1e-11)
    Ao, x_ref = _oracle_solution(a1)
    assert info["status"] == bo.BO_OK
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-6 * np.linalg.norm(x_ref)


def test_dual_pattern_errors(bo, ctx):
    dims = (4, 3, 2)
    a = D.assemble_dual(D.dual_case(0, *dims))
    N = int(np.prod(dims))
    col = a["col"].copy()
    # a matrix node coupled to another cell's fracture node
    col[a["rowptr"][N]] = 1 if col[a["rowptr"][N]] != 1 else 2
    with pytest.raises(bo.BoError) as e:
        bo.DualPorosity(ctx, *dims, a["rowptr"], col, a["val"])
    assert e.value.status == bo.BO_ERR_PATTERN
    # a singular matrix-node block
    val = a["val"].copy()
    rp = a["rowptr"]
    for e_ in range(rp[N + 3], rp[N + 4]):
        if a["col"][e_] == N + 3:
            val[e_] = 0.0
    with pytest.raises(bo.BoError) as e:
        bo.DualPorosity(ctx, *dims, a["rowptr"], a["col"], val)
    assert e.value.status == bo.BO_ERR_BREAKDOWN
    val = a["val"].copy()
    val[5, 1, 1] = np.nan
    with pytest.raises(bo.BoError) as e:
        bo.DualPorosity(ctx, *dims, a["rowptr"], a["col"], val)
    assert e.value.status == bo.BO_ERR_NONFINITE


def test_dual_batched_solve_matches_single_solves(bo, ctx):
    # an ensemble of dual-porosity realisations of uneven size solved
    # together: each full FP64 residual <= 1e-8 and each solution bitwise the
    # single solve's (the same kernels, one system per stream of the pool)
    dims_list = [(8, 6, 4), (20, 20, 5), (12, 10, 6), (32, 7, 9)]
    dps, precs, bs, xs, singles, refs = [], [], [], [], [], []
    for k, dims in enumerate(dims_list):
        a = D.assemble_dual(D.dual_case(40 + k, *dims))
        dp = bo.DualPorosity(ctx, *dims, a["rowptr"], a["col"], a["val"])
        P = bo.Preconditioner(dp.fracture_matrix, precision=bo.BO_PREC_FP32)
        b = torch.tensor(a["b"], device="cuda")
        x1 = torch.zeros_like(b)
        i1 = dp.solve(P, b, x1, tol=1e-8)
        dps.append(dp), precs.append(P), bs.append(b), xs.append(torch.zeros_like(b))
        singles.append((x1, i1)), refs.append(a)
    rc, infos = bo.bo_dp_solve_batched(dps, precs, bs, xs, tol=1e-8)
    assert rc == bo.BO_OK
    for x, inf, (x1, i1), a in zip(xs, infos, singles, refs):
        Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
        assert inf["status"] == bo.BO_OK and inf["true_rel_res"] <= 1e-8
        assert oracle.rel_residual(Ao, a["b"], x.cpu().numpy()) <= 1e-8
        if i1["iters"] == inf["iters"]:
            assert torch.equal(x, x1)
