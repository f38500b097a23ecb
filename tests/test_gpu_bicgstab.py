"""BiCGSTAB with the CPR preconditioner on the GPU (bo_solve_bicgstab, the
solver of the paper's scalability runs) against the FP64 oracle, through
the C ABI, with the bars of every solve: true relative residual <= 1e-8 by
the oracle's compensated FP64 residual, and ||x - x_ref|| <= 1e-6 ||x_ref||
against the oracle solved to 1e-13.  The oracle's own right-preconditioned
BiCGSTAB with the same CPR reaches the tolerance in a comparable number of
iterations."""
import numpy as np
import pytest

import bogen
import oracle

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


def _setup(bo, ctx, case, dims, precision):
    a = bogen.assemble(case)
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], a["val"])
    P = bo.Preconditioner(A, precision=precision)
    return a, Ao, A, P


def _xref(Ao, b):
    x, info = oracle.gmres(Ao, b, tol=1e-13, maxit=5000, prec=oracle.ilu0_prec(Ao))
    assert info["converged"]
    return x


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_bicgstab_tiny_matches_oracle(bo, ctx, seed, precision):
    dims = (20, 20, 5)
    a, Ao, A, P = _setup(bo, ctx, bogen.tiny_case(seed), dims, precision)
    b = torch.tensor(a["b"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = P.solve_bicgstab(b, x, tol=1e-8)
    xg = x.cpu().numpy()
    assert info["status"] == bo.BO_OK and info["iters"] > 0, info
    assert oracle.rel_residual(Ao, a["b"], xg) <= 1e-8
    assert info["true_rel_res"] <= 1e-8
    xr = _xref(Ao, a["b"])
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-6
    if precision == 0:
        # the same preconditioner in the oracle's BiCGSTAB (red-black ILU(0),
        # the same AMG): iteration counts agree up to rounding-driven drift
        _, oinfo = oracle.bicgstab(Ao, a["b"], tol=1e-8, prec=oracle.cpr_prec(Ao, dims))
        assert oinfo["converged"] and abs(info["iters"] - oinfo["iters"]) <= 2 + 0.3 * oinfo["iters"], (info, oinfo)


def test_bicgstab_edge_cases(bo, ctx):
    dims = (20, 20, 5)
    a, Ao, A, P = _setup(bo, ctx, bogen.tiny_case(2), dims, 1)
    n = Ao.n
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    info = P.solve_bicgstab(torch.zeros(n, dtype=torch.float64, device="cuda"), x)
    assert info["status"] == bo.BO_OK and float(x.abs().max()) == 0.0
    b = torch.tensor(a["b"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = P.solve_bicgstab(b, x, maxit=1)
    assert info["status"] == bo.BO_ERR_NOT_CONVERGED and info["iters"] == 1
    assert torch.isfinite(x).all() and info["true_rel_res"] < 1.0
    info = P.solve_bicgstab(b, x, x0_is_zero=False)  # warm start from that iterate
    assert info["status"] == bo.BO_OK and oracle.rel_residual(Ao, a["b"], x.cpu().numpy()) <= 1e-8
    # host buffers
    xh = np.zeros(n)
    info = P.solve_bicgstab(a["b"].copy(), xh)
    assert info["status"] == bo.BO_OK and oracle.rel_residual(Ao, a["b"], xh) <= 1e-8


def test_bicgstab_waterflood_64x64x32(bo, ctx):
    dims = (64, 64, 32)
    a, Ao, A, P = _setup(bo, ctx, bogen.waterflood_case(*dims, seed=42, day=0), dims, 1)
    b = torch.tensor(a["b"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = P.solve_bicgstab(b, x, tol=1e-8, maxit=300)
    assert info["status"] == bo.BO_OK, info
    assert oracle.rel_residual(Ao, a["b"], x.cpu().numpy()) <= 1e-8
