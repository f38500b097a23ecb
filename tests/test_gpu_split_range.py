"""The split (hi, lo) FP32 copy of the matrix that the Arnoldi product and
the FP32/BF16 black ILU pivots read holds values with |a| in [2^-120,
2^126] (48 significant bits from 2^-74 up).  A matrix with a value outside
that range sets a device flag, and those kernels then form their products
from the FP64 matrix instead.  These tests drive that fallback and check
the solves against the FP64 oracle, with the same bars as every other
solve: true relative residual <= 1e-8 and ||x - x_ref|| <= 1e-6 ||x_ref||."""
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


def _xref(Ao, b):
    x, info = oracle.gmres(Ao, b, tol=1e-13, maxit=5000, prec=oracle.ilu0_prec(Ao))
    assert info["converged"]
    return x


def _solve(bo, dims, a, val, b, precision):
    ctx = bo.Context(0)
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], val)
    P = bo.Preconditioner(A, precision=precision)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(bd)
    info = P.solve(bd, x, tol=1e-8)
    return info, x.cpu().numpy()


def test_tiny_scaled_matrix_takes_the_fp64_product(bo):
    # every value times 2^-113: the smallest (0.005 2^-113) lie below 2^-120,
    # the FP64 preconditioner stores them exactly, and the Arnoldi product
    # must come from FP64 A; the preconditioned vectors (about 1/|A|, below
    # 1e31) stay inside FP32's range; A and b scaled alike leave x unchanged
    dims = (20, 20, 5)
    a = bogen.assemble(bogen.tiny_case(3))
    s = 2.0 ** -113
    assert np.abs(a["val"][a["val"] != 0]).min() * s < 2.0 ** -120
    val, b = a["val"] * s, a["b"] * s
    info, x = _solve(bo, dims, a, val, b, bo.BO_PREC_FP64)
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], val)
    assert info["status"] == bo.BO_OK
    assert oracle.rel_residual(Ao, b, x) <= 1e-8
    xr = _xref(oracle.BsrMatrix(a["rowptr"], a["col"], a["val"]), a["b"])
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6


@pytest.mark.parametrize("precision", [1, 2])
def test_one_out_of_range_value_takes_the_fp64_products(bo, precision):
    # one off-diagonal value set to 1e-40 (below 2^-120): the flag sends the
    # Arnoldi product and the split black-pivot kernel to FP64 A; the
    # solution is the oracle's for the same matrix
    dims = (20, 20, 5)
    a = bogen.assemble(bogen.tiny_case(4))
    val = a["val"].copy()
    rp, col = a["rowptr"], a["col"]
    e = next(k for k in range(rp[7], rp[8]) if col[k] != 7)
    val[e][1, 2] = 1e-40
    info, x = _solve(bo, dims, a, val, a["b"], precision)
    Ao = oracle.BsrMatrix(rp, col, val)
    assert info["status"] == bo.BO_OK
    assert oracle.rel_residual(Ao, a["b"], x) <= 1e-8
    xr = _xref(Ao, a["b"])
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6
