"""Bounded device-side waits: the AMG's grid barriers give up after a set
number of polls, the launch ends early and the solve reports BO_ERR_TIMEOUT
instead of hanging, and the next solve on the same context is unaffected.

The wait is made to run out by lowering the poll limit to one (a barrier
then gives up while other blocks are still sweeping); nothing faults, traps
or spins without a bound."""
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


@pytest.mark.parametrize("mode", [2, 1])
def test_amg_barrier_timeout_is_reported_and_recoverable(bo, mode):
    # 64 x 64 x 32: level 0 spans 64 cooperative blocks, so barriers wait
    dims = (64, 64, 32)
    a = bogen.assemble(bogen.waterflood_case(*dims, seed=5, day=0, corr=(8, 8, 2)))
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    ctx = bo.Context(0)
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], a["val"])
    b = torch.tensor(a["b"], dtype=torch.float64, device="cuda")
    bo.bo_set_amg_cooperative(mode)
    for precision in (bo.BO_PREC_FP64, bo.BO_PREC_FP32):
        P = bo.Preconditioner(A, precision=precision)
        x = torch.zeros_like(b)
        bo.bo_set_amg_barrier_spins(1)
        try:
            info = P.solve(b, x, tol=1e-8, raise_on_error=False)
        finally:
            bo.bo_set_amg_barrier_spins(0)
        assert info["status"] == bo.BO_ERR_TIMEOUT, info
        assert torch.isfinite(x).all()
        # the context and the preconditioner still work at the default limit
        x.zero_()
        info = P.solve(b, x, tol=1e-8)
        assert info["status"] == bo.BO_OK
        assert oracle.rel_residual(Ao, a["b"], x.cpu().numpy()) <= 1e-8
        P.close()
    bo.bo_set_amg_cooperative(2)
    assert np.isfinite(float(b.norm()))
