"""The allocation-free residual entry point (bo_mat_residual_noalloc) against
the library's existing entry points, through the C ABI, on two calls in a
row.  It is for callers that must not call cudaMalloc when they check a
residual (an allocator that already owns the device memory, or a loop that
cannot afford the device-wide synchronisation cudaMalloc implies).

This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

import bogen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_residual_noalloc_matches_existing_entry_points():
    import paper_1606_00556_gb300 as bo
    bo.build()
    ctx = bo.Context(0)
    case = bogen.tiny_case(5)
    a = bogen.assemble(case)
    g = bo.grid(case.nx, case.ny, case.nz)
    A = bo.Matrix.from_bsr(ctx, g, a["rowptr"], a["col"], a["val"])
    P = bo.Preconditioner(A)
    b = torch.tensor(a["b"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8)
    assert info["status"] == 0
    # r from the public SpMV: b - A x = (-1) A x + 1 b
    r_ref = b.clone()
    A.spmv(x, r_ref, alpha=-1.0, beta=1.0)
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    xs = x.cpu().numpy()
    bound = 1e-13 * (oracle.spmv(oracle.BsrMatrix(Ao.rowptr, Ao.col, np.abs(Ao.val)), np.abs(xs)) + np.abs(a["b"]))
    for _ in range(2):
        r = torch.full_like(b, float("nan"))
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        bo.bo_mat_residual_noalloc(A, b, x, r, norms)
        torch.cuda.synchronize()
        assert np.all(np.abs(r.cpu().numpy() - r_ref.cpu().numpy()) <= bound)
        nr, nb = norms.cpu().numpy()
        assert nb == pytest.approx(np.linalg.norm(a["b"]), rel=1e-13)
        # | ||r|| - ||r_ref|| | <= ||r - r_ref|| <= ||bound|| (triangle inequality),
        # plus the rounding of the two norms' own sums
        nref = float(torch.linalg.norm(r_ref))
        assert abs(nr - nref) <= np.linalg.norm(bound) + 1e-12 * nref
        # the solve reports the same relative residual from its own reduction
        assert nr / nb == pytest.approx(info["true_rel_res"], rel=1e-6)
    # missing arguments are rejected, not dereferenced
    assert bo.lib().bo_mat_residual_noalloc(None, None, None, None, None) == bo.BO_ERR_ARG
