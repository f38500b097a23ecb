"""The allocation-free residual entry point (bo_mat_residual_noalloc) against
the library's existing entry points and the FP64 oracle, through the C ABI,
on two calls in a row.  It is for callers that must not call cudaMalloc when
they check a residual (an allocator that already owns the device memory, or
a loop that cannot afford the device-wide synchronisation cudaMalloc
implies).

Cases: the 2,000-cell grid (8 blocks, the final sum inside the last block's
first pass) and a 64 x 64 x 32 grid (131,072 cells, 512 blocks: more
partial-sum pairs than the last block has threads, so its strided sum over
the partials runs).  r is compared element by element with the oracle's
b - A x at 1e-13 (|A| |x| + |b|)_i (21 products and one subtraction in FP64
per entry) and with the public SpMV's; both norms with the oracle's.

This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

import bogen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(which):
    if which == "tiny":
        return bogen.tiny_case(5)
    return bogen.waterflood_case(64, 64, 32, seed=9, day=0, corr=(8, 8, 2))


@pytest.mark.parametrize("which", ["tiny", "64x64x32"])
def test_residual_noalloc_matches_oracle_and_existing_entry_points(which):
    import paper_1606_00556_gb300 as bo
    bo.build()
    ctx = bo.Context(0)
    case = _case(which)
    a = bogen.assemble(case)
    g = bo.grid(case.nx, case.ny, case.nz)
    A = bo.Matrix.from_bsr(ctx, g, a["rowptr"], a["col"], a["val"])
    P = bo.Preconditioner(A)
    b = torch.tensor(a["b"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8)
    assert info["status"] == 0
    # r from the public SpMV: b - A x = (-1) A x + 1 b
    r_pub = b.clone()
    A.spmv(x, r_pub, alpha=-1.0, beta=1.0)
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    xs = x.cpu().numpy()
    r_or = a["b"] - oracle.spmv(Ao, xs)
    bound = 1e-13 * (oracle.spmv(oracle.BsrMatrix(Ao.rowptr, Ao.col, np.abs(Ao.val)), np.abs(xs)) + np.abs(a["b"]))
    for _ in range(2):
        r = torch.full_like(b, float("nan"))
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        bo.bo_mat_residual_noalloc(A, b, x, r, norms)
        torch.cuda.synchronize()
        rg = r.cpu().numpy()
        assert np.all(np.abs(rg - r_or) <= bound)
        # (the public SpMV forms its products in split pairs: 2e-13 (|A| |x|)_i)
        assert np.all(np.abs(rg - r_pub.cpu().numpy()) <= 3 * bound)
        nr, nb = norms.cpu().numpy()
        assert nb == pytest.approx(np.linalg.norm(a["b"]), rel=1e-13)
        # | ||r|| - ||r_or|| | <= ||r - r_or|| <= ||bound|| (triangle inequality),
        # plus the rounding of the two norms' own sums
        nref = float(np.linalg.norm(r_or))
        assert abs(nr - nref) <= np.linalg.norm(bound) + 1e-12 * nref
        # the solve reports the same relative residual from its own reduction
        assert nr / nb == pytest.approx(info["true_rel_res"], rel=1e-6)
    # missing or overlapping arguments are rejected, not dereferenced
    L = bo.lib()
    assert L.bo_mat_residual_noalloc(None, None, None, None, None) == bo.BO_ERR_ARG
    nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
    vp = bo._VP
    assert L.bo_mat_residual_noalloc(A.h, vp(b.data_ptr()), vp(x.data_ptr()), vp(x.data_ptr()),
                                     vp(nrm.data_ptr())) == bo.BO_ERR_ARG
    assert L.bo_mat_residual_noalloc(A.h, vp(b.data_ptr()), vp(x.data_ptr()), vp(b.data_ptr() + 8),
                                     vp(nrm.data_ptr())) == bo.BO_ERR_ARG


def test_residual_noalloc_rejects_grids_above_its_scratch():
    # 256 x 128 x 130 = 4,259,840 cells > 4,194,304: BO_ERR_ARG before any
    # launch (the matrix is only created, never multiplied)
    import paper_1606_00556_gb300 as bo
    bo.build()
    ctx = bo.Context(0)
    dims = (256, 128, 130)
    rowptr, col = bogen.pattern(*dims)
    val = np.zeros((col.size, 3, 3))
    val[:, 0, 0] = 1.0
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), rowptr, col, val)
    n = 3 * int(np.prod(dims))
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    r = torch.zeros_like(b)
    nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
    vp = bo._VP
    assert bo.lib().bo_mat_residual_noalloc(A.h, vp(b.data_ptr()), vp(x.data_ptr()), vp(r.data_ptr()),
                                            vp(nrm.data_ptr())) == bo.BO_ERR_ARG
