"""Batched ensemble solves (bo_solve_batched): realisations of uneven grid
size solved at once must give exactly what solving each alone gives, and
every one must meet the paper's residual criterion (Alg. 1) per the oracle."""
import numpy as np
import pytest

import bogen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPECS = [dict(dims=(8, 6, 3), sigma=0.5, seed=1), dict(dims=(20, 20, 5), sigma=1.0, seed=2),
         dict(dims=(16, 10, 4), sigma=2.0, seed=3), dict(dims=(32, 8, 6), sigma=1.5, seed=4),
         dict(dims=(12, 30, 7), sigma=0.8, seed=5), dict(dims=(40, 36, 10), sigma=1.7, seed=6)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_individual_solves(precision):
    import paper_1606_00556_gb300 as bo
    bo.build()
    ctx = bo.Context(0)
    mats, precs, bs, sys = [], [], [], []
    for sp in SPECS:
        a = bogen.assemble(bogen.ensemble_case(sp))
        A = bo.Matrix.from_bsr(ctx, bo.grid(*sp["dims"]), a["rowptr"], a["col"], a["val"])
        mats.append(A)
        precs.append(bo.Preconditioner(A, precision=precision))
        bs.append(torch.tensor(a["b"], dtype=torch.float64, device="cuda"))
        sys.append((oracle.BsrMatrix(a["rowptr"], a["col"], a["val"]), a["b"]))
    xs = [torch.zeros_like(b) for b in bs]
    rc, infos = bo.bo_solve_batched(precs, bs, xs, tol=1e-8)
    assert rc == bo.BO_OK, infos
    torch.cuda.synchronize()
    for r, (P, b, x, (Ao, bh), info) in enumerate(zip(precs, bs, xs, sys, infos)):
        assert info["status"] == 0 and info["iters"] > 0
        assert oracle.rel_residual(Ao, bh, x.cpu().numpy()) <= 1e-8
        xr = torch.zeros_like(b)
        single = P.solve(b, xr, tol=1e-8)
        torch.cuda.synchronize()
        assert single["iters"] == info["iters"]
        assert torch.equal(xr, x), f"realisation {r} differs from its single solve"


def test_batched_rejects_shared_workspace():
    import paper_1606_00556_gb300 as bo
    ctx = bo.Context(0)
    sp = SPECS[0]
    a = bogen.assemble(bogen.ensemble_case(sp))
    A = bo.Matrix.from_bsr(ctx, bo.grid(*sp["dims"]), a["rowptr"], a["col"], a["val"])
    P = bo.Preconditioner(A)
    b = torch.tensor(a["b"], dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        bo.bo_solve_batched([P], [b], [])
    rc, _ = bo.bo_solve_batched([P, P], [b, b], [torch.zeros_like(b), torch.zeros_like(b)])
    assert rc == bo.BO_ERR_ARG
