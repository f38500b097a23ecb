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


def _ensemble(bo, ctx, precision=0, specs=SPECS):
    precs, bs, sys, mats = [], [], [], []
    for sp in specs:
        a = bogen.assemble(bogen.ensemble_case(sp))
        A = bo.Matrix.from_bsr(ctx, bo.grid(*sp["dims"]), a["rowptr"], a["col"], a["val"])
        mats.append(A)
        precs.append(bo.Preconditioner(A, precision=precision))
        bs.append(torch.tensor(a["b"], dtype=torch.float64, device="cuda"))
        sys.append((oracle.BsrMatrix(a["rowptr"], a["col"], a["val"]), a["b"]))
    return mats, precs, bs, sys


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_launch_is_bitwise_equal_to_stream_launch(precision):
    # the captured columns run the same kernels in the same order
    import paper_1606_00556_gb300 as bo
    ctx = bo.Context(0)
    mats, precs, bs, sys = _ensemble(bo, ctx, precision)
    ref = []
    for P, b in zip(precs, bs):
        x = torch.zeros_like(b)
        info = P.solve(b, x, tol=1e-8)
        ref.append((x, info["iters"], P.residual_history()))
    for P in precs:
        P.set_launch_mode(bo.BO_LAUNCH_GRAPH)
    for rep in range(2):  # the second run replays the graphs captured by the first
        for (P, b), (xr, it, hist) in zip(zip(precs, bs), ref):
            x = torch.zeros_like(b)
            info = P.solve(b, x, tol=1e-8)
            assert info["iters"] == it and torch.equal(x, xr)
            np.testing.assert_array_equal(P.residual_history(), hist)
        xs = [torch.zeros_like(b) for b in bs]
        rc, infos = bo.bo_solve_batched(precs, bs, xs, tol=1e-8)
        assert rc == bo.BO_OK
        for x, (xr, it, _), info in zip(xs, ref, infos):
            assert info["iters"] == it and torch.equal(x, xr)
    # lockstep: one graph per column for the whole batch; a system that has
    # converged idles through the others' columns, its result unchanged
    for P in precs:
        P.set_launch_mode(bo.BO_LAUNCH_BATCH_GRAPH)
    for rep in range(2):  # the second run replays the batch graphs
        xs = [torch.zeros_like(b) for b in bs]
        rc, infos = bo.bo_solve_batched(precs, bs, xs, tol=1e-8)
        assert rc == bo.BO_OK
        for x, (xr, it, hist), info, P in zip(xs, ref, infos, precs):
            assert info["iters"] == it and torch.equal(x, xr)
            np.testing.assert_array_equal(P.residual_history(), hist)


def test_graph_launch_follows_restart_and_coarse_space_changes():
    import paper_1606_00556_gb300 as bo
    ctx = bo.Context(0)
    mats, precs, bs, sys = _ensemble(bo, ctx, 0, SPECS[1:2])
    P, b, (Ao, bh) = precs[0], bs[0], sys[0]
    P.set_launch_mode(bo.BO_LAUNCH_GRAPH)
    for restart in (30, 10, 30):
        x = torch.zeros_like(b)
        info = P.solve(b, x, tol=1e-8, restart=restart)
        assert info["status"] == 0 and oracle.rel_residual(Ao, bh, x.cpu().numpy()) <= 1e-8
    x_ref = x.cpu().numpy()
    P.set_coarse_space(torch.tensor(x_ref[0::3], device="cuda"), (10, 10, 5))
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8)
    assert info["status"] == 0 and oracle.rel_residual(Ao, bh, x.cpu().numpy()) <= 1e-8
    P.set_launch_mode(bo.BO_LAUNCH_STREAM)
    x2 = torch.zeros_like(b)
    P.solve(b, x2, tol=1e-8)
    assert torch.equal(x, x2)


def test_autotuner_picks_and_caches(tmp_path):
    import paper_1606_00556_gb300 as bo
    ctx = bo.Context(0)
    mats, precs, bs, sys = _ensemble(bo, ctx, 0)
    xs = [torch.zeros_like(b) for b in bs]
    path = str(tmp_path / "tune.json")
    r1 = bo.bo_autotune_batched(precs, bs, xs, cache_path=path)
    assert not r1["from_cache"] and r1["launch_mode"] in (0, 1, 2) and r1["streams"] in (4, 8, 16)
    assert len(r1["trial_ms"]) == 9
    assert all(t > 0 for t in r1["trial_ms"])
    assert (r1["amg_cells"], r1["amg_threads"]) in ((1, 256), (2, 256), (4, 256), (1, 128), (2, 128), (1, 512))
    tiles = [t for t in r1["tile_ms"] if t > 0]
    assert len(tiles) == (5 if r1["launch_mode"] != bo.BO_LAUNCH_STREAM else 0)
    assert r1["best_ms"] == min(r1["trial_ms"] + tiles)
    r2 = bo.bo_autotune_batched(precs, bs, xs, cache_path=path)
    assert r2["from_cache"]
    for k in ("launch_mode", "streams", "amg_cells", "amg_threads"):
        assert r2[k] == r1[k]
    import json
    with open(path) as f:
        assert len(json.load(f)) == 1
    # the tuned configuration still solves the batch correctly
    xs = [torch.zeros_like(b) for b in bs]
    rc, infos = bo.bo_solve_batched(precs, bs, xs, tol=1e-8)
    assert rc == bo.BO_OK
    for x, (Ao, bh) in zip(xs, sys):
        assert oracle.rel_residual(Ao, bh, x.cpu().numpy()) <= 1e-8
    bo.bo_set_batch_streams(16)


def test_batched_update_equals_individual_updates():
    import paper_1606_00556_gb300 as bo
    ctx = bo.Context(0)
    specs2 = [dict(sp, seed=sp["seed"] + 100) for sp in SPECS]
    mats, precs, bs, _ = _ensemble(bo, ctx, 0)
    mats2, precs2, bs2, _ = _ensemble(bo, ctx, 0)
    new_vals, sys = [], []
    for sp in specs2:
        a = bogen.assemble(bogen.ensemble_case(sp))
        new_vals.append(torch.tensor(a["val"].reshape(-1), device="cuda"))
        sys.append((oracle.BsrMatrix(a["rowptr"], a["col"], a["val"]), a["b"]))
    bo.bo_update_batched(precs, new_vals)
    for A, P, v in zip(mats2, precs2, new_vals):
        A.update_values(v)
        P.update()
    for P, P2, (Ao, bh) in zip(precs, precs2, sys):
        b = torch.tensor(bh, device="cuda")
        x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
        P.solve(b, x1, tol=1e-8)
        P2.solve(b, x2, tol=1e-8)
        assert torch.equal(x1, x2)
        assert oracle.rel_residual(Ao, bh, x1.cpu().numpy()) <= 1e-8
    # errors are reported: a NaN in one system's values
    bad = [v.clone() for v in new_vals]
    bad[2][7] = float("nan")
    with pytest.raises(bo.BoError) as e:
        bo.bo_update_batched(precs, bad)
    assert e.value.status == bo.BO_ERR_NONFINITE


def test_amg_tile_shapes_give_identical_solves():
    # the per-kernel AMG form (the one captured graphs run) under every tile
    # shape: each cell's arithmetic is the same, only its thread changes
    import paper_1606_00556_gb300 as bo
    ctx = bo.Context(0)
    mats, precs, bs, sys = _ensemble(bo, ctx, 1, SPECS[4:6])
    ref = None
    for cells, threads in ((1, 256), (2, 256), (4, 256), (1, 128), (2, 128), (1, 512), (4, 512)):
        out = []
        for P, b in zip(precs, bs):
            P.set_launch_mode(bo.BO_LAUNCH_GRAPH)
            P.set_amg_tile(cells, threads)
            x = torch.zeros_like(b)
            info = P.solve(b, x, tol=1e-8)
            assert info["status"] == 0
            out.append((x, info["iters"]))
        if ref is None:
            ref = out
        for (x, it), (xr, itr) in zip(out, ref):
            assert it == itr and torch.equal(x, xr)
    with pytest.raises(bo.BoError):
        precs[0].set_amg_tile(3, 256)
    with pytest.raises(bo.BoError):
        precs[0].set_amg_tile(1, 64)
