"""The benchmark's multi-GPU path on CPU: two gloo ranks (world size 2)
take the job time as the maximum over ranks, count the units of every rank,
and solve different seeded Jacobians (independent replicas, no collective in
the data path).  The reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rm = bench.make_reduce_max(dist, "cpu")
    # rank r "took" 100 (r + 1) ms for 5 solves
    agg = bench.aggregate(100.0 * (rank + 1), 5, world, rm)
    dist.barrier()
    with open(os.path.join(outdir, f"r{rank}.txt"), "w") as f:
        f.write(f"{agg['elapsed_ms']} {agg['ms_per_solve']} {agg['solves_per_s']} {bench.rank_seed(rank)}\n")
    dist.destroy_process_group()


def test_two_rank_aggregation_and_seeds(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(world)]
    for r in rows:
        el, per, sps = map(float, r[:3])
        assert el == 200.0                  # max over ranks
        assert per == pytest.approx(20.0)   # 200 ms for 2 x 5 solves
        assert sps == pytest.approx(50.0)   # whole-job throughput
    assert rows[0][3] != rows[1][3]         # each rank its own Jacobians


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1))

    class A:
        warmup, steps, gpus = 1, 1, 2
    assert bench.run_reference(A()) is None and not called


def test_cpulist_parser():
    # the benchmark binds itself to the CPUs that sysfs lists next to the GPU
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()
    with pytest.raises(ValueError):
        bench.parse_cpulist("a-b")
