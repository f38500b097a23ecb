"""Benchmark: time to a 1e-8 relative residual for 1M-cell three-phase
black-oil Jacobians (128 x 128 x 64 grid, 3.1M unknowns), plus the BSR
SpMV's HBM bandwidth.

A step is one pass of the whole hot path on one Newton Jacobian resident
in HBM: value ingest into the solver's layout, Quasi-IMPES decoupling,
block-ILU(0) factorisation and AMG setup, CPR-FGMRES(30) to
||b - A x|| <= 1e-8 ||b||, and the Newton update.  The steps cycle through
ten seeded Jacobians (successive days of a synthetic five-spot waterflood),
524 MB of matrix values each, so every step's inputs are larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle, timed alone
  python bench.py --workload ensemble|learned|conv ...

The default preconditioner precision is the mixed form: FP32 decoupling,
ILU and AMG inside the FP64 flexible GMRES (Arnoldi, true residual and the
Newton update in FP64); the FP64 preconditioner is timed beside it
("secondary").

One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-8 rel. residual, 1M-cell 3-phase Jacobian; BSR SpMV HBM GB/s"
DIMS = (128, 128, 64)
SEED = 42
SAMPLE_DIMS = (64, 64, 32)  # the reference arm's warm-up sample
MIXED_DIMS = (256, 256, 128)  # the 8.4M-cell mixed-precision Jacobian
REF_TOL = 1e-13  # the oracle's reference solutions for the error report


def _nnzb(nx, ny, nz):
    return nx * ny * nz + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))


def _make_jacobian(args):
    dims, seed, day = args
    import bogen
    case = bogen.waterflood_case(*dims, seed=seed, day=day)
    a = bogen.assemble(case)
    return a["rowptr"], a["col"], a["val"].reshape(-1), a["b"], case.x


def generate(dims, seed, days, procs):
    """Seeded Jacobians for days 0..days-1 (spawned workers; before any CUDA call)."""
    import bogen
    bogen.build()
    jobs = [(dims, seed, d) for d in range(days)]
    if procs > 1 and days > 1:
        with mp.get_context("spawn").Pool(min(procs, days)) as pool:
            return pool.map(_make_jacobian, jobs)
    return [_make_jacobian(j) for j in jobs]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the GPU works."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        load = [c for c in sm if c > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def parse_cpulist(spec):
    """CPU numbers of a sysfs cpulist such as "0-3,8,10-11"."""
    cpus = set()
    for part in spec.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_near_gpu(index):
    """Run on the CPUs next to the GPU (its PCI device's local_cpulist), so
    that pinned host buffers allocated afterwards are first touched on the
    GPU's own memory node; returns the CPU list, or None where unknown."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dom, bus, rest = out.lower().split(":")
        path = f"/sys/bus/pci/devices/{dom[-4:]}:{bus}:{rest}/local_cpulist"
        with open(path) as f:
            cpus = parse_cpulist(f.read())
        cpus &= os.sched_getaffinity(0)
        if cpus and len(cpus) < len(os.sched_getaffinity(0)):
            os.sched_setaffinity(0, cpus)
            return sorted(cpus)
    except Exception:
        pass
    return None


def make_reduce_max(dist, device):
    """max over ranks of a host float (identity without a process group)."""
    def reduce_max(v):
        if dist is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return reduce_max


def rank_seed(rank):
    """Each rank of a multi-GPU run solves its own seeded Jacobians (replicas)."""
    return SEED + 1000 * rank


def aggregate(elapsed_ms, units, world, reduce_max):
    """Whole-job numbers: the max elapsed time over ranks; every rank solved
    `units` Jacobians, so the job solved units * world in that time."""
    t = reduce_max(elapsed_ms)
    return {"elapsed_ms": t, "ms_per_solve": t / (units * world), "solves_per_s": units * world / (t / 1e3)}


def host_cores():
    """(CPUs of the machine, CPUs this process may run on)."""
    try:
        aff = len(os.sched_getaffinity(0))
    except Exception:
        aff = os.cpu_count() or 1
    return os.cpu_count() or aff, aff


def oracle_solve(a, dims, tol=1e-8, x0=None, prec=None, maxit=600):
    """The FP64 oracle (one thread): CPR (red-black block ILU(0) + AMG) set up
    on the Jacobian a (unless given) and GMRES(30) to tol; returns
    (x, info, seconds, prec)."""
    import oracle
    A = oracle.BsrMatrix(a["rowptr"], a["col"], np.asarray(a["val"]).reshape(-1, 3, 3))
    t0 = time.perf_counter()
    P = prec or oracle.cpr_prec(A, dims, amg=oracle.AmgParams(coarse_max=128))
    x, info = oracle.gmres(A, a["b"], x0=x0, tol=tol, maxit=maxit, prec=P)
    return x, info, time.perf_counter() - t0, P


def oracle_sample(seed=SEED):
    """The oracle on the 64x64x32 waterflood Jacobian (the reference arm's
    warm-up): seconds of setup + solve to 1e-8."""
    import bogen
    a = bogen.assemble(bogen.waterflood_case(*SAMPLE_DIMS, seed=seed, day=0))
    _, info, sec, _ = oracle_solve(a, SAMPLE_DIMS)
    return sec, info


def oracle_full(dims=DIMS, seed=SEED):
    """The oracle on the benchmark's first Jacobian itself (128x128x64, day
    0): seconds of setup + solve to 1e-8."""
    import bogen
    a = bogen.assemble(bogen.waterflood_case(*dims, seed=seed, day=0))
    _, info, sec, _ = oracle_solve(a, dims)
    return sec, info


def oracle_reference_job(args):
    """Spawned worker of the CPU leg: the oracle's reference solution of a
    seeded Jacobian (GMRES(30) + CPR to REF_TOL from zero), for the error
    report of the GPU solves; returns (x_ref, info, seconds)."""
    dims, seed, day, tol = args
    import bogen
    import oracle
    oracle.build()
    a = bogen.assemble(bogen.waterflood_case(*dims, seed=seed, day=day))
    x, info, sec, _ = oracle_solve(a, dims, tol=tol)
    return x, info, sec


def cpu_baseline_record(seconds, info, dims=DIMS, what="the benchmark's first Jacobian (day 0)"):
    total, aff = host_cores()
    return {"value": seconds * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
            "host_cores": total, "affinity_cores": aff,
            "sample": (f"oracle CPR-GMRES(30) (red-black block ILU(0) + AMG, FP64, one thread) on {what}, "
                       f"{dims[0]}x{dims[1]}x{dims[2]} waterflood, setup + solve to 1e-8 from zero "
                       f"({info['iters']} its, {seconds:.2f} s)")}


def cpu_spmv_record(a, threads, reps=10):
    """The CPU's BSR SpMV bandwidth: the oracle's threaded y = A x over the
    process's CPUs, algorithmic bytes as for the GPU SpMV."""
    import oracle
    A = oracle.BsrMatrix(a["rowptr"], a["col"], np.asarray(a["val"]).reshape(-1, 3, 3))
    x = np.random.default_rng(1).standard_normal(A.n)
    y = np.zeros(A.n)
    for _ in range(2):
        oracle.spmv_threads(A, x, threads, y)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.spmv_threads(A, x, threads, y)
    sec = (time.perf_counter() - t0) / reps
    byts = 9 * 8 * A.col.size + 2 * A.n * 8
    return {"us": sec * 1e6, "algorithmic_bytes": byts, "gbs": byts / sec / 1e9, "threads": threads,
            "kind": "oracle BSR SpMV over host threads (FP64)"}


def solution_errors(x, xr):
    """||x - x_ref|| / ||x_ref||, overall and per component (p, Sw, Sg)."""
    x = np.asarray(x, dtype=np.float64)
    xr = np.asarray(xr, dtype=np.float64)
    out = {"all": float(np.linalg.norm(x - xr) / np.linalg.norm(xr))}
    for k, nm in enumerate(("p", "sw", "sg")):
        out[nm] = float(np.linalg.norm(x[k::3] - xr[k::3]) / np.linalg.norm(xr[k::3]))
    return out


def run_reference(args):
    """The FP64 oracle as the reference arm: every timed step is the
    oracle's setup and CPR-GMRES(30) solve of the benchmark's first
    128x128x64 Jacobian to 1e-8 (one thread); the warm-up steps run the
    64x64x32 sample, which exercises the same code."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_sample()
    import bogen
    a = bogen.assemble(bogen.waterflood_case(*DIMS, seed=SEED, day=0))
    times, info = [], None
    for _ in range(args.steps):
        _, info, sec, _ = oracle_solve(a, DIMS)
        times.append(sec)
    rec = cpu_baseline_record(statistics.mean(times), info)
    rec["sample"] += f"; mean of {args.steps} steps"
    line = {"impl": "reference", "metric": METRIC, "value": rec["value"], "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args), "cpu_baseline": rec,
            "e2e": {"value": rec["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args):
    dims = tuple(getattr(args, "dims", DIMS))
    nx, ny, nz = dims
    seq = getattr(args, "sequence", "newton")
    days = ("successive days advanced by the device Newton method" if seq == "newton"
            else "successive days of synthetic front growth")
    return {"workload": (f"waterflood black-oil Jacobians {nx}x{ny}x{nz} (3 unknowns/cell, 3x3 BSR 7-point), "
                         f"{args.jacobians} {days}, CPR-FGMRES({args.restart}) to 1e-8, "
                         f"preconditioner {args.precision}"),
            "sequence": seq,
            "grid": list(dims), "unknowns": 3 * nx * ny * nz, "nnzb": _nnzb(*dims), "tol": 1e-8,
            "restart": args.restart, "precision": args.precision, "seed": SEED, "jacobians": args.jacobians,
            "l2": "inputs larger than L2 (524 MB of matrix values per step, 10 Jacobians resident)"}


def _make_ensemble_member(spec):
    import bogen
    a = bogen.assemble(bogen.ensemble_case(spec))
    return a["rowptr"], a["col"], a["val"].reshape(-1), a["b"]


def _make_dual_member(spec):
    from bogen import dual as D
    a = D.assemble_dual(D.dual_case(spec["seed"], *spec["dims"], sigma_k=spec["sigma"]))
    return a["rowptr"], a["col"], a["val"].reshape(-1), a["b"]


def ensemble_inputs(n, procs, dual=False):
    """The ensemble's seeded realisations (spawned workers; before any CUDA
    call): specs and per realisation (rowptr, col, val, b)."""
    import bogen
    bogen.build()
    specs = bogen.ensemble_specs(n=n)
    with mp.get_context("spawn").Pool(max(1, min(16, procs))) as pool:
        data = pool.map(_make_dual_member if dual else _make_ensemble_member, specs)
    return specs, data


def ensemble_record(bo, ctx, dev, specs, data, steps, warmup, restart=30, launch="auto", dual=False):
    """A step re-ingests every realisation's values, refreshes its FP32
    preconditioner and solves all realisations together (bo_solve_batched,
    or bo_dp_solve_batched for the dual-porosity variant); a realisation
    whose FP32-preconditioned solve stalls is solved again with an FP64
    preconditioner (promotion).  Returns the record (solves/s, p50/p99 of
    the per-realisation times, iterations)."""
    import torch
    mats, precs, vals, bs, xs, dps = [], [], [], [], [], []
    for sp, (rp, cl, v, b) in zip(specs, data):
        if dual:
            dp = bo.DualPorosity(ctx, *sp["dims"], rp, cl, v)
            dps.append(dp)
            A = dp.fracture_matrix
        else:
            A = bo.Matrix.from_bsr(ctx, bo.grid(*sp["dims"]), rp, cl, v)
        mats.append(A)
        precs.append(bo.Preconditioner(A, precision=bo.BO_PREC_FP32))
        vals.append(torch.from_numpy(v).to(dev))
        bs.append(torch.from_numpy(b).to(dev))
        xs.append(torch.zeros(b.size, dtype=torch.float64, device=dev))
    tuned = None
    if not dual and launch == "auto":
        cache = os.path.join(ROOT, "paper_1606_00556_gb300", "_build", "tune_cache.json")
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tuned = bo.bo_autotune_batched(precs, bs, xs, cache_path=cache, restart=restart, maxit=1000)
    fallback = {}

    def step():
        if dual:
            for dp, P, v in zip(dps, precs, vals):
                dp.update_values(v)
                P.update()
            rc, infos = bo.bo_dp_solve_batched(dps, precs, bs, xs, tol=1e-8, restart=restart, maxit=1000)
        else:
            bo.bo_update_batched(precs, vals)
            rc, infos = bo.bo_solve_batched(precs, bs, xs, tol=1e-8, restart=restart, maxit=1000)
        for r, i in enumerate(infos):
            if i["status"] != 0:
                if r not in fallback:
                    fallback[r] = bo.Preconditioner(mats[r], precision=bo.BO_PREC_FP64)
                else:
                    fallback[r].update()
                if dual:
                    i2 = dps[r].solve(fallback[r], bs[r], xs[r], tol=1e-8, restart=restart, maxit=1000,
                                      raise_on_error=False)
                else:
                    i2 = fallback[r].solve(bs[r], xs[r], tol=1e-8, restart=restart, maxit=1000, raise_on_error=False)
                i2["promoted"] = True
                infos[r] = i2
        return infos

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    all_infos = [step() for _ in range(steps)]
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    per = sorted(i["solve_ms"] for infos in all_infos for i in infos)
    its = [i["iters"] for i in all_infos[-1]]
    unknowns = sum((6 if dual else 3) * int(np.prod(sp["dims"])) for sp in specs)
    rec = {"value": len(specs) * steps / el, "unit": "solves/s", "steps": steps, "warmup": warmup,
           "ms_per_step": el * 1e3 / steps, "realisations": len(specs), "unknowns": unknowns,
           "variant": ("dual porosity (fracture + matrix node per cell, shape factor 0.1 ft^-2), matrix unknowns "
                       "condensed, fracture systems solved together" if dual else "single porosity"),
           "per_realisation_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
           "iters": {"min": min(its), "mean": float(np.mean(its)), "max": max(its)},
           "true_rel_res_max": max(i["true_rel_res"] for infos in all_infos for i in infos),
           "failed": sum(i["status"] != 0 for infos in all_infos for i in infos),
           "promoted_to_fp64": sorted(fallback.keys()), "tuned": tuned,
           "grids": "nx,ny in 32..96 (nx even), nz in 8..24, sigma 0.5..2.0, seed 7"}
    for P in list(precs) + list(fallback.values()):
        P.close()
    return rec


def run_ensemble(args):
    """The batched-ensemble workload: 256 seeded realisations of uneven grid
    size (32..96 x 32..96 x 8..24 cells, 38.3M unknowns in all) solved
    together by bo_solve_batched.  A step re-ingests every realisation's
    values, rebuilds its preconditioner and solves all of them."""
    import bogen
    bogen.build()
    specs = bogen.ensemble_specs(n=args.ensemble)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        data = pool.map(_make_ensemble_member, specs)
    import torch
    import paper_1606_00556_gb300 as bo
    dev = torch.device("cuda", 0)
    ctx = bo.Context(0)
    prec = {"fp32": bo.BO_PREC_FP32, "bf16": bo.BO_PREC_BF16}.get(args.precision, bo.BO_PREC_FP64)
    mats, precs, vals, bs, xs = [], [], [], [], []
    for sp, (rp, cl, v, b) in zip(specs, data):
        A = bo.Matrix.from_bsr(ctx, bo.grid(*sp["dims"]), rp, cl, v)
        mats.append(A)
        precs.append(bo.Preconditioner(A, precision=prec))
        vals.append(torch.from_numpy(v).to(dev))
        bs.append(torch.from_numpy(b).to(dev))
        xs.append(torch.zeros(b.size, dtype=torch.float64, device=dev))

    fallback = {}
    tuned = None
    if args.launch == "graph":
        for P in precs:
            P.set_launch_mode(bo.BO_LAUNCH_GRAPH)
    elif args.launch == "auto":
        cache = os.path.join(ROOT, "paper_1606_00556_gb300", "_build", "tune_cache.json")
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tuned = bo.bo_autotune_batched(precs, bs, xs, cache_path=cache, restart=args.restart, maxit=1000)

    def step():
        bo.bo_update_batched(precs, vals)
        rc, infos = bo.bo_solve_batched(precs, bs, xs, tol=1e-8, restart=args.restart, maxit=1000)
        # mixed precision with promotion: a realisation whose FP32-preconditioned
        # solve stagnates is solved again with an FP64 preconditioner
        for r, i in enumerate(infos):
            if i["status"] != 0 and prec == bo.BO_PREC_FP32:
                if r not in fallback:
                    fallback[r] = bo.Preconditioner(mats[r], precision=bo.BO_PREC_FP64)
                else:
                    fallback[r].update()
                i2 = fallback[r].solve(bs[r], xs[r], tol=1e-8, restart=args.restart, maxit=1000, raise_on_error=False)
                i2["promoted"] = True
                infos[r] = i2
        return infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = bo.bo_kernel_launches()
    t0 = time.perf_counter()
    all_infos = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    launches = bo.bo_kernel_launches() - l0
    clk = clocks.stop()
    per = sorted(i["solve_ms"] for infos in all_infos for i in infos)
    its = [i["iters"] for i in all_infos[-1]]
    unknowns = sum(3 * int(np.prod(sp["dims"])) for sp in specs)
    line = {"metric": "ensemble solves/s (batched CPR-FGMRES to 1e-8)", "workload": "ensemble",
            "value": len(specs) * args.steps / el, "unit": "solves/s", "higher_is_better": True,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+f32+bf16"}[args.precision], "data": "synthetic",
            "config": {"realisations": len(specs), "unknowns": unknowns, "precision": args.precision,
                       "grids": "nx,ny in 32..96 (nx even), nz in 8..24, sigma 0.5..2.0, seed 7"},
            "per_realisation_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
            "iters": {"min": min(its), "mean": float(np.mean(its)), "max": max(its)},
            "true_rel_res_max": max(i["true_rel_res"] for infos in all_infos for i in infos),
            "failed": sum(i["status"] != 0 for infos in all_infos for i in infos),
            "promoted_to_fp64": sorted(fallback.keys()), "launch": args.launch, "tuned": tuned,
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def _conv_flops(V):
    """Forward and training (forward + weight and data gradients, no data
    gradient for the input layer) FLOPs of the network on V voxels."""
    layers = [(16, 32)] + [(32, 32)] * 12 + [(32, 16)]
    f = [2 * 27 * V * ci * co for ci, co in layers]
    return sum(f), 3 * sum(f) - f[0]


def run_learned(args):
    """The learned Newton update on 64x64x32 realisations (one injector, one
    producer): targets from this solver's FP64 CPR-FGMRES solves to 1e-8,
    training with the BF16 tensor-core kernels, then held-out solves from
    the zero guess and from the network's prediction (pressure only, all
    three components, and all three plus the learned coarse space)."""
    import bogen
    from bogen import learned as L
    bogen.build()
    import torch
    import paper_1606_00556_gb300 as bo
    from paper_1606_00556_gb300 import learned
    dims = (64, 64, 32)
    V = int(np.prod(dims))
    dev = torch.device("cuda", 0)
    ctx = bo.Context(0)
    procs = min(16, os.cpu_count() or 1)
    stream = torch.cuda.current_stream(dev)
    X = torch.empty(args.train, V, 16, dtype=torch.bfloat16, device=dev)
    Y = torch.empty(args.train, V, 4, dtype=torch.float32, device=dev)
    A = P = None
    t0 = time.perf_counter()
    gen_iters = []
    for i, (f, a) in enumerate(L.samples(range(1000, 1000 + args.train), dims, processes=procs)):
        if A is None:
            A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], a["val"])
            P = bo.Preconditioner(A)
        else:
            A.update_values(a["val"])
            P.update()
        b = torch.from_numpy(a["b"]).to(dev)
        x = torch.zeros_like(b)
        info = P.solve(b, x, tol=1e-8, restart=args.restart, maxit=1000, raise_on_error=False)
        gen_iters.append(info["iters"])
        X[i] = torch.from_numpy(f).to(dev).to(torch.bfloat16)
        Y[i] = torch.from_numpy(L.targets(x.cpu().numpy())).to(dev)
    gen_s = time.perf_counter() - t0
    net = bo.CNN(ctx, *dims, max_batch=args.batch, seed=0)
    steps = args.epochs * args.train // args.batch
    learned.train(net, X, Y, 3, args.batch, lr=args.lr, nout=3)  # warm-up (3 steps), then a fresh network
    net.close()
    net = bo.CNN(ctx, *dims, max_batch=args.batch, seed=0)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    l0 = bo.bo_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = learned.train(net, X, Y, steps, args.batch, lr=args.lr, nout=3, log_every=max(1, steps // 10))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    train_launches = bo.bo_kernel_launches() - l0
    train_ms = e0.elapsed_time(e1)
    fwd_flops, train_flops = _conv_flops(V)
    # forward-only throughput of the inference pass (batch 1) and of one conv layer
    pred = torch.empty(args.batch, V, 4, device=dev)
    for _ in range(3):
        net.forward(X[:args.batch], pred)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(10):
        net.forward(X[:args.batch], pred)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1) / 10
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16_peak, peak_kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        bf16_peak, peak_kind = 1900.0, "fallback"
    del X, Y
    # held-out evaluation
    modes = {"zero": None, "learned_p": (1, None), "learned_pss": (3, None), "learned_pss_coarse": (3, (16, 16, 8))}
    res = {m: {"iters": [], "ms": [], "kept": []} for m in modes}
    xf = torch.empty(1, V, 16, dtype=torch.bfloat16, device=dev)
    pred1 = torch.empty(1, V, 4, device=dev)
    for f, a in L.samples(range(5000, 5000 + args.test), dims, processes=procs):
        A.update_values(a["val"])
        P.update()
        b = torch.from_numpy(a["b"]).to(dev)
        xf[0] = torch.from_numpy(f).to(dev).to(torch.bfloat16)
        for m, opt in modes.items():
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            ta = time.perf_counter()
            if opt is None:
                info = P.solve(b, x, tol=1e-8, restart=args.restart, maxit=1000, raise_on_error=False)
                info["guess_used"] = False
            else:
                info = learned.learned_solve(P, net, xf, b, x, L.TARGET_SCALE, opt[0], coarse_tile=opt[1],
                                             restart=args.restart, pred=pred1)
            torch.cuda.synchronize()
            res[m]["ms"].append((time.perf_counter() - ta) * 1e3)
            if info["status"] != 0 or info["true_rel_res"] > 1e-8:
                raise RuntimeError(f"held-out solve failed in mode {m}: {info}")
            res[m]["iters"].append(info["iters"])
            res[m]["kept"].append(bool(info["guess_used"]))
    summ = {m: {"iters_mean": float(np.mean(r["iters"])), "ms_mean": float(np.mean(r["ms"])),
                "guess_kept": float(np.mean(r["kept"]))} for m, r in res.items()}
    ach = train_flops * args.batch * steps / (train_ms * 1e-3) / 1e12
    line = {"metric": "learned Newton update: training throughput and held-out iterations to 1e-8 (64x64x32)",
            "workload": "learned", "value": summ["learned_pss"]["iters_mean"], "unit": "iterations",
            "higher_is_better": False, "n_gpus": 1, "steps": steps, "warmup": 3,
            "ms_per_step": train_ms / steps, "dtype": "bf16", "data": "synthetic",
            "config": {"grid": list(dims), "train": args.train, "test": args.test, "epochs": args.epochs,
                       "batch": args.batch, "lr": args.lr,
                       "network": "conv 16->32, 6 residual blocks of 2 conv 32->32, conv 32->16; 3x3x3, ReLU",
                       "seeds": "train 1000.., test 5000..", "l2": "activations > L2 (4 x 131072 x 32 x 2 B per layer)"},
            "training": {"ms": train_ms, "samples_per_s": args.batch * steps / (train_ms * 1e-3),
                         "tflops": ach, "loss_first": losses[0][1], "loss_last": losses[-1][1],
                         "losses": losses, "gpu_launches": train_launches},
            "roofline": {"bound": "tensor", "kernel": "network training step (fwd + dgrad + wgrad)",
                         "achieved": ach, "peak": bf16_peak, "peak_kind": peak_kind, "unit": "TFLOP/s",
                         "frac": ach / bf16_peak, "traffic": None,
                         "forward_tflops": fwd_flops * args.batch / (fwd_ms * 1e-3) / 1e12,
                         "forward_ms_batch": fwd_ms},
            "heldout": summ, "generation": {"seconds": gen_s, "iters_mean": float(np.mean(gen_iters))},
            "clocks": clk, "gpu_launches": train_launches}
    print(json.dumps(line), flush=True)


def run_conv(args):
    """One 32 -> 32 3x3x3 convolution layer of the learned update at
    64x64x32 voxels, batch 16 (input 134 MB > L2): forward (ReLU) on each
    engine, data gradient and weight gradient, CUDA-event timed."""
    import torch
    import paper_1606_00556_gb300 as bo
    nx, ny, nz = args.dims if tuple(args.dims) != DIMS else (64, 64, 32)
    B = args.batch if args.batch != 4 else 16
    V = nx * ny * nz
    dev = torch.device("cuda", 0)
    ctx = bo.Context(0)
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev).manual_seed(SEED)
    x = (torch.randn(B, V, 32, device=dev, generator=g) * 0.5).to(torch.bfloat16)
    w = (torch.randn(27, 32, 32, device=dev, generator=g) * 0.05).to(torch.bfloat16)
    bias = torch.zeros(32, device=dev)
    y = torch.empty(B, V, 32, device=dev, dtype=torch.bfloat16)
    dx = torch.empty(B, V, 32, device=dev)
    dy = torch.randn(B, V, 32, device=dev, generator=g)
    dw = torch.empty(27, 32, 32, device=dev)
    db = torch.empty(32, device=dev)
    flops = 2 * 27 * 32 * 32 * V * B

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    res = {}
    for eng in (0, 1):
        bo.bo_set_conv_engine(eng)
        ms = timed(lambda: bo.bo_conv3d_forward(ctx, (nx, ny, nz), x, w, bias, relu=True, y=y))
        res[f"forward_engine{eng}"] = {"ms": ms, "tflops": flops / ms / 1e9}
        ms = timed(lambda: bo.bo_conv3d_backward_data(ctx, (nx, ny, nz), y, w, dx))
        res[f"dgrad_engine{eng}"] = {"ms": ms, "tflops": flops / ms / 1e9, "note": "includes the primitive's scratch alloc"}
    bo.bo_set_conv_engine(0)
    tc_ok = bo.bo_tc_status() == bo.BO_OK
    ms = timed(lambda: bo.bo_conv3d_backward_weights(ctx, (nx, ny, nz), x, dy, dw, db))
    res["wgrad"] = {"ms": ms, "tflops": flops / ms / 1e9, "note": "includes the primitive's scratch alloc"}
    best = max(res["forward_engine0"]["tflops"], res["forward_engine1"]["tflops"])
    line = {"metric": "3x3x3 conv 32->32 forward TFLOP/s (64x64x32, batch 16)", "workload": "conv", "value": best,
            "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "dtype": "bf16", "data": "synthetic", "config": {"grid": [nx, ny, nz], "batch": B, "flops": flops,
                                                            "l2": "input 134 MB > L2"},
            "roofline": {"bound": "tensor", "kernel": "k_conv3d_tc / k_conv3d_fwd", "achieved": best, "peak": peak,
                         "peak_kind": kind, "unit": "TFLOP/s", "frac": best / peak, "traffic": None},
            "kernels": res, "tc_status_ok": tc_ok}
    print(json.dumps(line), flush=True)


def newton_sequence(bo, ctx, dev, case, A, days, restart, eps_rel=1e-6):
    """The first Newton Jacobian of each of `days` successive 1-day steps of
    the waterflood `case`: day 0 at the case's state, each later day at the
    state the device Newton method (Alg. 1, third forcing term, FP32 CPR,
    ||b|| reduced by eps_rel) converged to on the previous day.  Returns
    (values, right-hand sides) as device tensors and a record of the Newton
    steps (iterations, linear iterations and CUDA-event time per day)."""
    import bogen
    import torch
    m = bogen.model_inputs(case)
    g = bo.grid(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz)
    M = bo.Model(ctx, g, bo.fluid(**m["fluid"]), m["kx"], m["ky"], m["kz"], m["phi0"], m["depth"],
                 m["perf_cell"], m["perf_type"], m["perf_bhp"], m["perf_dref"], m["perf_wi"])
    Pn = bo.Preconditioner(A, precision=bo.BO_PREC_FP32)
    stream = torch.cuda.current_stream(dev)
    x = torch.from_numpy(np.ascontiguousarray(case.x)).to(dev)
    vals, bs, steps = [], [], []
    for d in range(days):
        val = torch.empty(9 * M.nnzb, dtype=torch.float64, device=dev)
        b = torch.empty(M.n, dtype=torch.float64, device=dev)
        M.assemble(x, x, case.dt, b, val)  # the first system of the step: x = x^n
        vals.append(val)
        bs.append(b)
        if d + 1 == days:
            break
        xn = x.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = M.newton(Pn, x, xn, case.dt, forcing="ew3", eps_rel=eps_rel, maxit=20, restart=restart)
        e1.record(stream)
        torch.cuda.synchronize()
        if info["status"] != bo.BO_OK:
            raise RuntimeError(f"Newton step of day {d} failed: {info}")
        steps.append({"day": d, "newton_iters": info["iters"], "linear_iters": info["linear_iters"],
                      "ms": e0.elapsed_time(e1), "bnorm_reduction": info["norms"][-1] / info["norms"][0]})
    Pn.close()
    M.close()
    rec = {"kind": "device Newton method, third forcing term (Sec. 3.1), FP32 CPR, ||b|| reduced by "
                   f"{eps_rel:g} per day", "days": steps,
           "newton_iters_total": sum(st["newton_iters"] for st in steps),
           "ms_per_day_mean": float(np.mean([st["ms"] for st in steps])) if steps else None}
    return vals, bs, rec


def wells_record(bo, ctx, dev, dims, a, repeats=5):
    """The benchmark's day-0 Jacobian with every well rate-controlled (paper
    Sec. 2.3): the bordered system of 3N + 5 unknowns solved to 1e-8 with the
    FP32 CPR corrected for the well coupling (Woodbury), against the same
    solve without that correction and against the same reservoir matrix with
    the wells at fixed BHP (no border).  Wall times around synchronised
    solves (median of `repeats`); setup_ms is the correction's setup (one CPR
    application per well) after a preconditioner refresh."""
    import torch
    bd = a["border"]
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], a["val"])
    wl = bo.Wells(A, bd["aww"].size, bd["perf_cell"], bd["perf_well"], bd["apw"].ravel(), bd["awp"].ravel(),
                  bd["aww"])
    P = bo.Preconditioner(A, precision=bo.BO_PREC_FP32)
    b = torch.tensor(a["b_full"], device=dev)
    b3 = torch.tensor(a["b"], device=dev)
    x = torch.zeros_like(b)
    x3 = torch.zeros_like(b3)

    def timed(fn):
        ts, info = [], None
        for _ in range(repeats + 1):
            x.zero_()
            x3.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts[1:])), info

    ms, info = timed(lambda: wl.solve(P, b, x, tol=1e-8, maxit=400))
    P.update()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    wl.solve(P, b, x, tol=1e-8, maxit=400)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3 - ms
    wl.set_coupling(0)
    ms0, info0 = timed(lambda: wl.solve(P, b, x, tol=1e-8, maxit=400, raise_on_error=False))
    msb, infob = timed(lambda: P.solve(b3, x3, tol=1e-8, maxit=400))
    rec = {"workload": (f"{dims[0]}x{dims[1]}x{dims[2]} waterflood day 0, 5 rate-controlled wells (4 water-rate "
                        "injectors, 1 liquid-rate producer, targets 0.8 x their rates at the BHP), bordered system "
                        f"of {3 * int(np.prod(dims))} + 5 unknowns, FP32 CPR, tol 1e-8"),
           "ms": ms, "iters": info["iters"], "true_rel_res": info["true_rel_res"], "setup_ms": setup_ms,
           "no_coupling": {"ms": ms0, "iters": info0["iters"], "true_rel_res": info0["true_rel_res"]},
           "same_matrix_fixed_bhp": {"ms": msb, "iters": infob["iters"]}}
    for o in (P, wl, A):
        o.close()
    return rec


def oil_water_record(bo, ctx, dev, dims, a, a3, repeats=5):
    """The two-phase oil-water model (paper Sec. 2.2) on the benchmark's grid,
    rock and wells (the day-0 waterflood front mapped onto [s_wc, 1 - s_or]):
    time to 1e-8 with the FP32 CPR under Quasi-IMPES and ABF decoupling, by
    FGMRES and by BiCGSTAB; and the three-phase day-0 Jacobian with ABF
    against Quasi-IMPES.  Wall times around synchronised solves (median of
    `repeats`)."""
    import torch
    ow = bo.OilWater(ctx, *dims, a["rowptr"], a["col"], a["val"].ravel())
    b = torch.tensor(a["b"], device=dev)
    x = torch.zeros_like(b)

    def timed(fn, xv):
        ts, info = [], None
        for _ in range(repeats + 1):
            xv.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return {"ms": float(np.median(ts[1:])), "iters": info["iters"], "true_rel_res": info["true_rel_res"]}

    rec = {"workload": (f"two-phase oil-water {dims[0]}x{dims[1]}x{dims[2]} (2 unknowns/cell, 2x2 BSR stored "
                        "padded to 3x3), day-0 waterflood front, FP32 CPR, tol 1e-8")}
    for name, dec in (("qi", bo.BO_DECOUPLE_QI), ("abf", bo.BO_DECOUPLE_ABF)):
        P = bo.Preconditioner(ow.matrix, precision=bo.BO_PREC_FP32, decoupling=dec)
        rec[f"fgmres_{name}"] = timed(lambda: ow.solve(P, b, x, tol=1e-8, maxit=400), x)
        rec[f"bicgstab_{name}"] = timed(lambda: ow.solve(P, b, x, tol=1e-8, maxit=400, bicgstab=True), x)
        P.close()
    ow.close()
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a3["rowptr"], a3["col"], a3["val"])
    b3 = torch.tensor(a3["b"], device=dev)
    x3 = torch.zeros_like(b3)
    for name, dec in (("qi", bo.BO_DECOUPLE_QI), ("abf", bo.BO_DECOUPLE_ABF)):
        P = bo.Preconditioner(A, precision=bo.BO_PREC_FP32, decoupling=dec)
        rec[f"three_phase_fgmres_{name}"] = timed(lambda: P.solve(b3, x3, tol=1e-8, maxit=400), x3)
        P.close()
    A.close()
    return rec


def run_mixed(bo, ctx, dev, stream, a, args):
    """The 256x256x128 Jacobian with the FP32, BF16-storage and FP64
    preconditioners: per precision one untimed step, then args.mixed_steps
    timed steps (value ingest, preconditioner update, CPR-FGMRES to 1e-8
    from zero), CUDA events on the library's stream; returns (record, the
    solutions on the host for the error report)."""
    import torch
    dims = MIXED_DIMS
    n = 3 * int(np.prod(dims))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], a["val"])
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(dev)[0]
    val = torch.from_numpy(np.ascontiguousarray(a["val"]).reshape(-1)).to(dev)
    b = torch.from_numpy(a["b"]).to(dev)
    rec = {"grid": list(dims), "unknowns": n, "nnzb": _nnzb(*dims), "matrix_gb": (free0 - free1) / 1e9,
           "l2": "inputs larger than L2 (4.2 GB of FP64 matrix values)"}
    xs = {}
    for nm, pr in (("fp32", bo.BO_PREC_FP32), ("bf16", bo.BO_PREC_BF16), ("fp64", bo.BO_PREC_FP64)):
        torch.cuda.synchronize()
        f0 = torch.cuda.mem_get_info(dev)[0]
        P = bo.Preconditioner(A, precision=pr)
        x = torch.zeros(n, dtype=torch.float64, device=dev)

        def step():
            A.update_values(val)
            P.update()
            return P.solve(b, x, tol=1e-8, restart=args.restart, maxit=1000, x0_is_zero=True, raise_on_error=False)

        step()
        torch.cuda.synchronize()
        f1 = torch.cuda.mem_get_info(dev)[0]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [step() for _ in range(args.mixed_steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        rec[nm] = {"ms": e0.elapsed_time(e1) / max(1, args.mixed_steps), "iters": [i["iters"] for i in infos],
                   "status": [i["status"] for i in infos],
                   "true_rel_res_max": max(i["true_rel_res"] for i in infos),
                   "preconditioner_and_krylov_gb": (f0 - f1) / 1e9}
        xs[nm] = x.cpu().numpy()
        P.close()
    A.close()
    del val, b
    torch.cuda.empty_cache()
    return rec, xs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"],
                    help="preconditioner precision: fp32 (mixed: FP32 CPR inside FP64 FGMRES), bf16 (BF16 "
                         "storage of the preconditioner, FP32 arithmetic) or fp64")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--jacobians", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sequence", default="newton", choices=["newton", "synthetic"],
                    help="the 1M-cell Jacobians of successive days: advanced by the device Newton method "
                         "(default), or the generator's synthetic fronts")
    ap.add_argument("--no-wells", action="store_true",
                    help="skip the rate-controlled-wells and oil-water records of the default line")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the 256-realisation ensembles (single and dual porosity) of the default line")
    ap.add_argument("--ensemble-steps", type=int, default=3, help="timed steps of each ensemble in the default line")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the 256x256x128 (8.4M-cell) mixed-precision Jacobian")
    ap.add_argument("--mixed-steps", type=int, default=3, help="timed solves per precision at 256x256x128")
    ap.add_argument("--mixed-ref-tol", type=float, default=1e-12,
                    help="tolerance of the oracle's reference solution at 256x256x128")
    ap.add_argument("--secondary", default="fp64", choices=["fp32", "fp64", "bf16", "none"],
                    help="also time the other preconditioner precision on the same Jacobians")
    ap.add_argument("--dist-backend", default="nccl")
    ap.add_argument("--workload", default="jacobian", choices=["jacobian", "ensemble", "learned", "conv"])
    ap.add_argument("--train", type=int, default=2000, help="training realisations of the learned workload")
    ap.add_argument("--test", type=int, default=200, help="held-out realisations of the learned workload")
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--ensemble", type=int, default=256, help="realisations of the ensemble workload")
    ap.add_argument("--launch", default="auto", choices=["stream", "graph", "auto"],
                    help="ensemble: per-kernel launches, per-column CUDA graphs, or the autotuner's choice")
    ap.add_argument("--dims", type=int, nargs=3, default=list(DIMS),
                    help="grid (profiling runs only; the benchmark workload is 128 128 64)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "conv":
        return run_conv(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # inputs first (spawned generator workers must start before CUDA)
    dims = tuple(args.dims)
    cpu_leg = rank == 0 and world == 1 and not args.no_cpu_baseline
    mixed = rank == 0 and not args.no_mixed
    ref_pool = ref_async = None
    if cpu_leg and mixed:
        # the oracle's reference solution of the 8.4M-cell Jacobian takes
        # minutes on one core: a spawned worker of the CPU leg computes it
        # while the GPU runs
        ref_pool = mp.get_context("spawn").Pool(1)
        ref_async = ref_pool.apply_async(oracle_reference_job, ((MIXED_DIMS, SEED, 0, args.mixed_ref_tol),))
    if args.sequence == "synthetic":
        jac = generate(dims, rank_seed(rank), args.jacobians, procs=min(16, os.cpu_count() or 1))
        case0 = None
    else:
        # day 0 from the generator; the later days' Jacobians come from the
        # device Newton method advancing the state (below)
        import bogen
        bogen.build()
        case0 = bogen.waterflood_case(*dims, seed=rank_seed(rank), day=0)
        a = bogen.assemble(case0)
        jac = [(a["rowptr"], a["col"], a["val"].reshape(-1), a["b"], case0.x)]
    ens_in = dual_in = None
    if rank == 0 and not args.no_ensemble:
        ens_in = ensemble_inputs(args.ensemble, os.cpu_count() or 1)
        dual_in = ensemble_inputs(args.ensemble, os.cpu_count() or 1, dual=True)
    wells_a = ow_a = None
    if rank == 0 and not args.no_wells:
        import bogen
        bogen.build()
        wells_a = bogen.assemble(bogen.with_rate_controls(bogen.waterflood_case(*dims, seed=SEED, day=0)))
        ow_a = bogen.assemble_ow(bogen.oil_water_case(*dims, seed=SEED, day=0))
    mix_a = None
    if mixed:
        import bogen
        mix_a = bogen.assemble(bogen.waterflood_case(*MIXED_DIMS, seed=SEED, day=0))
    cpu_rec = cpu_spmv = xref = None
    if cpu_leg:
        # the oracle timed on the benchmark's first Jacobian itself, then
        # continued (untimed) to the reference solution of the error report
        import oracle
        oracle.build()
        a0 = {"rowptr": jac[0][0], "col": jac[0][1], "val": jac[0][2], "b": jac[0][3]}
        x8, info8, sec, Po = oracle_solve(a0, dims)
        cpu_rec = cpu_baseline_record(sec, info8, dims)
        xref, info_ref, sec_ref, _ = oracle_solve(a0, dims, tol=REF_TOL, x0=x8, prec=Po)
        cpu_rec["reference_solution"] = {"tol": REF_TOL, "iters": info8["iters"] + info_ref["iters"],
                                         "rel_res": info_ref["relres"], "converged": info_ref["converged"]}
        cpu_spmv = cpu_spmv_record(a0, host_cores()[1])
        del Po

    import torch
    import paper_1606_00556_gb300 as bo
    torch.cuda.set_device(local)
    numa_cpus = bind_near_gpu(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(args.dist_backend)

    def barrier():
        if dist is not None:
            dist.barrier()

    reduce_max = make_reduce_max(dist, "cuda" if args.dist_backend == "nccl" else "cpu")

    bo.lib()
    dev = torch.device("cuda", local)
    ctx = bo.Context(local)
    nx, ny, nz = dims
    N = nx * ny * nz
    n = 3 * N
    nnzb = _nnzb(*dims)
    rowptr, col = jac[0][0], jac[0][1]
    state = torch.from_numpy(jac[0][4]).to(dev)
    g = bo.grid(*dims)
    A = bo.Matrix.from_bsr(ctx, g, rowptr, col, jac[0][2])
    newton_rec = None
    if case0 is not None:
        vals, bs, newton_rec = newton_sequence(bo, ctx, dev, case0, A, args.jacobians, args.restart)
    else:
        vals = [torch.from_numpy(j[2]).to(dev) for j in jac]
        bs = [torch.from_numpy(j[3]).to(dev) for j in jac]
    prec = {"fp32": bo.BO_PREC_FP32, "bf16": bo.BO_PREC_BF16}.get(args.precision, bo.BO_PREC_FP64)
    P = bo.Preconditioner(A, precision=prec)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(k, profile):
        j = k % len(vals)
        A.update_values(vals[j])
        P.update()
        info = P.solve(bs[j], x, tol=1e-8, restart=args.restart, maxit=1000, x0_is_zero=True, profile=profile)
        if info["status"] != 0:
            raise RuntimeError(f"solve failed: {info}")
        bo.bo_newton_update(ctx, state, x)
        return info

    clocks = ClockSampler(local)
    clocks.start()
    for k in range(args.warmup):
        step(k, True)
    barrier()
    torch.cuda.synchronize()
    l0 = bo.bo_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [step(args.warmup + k, True) for k in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = bo.bo_kernel_launches() - l0
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1)
    agg = aggregate(elapsed, args.steps, world, reduce_max)

    # the dominant kernel, timed live inside the steps above: the Arnoldi
    # SpMV w = A z.  It reads a split (hi, lo) FP32 copy of A (8 bytes per
    # value, like FP64) and forms the product with FP32 instructions, so it
    # is bound by HBM: the roofline is its algorithmic bytes (values, z, w;
    # column indices are implied by the stencil) over the measured HBM copy
    # bandwidth, with the FP64-equivalent flop rate beside it.
    spmv_bytes = 9 * 8 * nnzb + n * 8 + n * 8
    spmv_flops = 2 * 9 * nnzb
    spmv_ms = sum(i["spmv_ms"] for i in infos)
    spmv_n = sum(i["spmv_launches"] for i in infos)
    hbm, peak_kind = peaks()
    avg_s = spmv_ms / spmv_n * 1e-3 if spmv_n else None
    ach = spmv_bytes / avg_s / 1e9 if avg_s else None
    ach_tf = spmv_flops / avg_s / 1e12 if avg_s else None
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            traffic = json.load(f).get("arnoldi_spmv") if tuple(dims) == DIMS else None
    except Exception:
        pass

    # standalone BSR SpMV (bo_mat_spmv, natural-order vectors), FP64 and FP32 values
    xs = torch.randn(n, dtype=torch.float64, device=dev)
    ys = torch.zeros_like(xs)
    sp = {}
    for name, pr, vb in (("fp64", bo.BO_PREC_FP64, 8), ("fp32", bo.BO_PREC_FP32, 4), ("bf16", bo.BO_PREC_BF16, 2)):
        for _ in range(3):
            A.spmv(xs, ys, precision=pr)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        reps = 20
        s0.record(stream)
        for _ in range(reps):
            A.spmv(xs, ys, precision=pr)
        s1.record(stream)
        torch.cuda.synchronize()
        us = s0.elapsed_time(s1) / reps * 1e3
        byts = 9 * vb * nnzb + 2 * n * 8
        sp[name] = {"us": us, "algorithmic_bytes": byts, "gbs": byts / (us * 1e-6) / 1e9,
                    "frac": byts / (us * 1e-6) / 1e9 / hbm}

    # the mixed-precision form on the same Jacobians: FP32 preconditioner
    # inside the FP64 FGMRES (Arnoldi, true residual and update in FP64)
    second = None
    if args.secondary != "none" and args.secondary != args.precision:
        P2 = bo.Preconditioner(A, precision={"fp32": bo.BO_PREC_FP32, "bf16": bo.BO_PREC_BF16}.get(args.secondary,
                                                                                                  bo.BO_PREC_FP64))

        def step2(k):
            j = k % len(vals)
            A.update_values(vals[j])
            P2.update()
            info = P2.solve(bs[j], x, tol=1e-8, restart=args.restart, maxit=1000, x0_is_zero=True)
            if info["status"] != 0:
                raise RuntimeError(f"solve failed: {info}")
            bo.bo_newton_update(ctx, state, x)
            return info

        for k in range(args.warmup):
            step2(k)
        barrier()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        infos2 = [step2(args.warmup + k) for k in range(args.steps)]
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        agg2 = aggregate(f0.elapsed_time(f1), args.steps, world, reduce_max)
        second = {"precision": args.secondary, "value": agg2["ms_per_solve"], "unit": "ms",
                  "iters": [i["iters"] for i in infos2],
                  "true_rel_res_max": max(i["true_rel_res"] for i in infos2)}
        P2.close()

    # end to end through the C ABI with host buffers: matrix values, b and x
    # cross PCIe/C2C inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        hv = [v.cpu().pin_memory() for v in vals[:args.e2e_steps]]
        hb = [b.cpu().pin_memory() for b in bs[:args.e2e_steps]]
        hx = torch.zeros(n, dtype=torch.float64).pin_memory()
        # one untimed step first: the host-buffer path's staging is set up
        # on its first use
        A.update_values(hv[-1])
        P.update()
        P.solve(hb[-1], hx, tol=1e-8, restart=args.restart, maxit=1000, x0_is_zero=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            A.update_values(hv[k % len(hv)])
            P.update()
            info = P.solve(hb[k % len(hb)], hx, tol=1e-8, restart=args.restart, maxit=1000, x0_is_zero=True)
            if info["status"] != 0:
                raise RuntimeError(f"e2e solve failed: {info}")
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) * 1e3
        te = reduce_max(te)
        e2e = {"value": te / (args.e2e_steps * world), "unit": "ms", "h2d_bytes_per_step": 9 * 8 * nnzb + n * 8,
               "d2h_bytes_per_step": n * 8,
               "host_cpus": f"{len(numa_cpus)} CPUs local to the GPU" if numa_cpus else "unbound"}

    # error report: each preconditioner precision on the first Jacobian
    # against the oracle's reference solution (overall and per component)
    errors = {}
    if xref is not None:
        # the generator's day-0 Jacobian itself (the one the oracle solved)
        A.update_values(torch.from_numpy(a0["val"]).to(dev))
        b0 = torch.from_numpy(a0["b"]).to(dev)
        errors["reference"] = {"128x128x64": cpu_rec["reference_solution"]}
        errors["128x128x64"] = {}
        for nm, pr in (("fp64", bo.BO_PREC_FP64), ("fp32", bo.BO_PREC_FP32), ("bf16", bo.BO_PREC_BF16)):
            Pe = bo.Preconditioner(A, precision=pr)
            xe = torch.zeros(n, dtype=torch.float64, device=dev)
            ie = Pe.solve(b0, xe, tol=1e-8, restart=args.restart, maxit=1000, x0_is_zero=True,
                          raise_on_error=False)
            errors["128x128x64"][nm] = {"status": ie["status"], "iters": ie["iters"],
                                        "true_rel_res": ie["true_rel_res"],
                                        **solution_errors(xe.cpu().numpy(), xref)}
            Pe.close()

    # the 256x256x128 Jacobian (8.4M cells, 25.2M unknowns) in every
    # preconditioner precision: time to 1e-8 (ingest, setup and solve, as a
    # step above), iterations, device memory
    mixed_rec = None
    mixed_x = {}
    if mix_a is not None:
        mixed_rec, mixed_x = run_mixed(bo, ctx, dev, stream, mix_a, args)
        del mix_a
    wells_rec = ow_rec = None
    if wells_a is not None:
        wells_rec = wells_record(bo, ctx, dev, dims, wells_a)
        del wells_a
    if ow_a is not None:
        a3 = {"rowptr": jac[0][0], "col": jac[0][1], "val": jac[0][2], "b": jac[0][3]}
        ow_rec = oil_water_record(bo, ctx, dev, dims, ow_a, a3)
        del ow_a
    ens_rec = dual_rec = None
    if ens_in is not None:
        # the batched ensembles (configs of 256 realisations, 38M unknowns)
        ens_rec = ensemble_record(bo, ctx, dev, *ens_in, steps=args.ensemble_steps, warmup=1, restart=args.restart)
        del ens_in
        dual_rec = ensemble_record(bo, ctx, dev, *dual_in, steps=args.ensemble_steps, warmup=1,
                                   restart=args.restart, dual=True)
        del dual_in
    if ref_async is not None:
        xr8, info_r8, sec_r8 = ref_async.get()
        ref_pool.close()
        errors.setdefault("reference", {})["256x256x128"] = {
            "tol": args.mixed_ref_tol, "iters": info_r8["iters"], "rel_res": info_r8["relres"],
            "converged": info_r8["converged"], "oracle_seconds": sec_r8}
        errors["256x256x128"] = {nm: solution_errors(xm, xr8) for nm, xm in mixed_x.items()}

    if rank == 0:
        iters = [i["iters"] for i in infos]
        line = {
            "metric": METRIC, "value": agg["ms_per_solve"], "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": agg["elapsed_ms"] / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f64+f32", "bf16": "f64+f32+bf16"}[args.precision],
            "data": "synthetic", "config": config_dict(args),
            "roofline": {"bound": "hbm", "kernel": "k_arnoldi_spmv (split-FP32 product, tiled matrix copy)",
                         "achieved": ach, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": (ach / hbm) if ach else None, "traffic": traffic,
                         "algorithmic_bytes": spmv_bytes, "algorithmic_flops": spmv_flops,
                         "fp64_equivalent_tflops": ach_tf,
                         "avg_us": avg_s * 1e6 if avg_s else None, "launches": spmv_n},
            "spmv": sp, "spmv_cpu": cpu_spmv, "secondary": second, "cpu_baseline": cpu_rec, "e2e": e2e,
            "errors": errors or None, "mixed_256x256x128": mixed_rec, "newton_sequence": newton_rec,
            "ensemble": ens_rec, "ensemble_dual_porosity": dual_rec, "rate_controlled_wells": wells_rec,
            "oil_water": ow_rec,
            "precision_note": ("no all-FP64 path is timed: even the FP64 preconditioner form computes the Arnoldi "
                               "product in split FP32 pairs (2^-46 relative per term); convergence is decided "
                               "on the FP64 true residual of the original system"),
            "gpu_launches": launches, "clocks": clk,
            "iters": iters, "iters_mean": float(np.mean(iters)),
            "true_rel_res_max": max(i["true_rel_res"] for i in infos),
            "solves_per_s": agg["solves_per_s"],
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
