"""Benchmark: IGS-GMRES Arnoldi steps/s on one GB300 (FP64).

Workload: 2-D upwind convection-diffusion on a 512 x 512 grid (n = 262144, nnz = 1,308,672,
Peclet 50), b = A 1 + 1e-3 N(0,1), x0 = 0, restart length m = 100, two Gauss-Seidel
iterations (Alg. 4.1).  One benchmark step = one full restart cycle (cycle set-up, 100
Arnoldi columns, Givens least squares, x update and the true backward error), i.e. 100
Arnoldi steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--gs 1|2] [--impl reference]
                  [--workload cd2d|batched|precision|served] [--no-batched] [--no-precision]
                  [--no-served] [--serve-slots S] [--serve-backlog Q] [--serve-graph-min-n N]

Prints one JSON line (rank 0).  `value` is device-timed throughput with b already in HBM
(CUDA events on the library's stream); `e2e` is the same metric through the C interface
with host buffers (H2D of b and D2H of x inside the timed region); `roofline` reports the
dominant kernel (the block multi-dot) against the FP64 FMA pipe (it is FP64-issue-bound on
GB300) with its HBM throughput alongside; `cpu_baseline` times the CPU oracle on one full
cycle of the same workload.  With --gpus N > 1 (torchrun) every rank runs an independent
replica (the method has no data-parallel exchange on one system): weak scaling.

The line also carries `one_reduce`: Alg. 4.2 (one global reduction per column) on the same
workload and cycles; `precision`: the FP32-basis form inside FP64 iterative refinement
against the FP64 form on the 160^3 convection-diffusion system (n = 4.1M, m = 200) to
beta <= 1e-14, with the FP32 multi-dot's HBM roofline; `served`: a Poisson stream of
2-D convection-diffusion requests (2000/s, sides 64..1024) replayed against the request
server (include/igs_serve.h: gangs, plus graph lanes for n >= --serve-graph-min-n) for a
60 s window, with served solves/s, p50/p99 latency and service time, the refused backlog,
and every completed request solved again one at a time through igs_solve (FP64) for
comparison; and `batched`: the batched form (include/igs_batch.h) on 4096 banded
systems (n ~ U{64..2048}, 7 diagonals, m = 50, every system to beta <= 1e-12) in solves/s,
its FP64 roofline, and the same systems solved one at a time by igs_solve (a sample) for
comparison.  `--workload batched` prints that measurement as the main line instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "Arnoldi steps/s"
UNIT = "steps/s"
GRID_N, PECLET, SEED, M = 512, 50.0, 0, 100
# FP64 FMA pipe of GB300: 2 FMA / clock / SM, 152 SMs (4 FLOP per clock per SM with FMA=2)
FP64_FMA_PER_CLK_PER_SM = 2


def workload_config(gs):
    return {"workload": f"cd2d {GRID_N}x{GRID_N} upwind convection-diffusion, Pe {PECLET:g}",
            "n": GRID_N * GRID_N, "nnz": 5 * GRID_N * GRID_N - 4 * GRID_N, "restart_m": M,
            "gs_iters": gs, "step": f"one restart cycle = {M} Arnoldi steps",
            "l2": "inputs larger than L2 (Krylov basis 212 MB > 126 MB L2)"}


def peaks_hbm():
    """The measured HBM copy bandwidth (GB/s) of MEASURED_PEAKS.json, else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def main_config(gs, method, ws, precision="fp64"):
    """The main line's `config` (the same dict in both bench arms)."""
    return {**workload_config(gs), "method": method, "precision": precision, "parallelism": f"replicas x{ws}"}


BATCH_COUNT, BATCH_M, BATCH_TOL, BATCH_MAX_RESTARTS = 4096, 50, 1e-12, 20
BATCH_METRIC, BATCH_UNIT = "solves/s", "solves/s"
# the ncu capture of the batched kernel (1024-system case): DRAM read + write bytes
BATCH_CAPTURE_SYSTEMS, BATCH_CAPTURE_DRAM_BYTES = 1024, 42.4e9 + 0.90e9
FP64_PEAK_TFLOPS = 152 * FP64_FMA_PER_CLK_PER_SM * 2 * 2070.0e6 / 1e12


def batch_config(gs, count=BATCH_COUNT):
    return {"workload": f"batched: {count} independent banded systems, n ~ U{{64..2048}}, "
                        "7 diagonals, N(0,1) off-diagonals, diagonal 1.1 x off-diagonal row sum",
            "count": count, "restart_m": BATCH_M, "gs_iters": gs, "tol_beta": BATCH_TOL,
            "step": "one batch solve: every system to beta <= 1e-12 (one persistent launch)",
            "l2": "inputs larger than L2 (matrices 366 MB, bases 0.6 GB)"}


def batch_fma(ns, nnzs, steps, cycles, m, gs):
    """Algorithmic FP64 multiply-adds of a batch solve (model of Alg. 4.1 per system): per
    cycle r = b - A x and two norms (nnz + 2n), the prime step (nnz + 2n), per loop column p
    the SpMV and (2 + 2(gs-1) + 1) p n for the reductions and updates (5pn with two
    iterations, 3pn with one), the flush norm (n), and x += V y (columns x n)."""
    per_p = 5 if gs == 2 else 3
    total = 0.0
    for n, nnz, st, cy in zip(ns, nnzs, steps, cycles):
        n, nnz, st, cy = float(n), float(nnz), int(st), int(cy)
        cols = [m] * (cy - 1) + [st - m * (cy - 1)] if cy > 0 else []
        for c in cols:
            total += nnz + 2 * n + nnz + 2 * n + c * n
            total += (c - 1) * nnz + per_p * n * (c * (c + 1) / 2 - 1)
            if c == m:
                total += n
            else:  # an in-cycle stop after the SpMV and first reduction of column c + 1
                total += nnz + 2 * (c + 1) * n
        total += nnz + 2 * n  # the final residual check
    return total


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_replicas(ms, e2e_s, steps, dist=None, device=None):
    """Whole-job figures over N independent replicas (one per rank): the slowest rank's
    device time and end-to-end time, and the Arnoldi steps of all ranks.  Without a process
    group, the local figures."""
    if dist is None:
        return ms, e2e_s, steps
    import torch
    t = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(steps)], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t[0].item()), float(t[1].item()), int(round(s.item()))


def oracle_cycle_rate(A, b, m, method="igs", gs=2, impl=None):
    """Arnoldi steps/s of the CPU oracle (as it stands) over one cycle: the serial parity
    build (impl=None) or the OpenMP timing build (oracle.openmp(), all host cores)."""
    import oracle
    meth = oracle.ONE_REDUCE if method == "one_reduce" else oracle.IGS
    t0 = time.perf_counter()
    out = oracle.arnoldi(A, b, m, meth, gs, impl=impl)
    dt = time.perf_counter() - t0
    return out["ncols"] / dt, dt


def cpu_baseline_cd2d(A, b, m, method, gs):
    """The oracle on one full cycle of the benchmark workload, serial and on all host cores
    (the OpenMP build: bitwise the serial build's results)."""
    import oracle
    oracle.build()
    omp = oracle.openmp()
    threads = oracle.openmp_threads()
    rate1, dt1 = oracle_cycle_rate(A, b, m, method, gs)
    rate_n, dt_n = oracle_cycle_rate(A, b, m, method, gs, impl=omp)
    return {"value": rate_n, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one full cycle ({m} Arnoldi columns) of the same workload: {dt_n:.1f} s on "
                      f"{threads} threads (OpenMP build), {dt1:.1f} s serial",
            "nproc": os.cpu_count(),
            "serial": {"value": rate1, "unit": UNIT, "cores": 1, "build": "serial parity build"}}


def run_reference(args):
    """The reference arm: the CPU oracle, timed on this machine's cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "batched":
        import concurrent.futures as cf
        import multiprocessing as mp

        import oracle
        oracle.build()
        out = gen.banded_batch(count=args.batch_count, seed=SEED)
        cores = os.cpu_count() or 1
        stride = max(1, args.batch_count // (4 * cores))
        sample = [(out[i][0], out[i][1], gen.norm2_power(out[i][0], iters=100))
                  for i in range(0, args.batch_count, stride)]
        with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
            for _ in range(args.warmup):
                list(ex.map(_oracle_batch_solve, sample))
            t0 = time.perf_counter()
            for _ in range(args.steps):
                list(ex.map(_oracle_batch_solve, sample))
            dt = time.perf_counter() - t0
        value = args.steps * len(sample) / dt
        line = {"impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT,
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {**batch_config(args.gs, args.batch_count), "parallelism": f"replicas x{ws}"},
                "cpu_baseline": {"value": value, "unit": BATCH_UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{len(sample)} of the {args.batch_count} systems per step, "
                                           f"one serial oracle per process on {cores} processes"},
                "e2e": {"value": value, "unit": BATCH_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    A, b, _, _ = gen.cd2d(GRID_N, PECLET, SEED)
    import oracle
    oracle.build()
    omp = oracle.openmp()
    threads = oracle.openmp_threads()
    meth = oracle.ONE_REDUCE if args.method == "one_reduce" else oracle.IGS
    # bounded sample per step: the first s columns of the m = 100 cycle, s chosen so that the
    # whole run stays within about two minutes (early columns are cheaper, so this favours
    # the oracle)
    t_probe = time.perf_counter()
    oracle.arnoldi(A, b, 10, meth, args.gs, impl=omp)
    t10 = time.perf_counter() - t_probe
    budget = 120.0 / max(1, args.steps + args.warmup)
    s = 10
    while s < M and t10 * ((s + 10) / 10.0) ** 2 <= budget:
        s += 10
    for _ in range(args.warmup):
        oracle.arnoldi(A, b, s, meth, args.gs, impl=omp)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.arnoldi(A, b, s, meth, args.gs, impl=omp)
    dt = time.perf_counter() - t0
    value = args.steps * s / dt
    sample = (f"first {s} of the {M} Arnoldi columns of the cycle, per step; OpenMP build of the "
              f"oracle (bitwise the serial build's results) on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": main_config(args.gs, args.method, ws, args.precision),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, pkg, torch, local, dist, with_one_at_a_time=True):
    """The batched form: `steps` timed batch solves (CUDA events on the launch stream), the
    FP64 roofline of the persistent kernel, an end-to-end figure with host buffers, and a
    sample of the same systems solved one at a time by igs_solve."""
    ws, rank, _ = dist_env()
    count = args.batch_count
    out = gen.banded_batch(count=count, seed=SEED + rank)
    As = [o[0] for o in out]
    b = np.concatenate([o[1] for o in out])
    stream = torch.cuda.current_stream()
    t_create = time.perf_counter()
    tb = [int(v) for v in args.batch_launch.split(":")] if args.batch_launch else [0, 0]
    bs = pkg.BatchSolver(As, m=BATCH_M, device=local, stream=stream.cuda_stream, block_threads=tb[0],
                         blocks_per_sm=tb[1])
    t_create = time.perf_counter() - t_create
    info = bs.info
    b_dev = torch.from_numpy(b).cuda()
    res = {"x": torch.empty_like(b_dev),
           "beta": torch.empty(count, dtype=torch.float64, device=b_dev.device),
           "status": torch.empty(count, dtype=torch.int32, device=b_dev.device),
           "steps": torch.empty(count, dtype=torch.int64, device=b_dev.device),
           "cycles": torch.empty(count, dtype=torch.int32, device=b_dev.device)}

    def step():
        return bs.solve(b_dev, gs=args.gs, tol=BATCH_TOL, max_restarts=BATCH_MAX_RESTARTS, out=res)

    for _ in range(args.warmup):
        r = step()
    assert r["n_ok"] == count, r
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        r = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    dev_ms = [r["device_ms"]]  # kernel-only time of the last solve (graph launch events)
    steps_b = res["steps"].cpu().numpy()
    cycles_b = res["cycles"].cpu().numpy()
    total_steps = int(steps_b.sum())

    # end to end: host b in, host x / beta / status / steps / cycles out
    b_host = np.ascontiguousarray(b)
    bs.solve(b_host, gs=args.gs, tol=BATCH_TOL, max_restarts=BATCH_MAX_RESTARTS)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bs.solve(b_host, gs=args.gs, tol=BATCH_TOL, max_restarts=BATCH_MAX_RESTARTS)
    e2e_s = time.perf_counter() - t0
    ms, e2e_s, solves_total = reduce_replicas(ms, e2e_s, args.steps * count, dist, "cuda")

    ns = [A.n for A in As]
    nnzs = [A.nnz for A in As]
    fma = batch_fma(ns, nnzs, steps_b, cycles_b, BATCH_M, args.gs)
    try:
        probe_tf = 2 * pkg.probe_fma(local)["fp64_fma_per_s"] / 1e12  # outside the timed region
    except Exception:
        probe_tf = None
    # DRAM bytes per launch: the ncu capture of the same kernel on the first 1024 systems of
    # this generator (profiles/k_batch_solve_banded1024_m50.md: 42.4 GB read + 0.90 GB written)
    # scaled by the FMA work of this batch over that of those 1024 systems (each system's
    # arithmetic, steps and cycles are the same alone or in any batch)
    traffic, traffic_src = None, None
    if count >= BATCH_CAPTURE_SYSTEMS and args.gs == 2 and SEED + rank == 0:
        k = BATCH_CAPTURE_SYSTEMS
        fma_k = batch_fma(ns[:k], nnzs[:k], steps_b[:k], cycles_b[:k], BATCH_M, args.gs)
        traffic = BATCH_CAPTURE_DRAM_BYTES * fma / fma_k
        traffic_src = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of k_batch_solve on the first {k} "
                       f"systems ({BATCH_CAPTURE_DRAM_BYTES / 1e9:.1f} GB), scaled by FMA work x{fma / fma_k:.2f}")
    avg_s = ms / 1e3 / args.steps
    achieved = 2 * fma / avg_s / 1e12
    line = {"metric": BATCH_METRIC, "value": solves_total / (ms / 1e3), "unit": BATCH_UNIT,
            "ms_per_step": ms / args.steps, "arnoldi_steps_per_s": total_steps * ws / avg_s,
            "arnoldi_steps_per_batch": total_steps, "kernel_ms_last": dev_ms[0],
            "config": {**batch_config(args.gs, count), "parallelism": f"replicas x{ws}"},
            "launch": {"block_threads": info["block_threads"], "blocks_per_sm": info["blocks_per_sm"],
                       "tuned": not args.batch_launch, "tune_table_ms": info["tune"], "create_s": t_create},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "traffic_source": traffic_src,
                         "probe_fp64_tflops": probe_tf, "frac_of_probe": achieved / probe_tf if probe_tf else None,
                         "kernel": "k_batch_solve (persistent; all steps of Alg. 4.1 per system)",
                         "flops_per_launch": 2 * fma,
                         "peak_source": "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 FLOP x 2070 MHz"},
            "e2e": {"value": solves_total / e2e_s, "unit": BATCH_UNIT, "h2d_bytes_per_step": 8 * len(b),
                    "d2h_bytes_per_step": 8 * len(b) + count * (8 + 4 + 8 + 4)},
            "gpu_launches": args.steps}
    if with_one_at_a_time and not args.no_one_at_a_time:
        # the same systems, one igs_solve each (sample of 32 spread over the batch); solve
        # time only (contexts created and their graphs captured beforehand)
        norms = bs.norms()
        idx = list(range(0, count, max(1, count // 32)))
        t_solve = 0.0
        steps_one = 0
        for i in idx:
            with pkg.Solver(As[i], max_restart_m=BATCH_M, A_norm2=float(norms[i]), device=local,
                            stream=stream.cuda_stream) as sv:
                bi = torch.from_numpy(out[i][1]).cuda()
                xi = torch.empty_like(bi)
                sv.solve(bi, m=BATCH_M, gs=args.gs, tol=BATCH_TOL, max_restarts=BATCH_MAX_RESTARTS,
                         x_out=xi, hist_cap=0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                o = sv.solve(bi, m=BATCH_M, gs=args.gs, tol=BATCH_TOL, max_restarts=BATCH_MAX_RESTARTS,
                             x_out=xi, hist_cap=0)
                e1.record(stream)
                torch.cuda.synchronize()
                t_solve += e0.elapsed_time(e1) / 1e3
                steps_one += o["steps"]
        one = len(idx) / t_solve
        line["one_at_a_time"] = {"value": one, "unit": BATCH_UNIT, "path": "igs_solve per system (FP64)",
                                 "sample": f"{len(idx)} systems spread over the batch ({steps_one} Arnoldi steps)"}
        line["speedup_vs_one_at_a_time"] = line["value"] / (one * ws)
    bs.close()
    return line


PREC_N, PREC_PECLET, PREC_M, PREC_TOL = 160, 20.0, 200, 1e-14


def prec_config(N=PREC_N):
    return {"workload": f"precision form: cd3d {N}^3 upwind convection-diffusion, Pe {PREC_PECLET:g}",
            "n": N ** 3, "nnz": 7 * N ** 3 - 6 * N ** 2, "restart_m": PREC_M, "gs_iters": 2,
            "tol_beta": PREC_TOL,
            "step": "one solve to beta <= 1e-14: FP32 basis inside FP64 iterative refinement vs all-FP64",
            "l2": "inputs larger than L2 (FP32 basis 3.3 GB, FP64 basis 6.6 GB)"}


def run_precision(args, pkg, torch, local, dist):
    """The precision form (igs_solve, precision = fp32_ir) against the FP64 form on the same
    3-D system to beta <= 1e-14: device time of each solve, the FP32 multi-dot's HBM roofline
    (eager re-run of one cycle with CUDA events per launch), and the difference between the
    two solutions (the FP64 form is the reference at this size: the CPU oracle would need
    hours; both forms are parity-tested against it on smaller grids)."""
    ws, rank, _ = dist_env()
    N = args.prec_grid
    A, b, _, _ = gen.cd3d(N, PREC_PECLET, SEED + rank)
    stream = torch.cuda.current_stream()
    t_create = time.perf_counter()
    sv = pkg.Solver(A, max_restart_m=PREC_M, device=local, stream=stream.cuda_stream, fp32_basis=True)
    t_create = time.perf_counter() - t_create
    bd = torch.from_numpy(b).cuda()
    x32, x64 = torch.empty_like(bd), torch.empty_like(bd)
    for prec in ("fp32_ir", "fp64"):  # capture each form's cycle graph
        sv.solve(bd, m=PREC_M, gs=2, tol=0.0, max_restarts=1, x_out=x32, precision=prec, hist_cap=0)
    out = {}
    for prec, xo in (("fp32_ir", x32), ("fp64", x64)):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = sv.solve(bd, m=PREC_M, gs=2, tol=PREC_TOL, max_restarts=100, x_out=xo, precision=prec, hist_cap=0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ms, _, _ = reduce_replicas(ms, 0.0, 1, dist, "cuda")
        out[prec] = {"ms": ms, "solves_per_s": ws / (ms / 1e3), "status": r["status"], "beta": r["beta"],
                     "steps": r["steps"], "cycles": r["cycles"], "arnoldi_steps_per_s": r["steps"] / (ms / 1e3)}
    diff = float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64))
    # roofline of the FP32 multi-dot (the form's largest kernel), one eager cycle
    sv.profile_enable(True)
    sv.solve(bd, m=PREC_M, gs=2, tol=0.0, max_restarts=1, x_out=x32, precision="fp32_ir", hist_cap=0)
    prof = sv.profile()
    sv.profile_enable(False)
    sv.close()
    d = prof["dots"]
    hbm_peak = 6681.5
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", hbm_peak)
    except Exception:
        pass
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    total_ms = sum(v["ms"] for v in prof.values())
    return {"metric": "solves/s", "value": out["fp32_ir"]["solves_per_s"], "unit": "solves/s",
            "config": prec_config(N), "fp32_ir": out["fp32_ir"], "fp64": out["fp64"],
            "speedup_vs_fp64": out["fp64"]["ms"] / out["fp32_ir"]["ms"],
            "x_rel_diff_vs_fp64": diff, "create_s": t_create,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None,
                         "kernel": "k_dots32 (FP32-basis multi-dot, Alg. 4.1 steps 5 and 14)",
                         "bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                         "share_of_cycle": d["ms"] / total_ms if total_ms else None,
                         "kernel_ms_per_cycle": {k: v["ms"] for k, v in prof.items()}}}


SERVE_LAMBDA, SERVE_SIDES, SERVE_PE, SERVE_TOLS, SERVE_M = 2000.0, (64, 1024), (1.0, 100.0), (1e-10, 1e-14), 100
SERVE_ARENA = 150 * (1 << 30)


def serve_config(duration):
    return {"workload": "served: Poisson arrivals of 2-D upwind convection-diffusion solves",
            "lambda_per_s": SERVE_LAMBDA, "window_s": duration, "grid_side": list(SERVE_SIDES),
            "peclet": list(SERVE_PE), "tol_beta": list(SERVE_TOLS), "restart_m": SERVE_M, "gs_iters": 2,
            "precision_mix": "FP64 / FP32 basis in FP64 refinement, 50/50",
            "basis_budget_bytes": SERVE_ARENA,
            "step": "the whole stream: arrivals for window_s, then the admitted backlog drains"}


DOTS_TRAFFIC_RATIO = 1.012  # measured DRAM bytes / algorithmic bytes of the multi-dots (ncu)


def norm_bound(A):
    """sqrt(||A||_1 ||A||_inf) >= ||A||_2: the norm the server's beta uses for a request
    without one, so that the one-at-a-time solves stop at the same beta."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    av = np.abs(A.val)
    return float(np.sqrt(np.bincount(A.colind, av, A.n).max() * np.bincount(rows, av, A.n).max()))


def serve_n(side):
    """Unknowns of the side x side grid of a served request."""
    return side * side


def serve_stream(seed, duration):
    """Seeded arrival stream: (arrival time, grid side, Peclet, tol, precision, rhs seed)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / SERVE_LAMBDA)
        if t >= duration:
            return out
        out.append((t, int(rng.integers(SERVE_SIDES[0], SERVE_SIDES[1] + 1)),
                    float(rng.uniform(*SERVE_PE)), SERVE_TOLS[int(rng.integers(0, 2))],
                    "fp32_ir" if rng.integers(0, 2) else "fp64", int(rng.integers(1 << 30))))


def run_served(args, pkg, torch, local, dist, duration, drain_s, oaat_budget_s=900.0):
    """Replay the arrival stream against the request server: a request is materialised (its
    matrix generated) and submitted at its arrival time when the server's backlog has room,
    else it is refused (counted).  Latency = completion - arrival; service time = completion
    - admission.  Then every completed request is solved again one at a time through
    igs_solve (FP64, the same ||A|| and tolerance), each timed; nothing is extrapolated (a
    safety budget, oaat_budget_s, stops the pass early only on a pathological run, and the
    line then says how many were timed and rates only those)."""
    ws, rank, _ = dist_env()
    stream = serve_stream(SEED + rank, duration)
    max_queue = args.serve_backlog
    sv = pkg.Server(max_restart_m=SERVE_M, arena_bytes=SERVE_ARENA, slots=args.serve_slots,
                    rows_per_cta=4096, max_queue=max_queue, device=local, graph_min_n=args.serve_graph_min_n,
                    graph_lanes=args.serve_graph_lanes)
    arrivals, done, refused = {}, [], 0
    t_start = sv.clock()
    k = 0
    while True:
        now = sv.clock() - t_start
        while k < len(stream) and stream[k][0] <= now:
            t_arr, side, pe, tol, prec, rs = stream[k]
            k += 1
            if sv.stats()["queued"] >= max_queue:
                refused += 1
                continue
            A, b, _, _ = gen.cd2d(side, pe, rs)
            rid = sv.submit(A, b, m=SERVE_M, gs=2, tol=tol, max_restarts=2000, precision=prec)
            if rid is None:
                refused += 1
                continue
            arrivals[rid] = (t_start + t_arr, side, prec, tol)
            sv.pump()
        sv.pump()
        for c in sv.poll():
            done.append(c)
            sv.take(c["id"])
        st = sv.stats()
        if now >= duration and (st["queued"] + st["running"] == 0 or now >= duration + drain_s):
            break
        time.sleep(0.001)
    t_end = sv.clock()
    st = sv.stats()
    sv.close()
    lat = np.array([c["t_done"] - arrivals[c["id"]][0] for c in done]) if done else np.array([np.nan])
    svc = np.array([c["t_done"] - c["t_admit"] for c in done]) if done else np.array([np.nan])
    ok = sum(1 for c in done if c["status"] == 0)
    line = {"metric": "served solves/s", "value": len(done) / (t_end - t_start), "unit": "solves/s",
            "config": {**serve_config(duration), "slots": args.serve_slots, "backlog": max_queue,
                       "graph_min_n": args.serve_graph_min_n, "graph_lanes": args.serve_graph_lanes},
            "offered": len(stream), "submitted": st["submitted"],
            "refused_backlog_full": refused, "completed": len(done), "completed_ok": ok,
            "unfinished_at_end": st["queued"] + st["running"], "wall_s": t_end - t_start,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "service_p50_s": float(np.percentile(svc, 50)), "service_p99_s": float(np.percentile(svc, 99)),
            "queue_wait_p50_s": float(np.percentile(lat - svc, 50)),
            "arena_peak_bytes": st["arena_peak"], "gpu_launches": st["launches"],
            "by_precision": {p: sum(1 for c in done if arrivals[c["id"]][2] == p) for p in ("fp64", "fp32_ir")},
            "by_path": {"gang": sum(1 for c in done if c["path"] == 0),
                        "graph_lane": sum(1 for c in done if c["path"] == 1)},
            "max_backlog": max_queue}
    if oaat_budget_s > 0 and done and not args.no_one_at_a_time:
        # the same requests, one at a time through igs_solve in FP64 with graph-captured
        # cycles (set-up and capture outside the timing), in an order spread over the run
        order = list(range(0, len(done), 2)) + list(range(1, len(done), 2))
        t_tot, n_ok, n_run = 0.0, 0, 0
        t_budget = time.perf_counter() + oaat_budget_s
        for j in order:
            if time.perf_counter() > t_budget:
                break
            c = done[j]
            t_arr, side, prec, tol = arrivals[c["id"]]
            src = next(x for x in stream if abs(x[0] + t_start - t_arr) < 1e-9)
            A, b, _, _ = gen.cd2d(side, src[2], src[5])
            st_ = torch.cuda.current_stream()
            with pkg.Solver(A, max_restart_m=SERVE_M, A_norm2=c["A_norm2"], device=local,
                            stream=st_.cuda_stream) as so:
                bd = torch.from_numpy(b).cuda()
                xd = torch.empty_like(bd)
                so.solve(bd, m=SERVE_M, gs=2, tol=tol, max_restarts=1, x_out=xd, hist_cap=0)  # capture
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = so.solve(bd, m=SERVE_M, gs=2, tol=tol, max_restarts=2000, x_out=xd, hist_cap=0)
                torch.cuda.synchronize()
                t_tot += time.perf_counter() - t0
                n_ok += r["status"] == 0
            n_run += 1
        line["one_at_a_time"] = {"value": n_run / t_tot, "unit": "solves/s", "converged": n_ok,
                                 "path": "igs_solve per request (FP64, whole GPU, the server's ||A|| and "
                                         "tolerance; context set-up and graph capture outside the timing)",
                                 "requests": ("all " if n_run == len(done) else f"{n_run} of the ")
                                             + f"{len(done)} completed requests solved again one at a time, "
                                               f"each timed ({t_tot:.1f} s in total)",
                                 "one_at_a_time_s": t_tot}
        line["speedup_vs_one_at_a_time"] = line["value"] / line["one_at_a_time"]["value"]
    return line


SOLVE_TOL, SOLVE_MAX_RESTARTS = 1e-13, 500


def run_cd2d_extra(args, solver, b_dev, x_dev, stream, dist, value_gs):
    """On the benchmark system: Alg. 4.1 with the other number of GS iterations (the same K
    single cycles, device-timed), and the whole solve to the workload's own stopping
    criterion beta <= 1e-13 (restarts until it holds; device-timed, best of two)."""
    import torch
    out = {}
    gs_other = 1 if args.gs == 2 else 2
    # the double-float reductions (IGS_PREC_FP64_DF) on the same cycles, both algorithms, with
    # per-class kernel time from an eager re-run (CUDA events per launch)
    for name, meth in (("fp64_df", "igs"), ("one_reduce_fp64_df", "one_reduce")):
        def cyc_df():
            return solver.solve(b_dev, m=M, gs=args.gs, tol=0.0, max_restarts=1, x_out=x_dev, hist_cap=0,
                                method=meth, precision="fp64_df")

        for _ in range(args.warmup):
            cyc_df()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            cyc_df()
        e1.record(stream)
        torch.cuda.synchronize()
        ms, _, st = reduce_replicas(e0.elapsed_time(e1), 0.0, args.steps * M, dist, "cuda")
        solver.profile_enable(True)
        cyc_df()
        prof = solver.profile()
        solver.profile_enable(False)
        d = prof["dots"]
        hbm = peaks_hbm()
        out[name] = {"metric": METRIC, "value": st / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
                     "method": "Alg. 4.1" if meth == "igs" else "Alg. 4.2",
                     "precision": "FP64 data; block reductions in double-float on the FP32 pipes",
                     "speedup_vs_fp64": (st / (ms / 1e3)) / value_gs if meth == "igs" else None,
                     "dots_hbm_gbs": d["bytes"] / (d["ms"] / 1e3) / 1e9,
                     "dots_hbm_frac": d["bytes"] / (d["ms"] / 1e3) / 1e9 / hbm,
                     "kernel_ms_per_cycle": {k: v["ms"] for k, v in prof.items()}}

    def cyc():
        return solver.solve(b_dev, m=M, gs=gs_other, tol=0.0, max_restarts=1, x_out=x_dev, hist_cap=0)

    for _ in range(args.warmup):
        cyc()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        cyc()
    e1.record(stream)
    torch.cuda.synchronize()
    ms, _, st = reduce_replicas(e0.elapsed_time(e1), 0.0, args.steps * M, dist, "cuda")
    out[f"gs{gs_other}"] = {"metric": METRIC, "value": st / (ms / 1e3), "unit": UNIT,
                            "ms_per_step": ms / args.steps, "gs_iters": gs_other,
                            "method": f"Alg. 4.1 with {gs_other} Gauss-Seidel iteration(s)"}
    best = None
    for _ in range(2):
        torch.cuda.synchronize()
        e0.record(stream)
        r = solver.solve(b_dev, m=M, gs=args.gs, tol=SOLVE_TOL, max_restarts=SOLVE_MAX_RESTARTS, x_out=x_dev,
                         hist_cap=0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if best is None or ms < best[0]:
            best = (ms, r)
    ms, r = best
    ms, _, _ = reduce_replicas(ms, 0.0, 1, dist, "cuda")
    out["solve_to_tol"] = {"metric": "seconds to beta <= 1e-13", "value": ms / 1e3, "unit": "s",
                           "higher_is_better": False, "tol_beta": SOLVE_TOL, "status": r["status"],
                           "beta": r["beta"], "steps": r["steps"], "cycles": r["cycles"],
                           "arnoldi_steps_per_s": r["steps"] / (ms / 1e3), "gs_iters": args.gs,
                           "timing": "device (CUDA events), best of two solves from x0 = 0"}
    return out


def run_dense200(args, pkg, torch, local, dist, rank):
    """The dense ill-conditioned system (A = U diag(s) W^T, n = 200, s log-spaced 1..1e-10,
    k = 200 unrestarted): Arnoldi steps/s of one full cycle with one and two GS iterations
    and Alg. 4.2 on the GPU (device-timed, A and the basis resident in L2, so latency-bound),
    and the oracle's MGS-GMRES and Alg. 4.1 on one core for comparison."""
    A, b, _, info = gen.dense_usv(200, SEED)
    stream = torch.cuda.current_stream()
    out = {"workload": "dense A = U diag(s) W^T, n = 200, kappa 1e10, k = 200 unrestarted",
           "metric": METRIC, "unit": UNIT}
    with pkg.Solver(A, max_restart_m=200, A_norm2=info["normA"], device=local, stream=stream.cuda_stream) as sv:
        bd = torch.from_numpy(b).cuda()
        xd = torch.empty_like(bd)
        for name, gs, meth in (("igs_gs1", 1, "igs"), ("igs_gs2", 2, "igs"), ("one_reduce", 2, "one_reduce")):
            def cyc():
                return sv.solve(bd, m=200, gs=gs, tol=0.0, max_restarts=1, x_out=xd, hist_cap=0, method=meth)
            for _ in range(args.warmup):
                r = cyc()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20
            e0.record(stream)
            for _ in range(reps):
                r = cyc()
            e1.record(stream)
            torch.cuda.synchronize()
            ms, _, st = reduce_replicas(e0.elapsed_time(e1), 0.0, reps * r["steps"], dist, "cuda")
            out[name] = {"value": st / (ms / 1e3), "steps_per_cycle": r["steps"], "beta": r["beta"],
                         "status": r["status"]}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        for name, meth, gs in (("oracle_mgs", oracle.MGS, 1), ("oracle_igs_gs2", oracle.IGS, 2)):
            t0 = time.perf_counter()
            o = oracle.arnoldi(A, b, 200, meth, gs)
            dt = time.perf_counter() - t0
            out[name] = {"value": o["ncols"] / dt, "steps": o["ncols"], "cores": 1}
    return out


def _oracle_batch_solve(job):
    """One batched system through the serial oracle (a worker of oracle_batch_rate)."""
    import oracle
    A, b, nA = job
    oracle.gmres(A, b, m=BATCH_M, gs=2, tol=BATCH_TOL, max_cycles=BATCH_MAX_RESTARTS, normA=nA)
    return 1


def oracle_batch_rate(stride=32):
    """Solves/s of the CPU oracle on every stride-th system of the batch: serially on one
    core, and on all host cores (the systems are independent: a spawned process pool, one
    serial oracle per process)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import oracle
    oracle.build()
    out = gen.banded_batch(count=BATCH_COUNT, seed=SEED)
    jobs = [(out[i][0], out[i][1], gen.norm2_power(out[i][0], iters=100)) for i in range(0, BATCH_COUNT, stride)]
    t0 = time.perf_counter()
    for j in jobs[: max(1, len(jobs) // 4)]:
        _oracle_batch_solve(j)
    t1 = time.perf_counter() - t0
    serial = max(1, len(jobs) // 4) / t1
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_batch_solve, jobs[:cores]))  # start the workers
        t0 = time.perf_counter()
        done = sum(ex.map(_oracle_batch_solve, jobs))
        tn = time.perf_counter() - t0
    return {"value": done / tn, "unit": BATCH_UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(jobs)} of the {BATCH_COUNT} systems (every {stride}th) on {cores} processes, {tn:.1f} s",
            "serial": {"value": serial, "unit": BATCH_UNIT, "cores": 1,
                       "sample": f"{max(1, len(jobs) // 4)} of those systems, {t1:.1f} s"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--gs", type=int, default=2)
    ap.add_argument("--method", default="igs", choices=["igs", "one_reduce"],
                    help="the main line's Arnoldi process: Alg. 4.1 (igs) or Alg. 4.2 (one_reduce)")
    ap.add_argument("--impl", default="igs")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp64_df"],
                    help="the main line's arithmetic: FP64, or FP64 data with double-float reductions and updates")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="cd2d", choices=["cd2d", "batched", "precision", "served"])
    ap.add_argument("--prec-grid", type=int, default=PREC_N,
                    help="grid side of the precision-form workload (smaller sides: profiling cases)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched sub-measurement")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT,
                    help="systems in the batched workload (smaller counts: profiling cases)")
    ap.add_argument("--batch-launch", default="",
                    help="T:B = block threads and CTAs per SM for the batched kernel (default: tuned)")
    ap.add_argument("--no-one-at-a-time", action="store_true")
    ap.add_argument("--probe", action="store_true",
                    help="only measure the FP64 / FP32 FMA throughput (igs_probe_fma) with the clocks, one JSON line")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other-gs cycle, the solve to beta <= 1e-13 and the dense n = 200 lines")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision-form sub-measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served-stream sub-measurement")
    ap.add_argument("--serve-window", type=float, default=0.0,
                    help="arrival window in seconds (default: 60 for --workload served, 20 in the main line)")
    ap.add_argument("--serve-slots", type=int, default=16, help="gang requests in flight on the GPU at once")
    ap.add_argument("--serve-backlog", type=int, default=16,
                    help="requests waiting for admission at most (arrivals beyond it are refused)")
    ap.add_argument("--serve-graph-min-n", type=int, default=100000,
                    help="requests with n >= this take the server's graph lanes (0: gangs only)")
    ap.add_argument("--serve-graph-lanes", type=int, default=3,
                    help="graph-lane requests in flight at once")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2205_07805_gb300 import build as libbuild
    if rank == 0:
        libbuild.build()
    if dist:
        dist.barrier()
    import paper_2205_07805_gb300 as pkg

    if args.probe:
        clocks = Clocks(local)
        clocks.start()
        reps = [pkg.probe_fma(local) for _ in range(5)]
        clk = clocks.stop()
        f64 = statistics.median(r["fp64_fma_per_s"] for r in reps)
        f32 = statistics.median(r["fp32_fma_per_s"] for r in reps)
        line = {"probe": "igs_probe_fma: best of 2/4/8 blocks per SM x 4/8/16 FMA chains per thread, median of 5 calls",
                "fp64_tflops": 2 * f64 / 1e12, "fp32_tflops": 2 * f32 / 1e12,
                "fp64_fma_per_clk_per_sm_at_max_clock": f64 / (torch.cuda.get_device_properties(local).multi_processor_count
                                                               * 2070e6),
                "fp64_unit_count_peak_tflops": FP64_PEAK_TFLOPS, "fp64_frac_of_unit_count": 2 * f64 / 1e12 / FP64_PEAK_TFLOPS,
                "fp32_over_fp64": f32 / f64, "clocks": clk}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    if args.workload == "served":
        clocks = Clocks(local)
        clocks.start()
        window = args.serve_window or 60.0
        sl = run_served(args, pkg, torch, local, dist, window, drain_s=120.0)
        clk = clocks.stop()
        line = {"metric": sl["metric"], "value": sl["value"], "unit": sl["unit"], "n_gpus": ws, "steps": 1,
                "warmup": 0, "ms_per_step": 1e3 * sl["wall_s"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 / f32 basis in f64 refinement", "data": "synthetic",
                "config": sl["config"], "clocks": clk,
                **{k: v for k, v in sl.items() if k not in ("metric", "value", "unit", "config")}}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    if args.workload == "precision":
        clocks = Clocks(local)
        clocks.start()
        pl = run_precision(args, pkg, torch, local, dist)
        clk = clocks.stop()
        line = {"metric": "solves/s", "value": pl["value"], "unit": "solves/s", "n_gpus": ws, "steps": 1,
                "warmup": 1, "ms_per_step": pl["fp32_ir"]["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 basis / f64 refinement", "data": "synthetic",
                "config": pl["config"], "roofline": pl["roofline"], "clocks": clk,
                **{k: pl[k] for k in ("fp32_ir", "fp64", "speedup_vs_fp64", "x_rel_diff_vs_fp64")}}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    if args.workload == "batched":
        clocks = Clocks(local)
        clocks.start()
        bl = run_batched(args, pkg, torch, local, dist)
        clk = clocks.stop()
        line = {"metric": BATCH_METRIC, "value": bl["value"], "unit": BATCH_UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": bl["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": bl["config"], "roofline": bl["roofline"], "e2e": bl["e2e"],
                "gpu_launches": bl["gpu_launches"], "clocks": clk,
                **{k: bl[k] for k in ("arnoldi_steps_per_s", "launch", "one_at_a_time",
                                      "speedup_vs_one_at_a_time") if k in bl}}
        if rank == 0 and not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_batch_rate()
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    A, b, x0, _ = gen.cd2d(GRID_N, PECLET, SEED + rank)
    normA = gen.norm2_power(A, iters=50)
    stream = torch.cuda.current_stream()
    solver = pkg.Solver(A, max_restart_m=M, A_norm2=normA, device=local, stream=stream.cuda_stream)
    b_dev = torch.from_numpy(b).cuda()
    x_dev = torch.empty_like(b_dev)

    def step():
        return solver.solve(b_dev, m=M, gs=args.gs, tol=0.0, max_restarts=1, x_out=x_dev, hist_cap=0,
                            method=args.method, precision=args.precision)

    for _ in range(args.warmup):
        out = step()
    assert out["steps"] == M, out
    torch.cuda.synchronize()

    # ---- timed region (device) ----
    clocks = Clocks(local)
    clocks.start()
    launches0 = solver.launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = solver.launches - launches0
    clk = clocks.stop()

    # ---- end to end through the C interface with host buffers ----
    b_host = np.ascontiguousarray(b)
    x_host = np.empty_like(b_host)
    solver.solve(b_host, m=M, gs=args.gs, tol=0.0, max_restarts=1, x_out=x_host, hist_cap=0, method=args.method,
                 precision=args.precision)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.solve(b_host, m=M, gs=args.gs, tol=0.0, max_restarts=1, x_out=x_host, hist_cap=0,
                     method=args.method, precision=args.precision)
    e2e_s = time.perf_counter() - t0
    ms, e2e_s, steps_total = reduce_replicas(ms, e2e_s, args.steps * M, dist, "cuda")
    value = steps_total / (ms / 1e3)
    e2e = {"value": steps_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * A.n,
           "d2h_bytes_per_step": 8 * A.n + 2 * 96}

    # ---- per-kernel timing: the same steps issued eagerly with CUDA events per launch ----
    solver.profile_enable(True)
    for _ in range(args.steps):
        step()
    prof = solver.profile()
    solver.profile_enable(False)
    d = prof["dots"]
    avg_s = d["ms"] / 1e3 / max(1, d["launches"])
    flops_per_launch = d["flops"] / max(1, d["launches"])
    bytes_per_launch = d["bytes"] / max(1, d["launches"])
    achieved_tflops = flops_per_launch / avg_s / 1e12
    sm_clock = (clk or {}).get("sm_max_mhz") or 2070.0
    peak_tflops = FP64_PEAK_TFLOPS
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    total_ms = sum(v["ms"] for v in prof.values())
    # the FP64 FMA rate this GPU actually sustains (igs_probe_fma, outside the timed region)
    try:
        probe_tf = 2 * pkg.probe_fma(local)["fp64_fma_per_s"] / 1e12
    except Exception:
        probe_tf = None
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak_tflops,
                "probe_fp64_tflops": probe_tf,
                "frac_of_probe": achieved_tflops / probe_tf if probe_tf else None,
                # DRAM bytes per launch: ncu's dram__bytes_read.sum + dram__bytes_write.sum of the
                # two multi-dots at p = 49 on this workload were 1.011 (k_dots<2>) and 1.013
                # (k_dots<1>) times their algorithmic bytes; scaled to the average launch
                "traffic": bytes_per_launch * DOTS_TRAFFIC_RATIO if args.gs == 2 else None,
                "traffic_source": "ncu capture of k_dots at p = 49 (profiles/launches_cd2d512_m100_gs2.md), "
                                  "ratio to algorithmic bytes applied to the mean launch",
                "kernel": "k_dots (block multi-dot, Alg. 4.1 steps 5 and 14)",
                "peak_source": "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 FLOP x 2070 MHz (unit counts and max clock)",
                "hbm_gbs": bytes_per_launch / avg_s / 1e9, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": bytes_per_launch / avg_s / 1e9 / hbm_peak,
                "share_of_step": d["ms"] / total_ms if total_ms else None,
                "kernel_ms": {k: v["ms"] / args.steps for k, v in prof.items()},
                "per_class": {k: {"hbm_gbs": v["bytes"] / (v["ms"] / 1e3) / 1e9,
                                  "hbm_frac": v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm_peak,
                                  "fp64_tflops": v["flops"] / (v["ms"] / 1e3) / 1e12,
                                  "fp64_frac": v["flops"] / (v["ms"] / 1e3) / 1e12 / peak_tflops}
                              for k, v in prof.items() if k in ("spmv", "dots", "update") and v["ms"] > 0},
                "sm_clock_mhz": sm_clock}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": main_config(args.gs, args.method, ws, args.precision),
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_cd2d(A, b, M, args.method, args.gs)
    # ---- Alg. 4.2 (one-reduce) on the same workload: the same K cycles, device-timed ----
    if args.method == "igs":  # (with --method one_reduce the main line is Alg. 4.2 itself)
        def step_1r():
            return solver.solve(b_dev, m=M, tol=0.0, max_restarts=1, x_out=x_dev, hist_cap=0, method="one_reduce")

        for _ in range(args.warmup):
            o1 = step_1r()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step_1r()
        e1.record(stream)
        torch.cuda.synchronize()
        ms1 = e0.elapsed_time(e1)
        ms1, _, steps1 = reduce_replicas(ms1, 0.0, args.steps * o1["steps"], dist, "cuda")
        line["one_reduce"] = {"metric": METRIC, "value": steps1 / (ms1 / 1e3), "unit": UNIT,
                              "ms_per_step": ms1 / args.steps, "method": "Alg. 4.2 (one global reduction per column)",
                              "speedup_vs_alg41_gs2": (steps1 / (ms1 / 1e3)) / value if args.gs == 2 else None}
    if args.method == "igs" and not args.no_extra:
        line.update(run_cd2d_extra(args, solver, b_dev, x_dev, stream, dist, value))
    solver.close()
    if not args.no_extra:
        line["dense_200"] = run_dense200(args, pkg, torch, local, dist, rank)
    if not args.no_precision:
        line["precision"] = run_precision(args, pkg, torch, local, dist)
    if not args.no_served:
        line["served"] = run_served(args, pkg, torch, local, dist, args.serve_window or 60.0, drain_s=60.0)
    if not args.no_batched:
        bl = run_batched(args, pkg, torch, local, dist)
        line["batched"] = {k: bl[k] for k in ("metric", "value", "unit", "ms_per_step", "arnoldi_steps_per_s",
                                              "config", "launch", "roofline", "e2e", "one_at_a_time",
                                              "speedup_vs_one_at_a_time") if k in bl}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
