"""Benchmark: IGS-GMRES Arnoldi steps/s on one GB300 (FP64).

Workload: 2-D upwind convection-diffusion on a 512 x 512 grid (n = 262144, nnz = 1,308,672,
Peclet 50), b = A 1 + 1e-3 N(0,1), x0 = 0, restart length m = 100, two Gauss-Seidel
iterations (Alg. 4.1).  One benchmark step = one full restart cycle (cycle set-up, 100
Arnoldi columns, Givens least squares, x update and the true backward error), i.e. 100
Arnoldi steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--gs 1|2] [--impl reference]

Prints one JSON line (rank 0).  `value` is device-timed throughput with b already in HBM
(CUDA events on the library's stream); `e2e` is the same metric through the C interface
with host buffers (H2D of b and D2H of x inside the timed region); `roofline` reports the
dominant kernel (the block multi-dot) against the FP64 FMA pipe (it is FP64-issue-bound on
GB300) with its HBM throughput alongside; `cpu_baseline` times the CPU oracle on one full
cycle of the same workload.  With --gpus N > 1 (torchrun) every rank runs an independent
replica (the method has no data-parallel exchange on one system): weak scaling.
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


def oracle_cycle_rate(A, b, m):
    """Arnoldi steps/s of the CPU oracle (as it stands, one thread) over one cycle."""
    import oracle
    t0 = time.perf_counter()
    out = oracle.arnoldi(A, b, m, oracle.IGS, 2)
    dt = time.perf_counter() - t0
    return out["ncols"] / dt, dt


def run_reference(args):
    """The reference arm: the CPU oracle, timed on this machine's cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    A, b, _, _ = gen.cd2d(GRID_N, PECLET, SEED)
    import oracle
    oracle.build()
    # bounded sample per step: the first s columns of the m = 100 cycle, s chosen so that the
    # whole run stays within about two minutes (early columns are cheaper, so this favours
    # the oracle)
    t_probe = time.perf_counter()
    oracle.arnoldi(A, b, 10, oracle.IGS, args.gs)
    t10 = time.perf_counter() - t_probe
    budget = 120.0 / max(1, args.steps + args.warmup)
    s = 10
    while s < M and t10 * ((s + 10) / 10.0) ** 2 <= budget:
        s += 10
    for _ in range(args.warmup):
        oracle.arnoldi(A, b, s, oracle.IGS, args.gs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.arnoldi(A, b, s, oracle.IGS, args.gs)
    dt = time.perf_counter() - t0
    value = args.steps * s / dt
    sample = f"first {s} of the {M} Arnoldi columns of the cycle, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.gs),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--gs", type=int, default=2)
    ap.add_argument("--impl", default="igs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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

    A, b, x0, _ = gen.cd2d(GRID_N, PECLET, SEED + rank)
    normA = gen.norm2_power(A, iters=50)
    stream = torch.cuda.current_stream()
    solver = pkg.Solver(A, max_restart_m=M, A_norm2=normA, device=local, stream=stream.cuda_stream)
    b_dev = torch.from_numpy(b).cuda()
    x_dev = torch.empty_like(b_dev)

    def step():
        return solver.solve(b_dev, m=M, gs=args.gs, tol=0.0, max_restarts=1, x_out=x_dev, hist_cap=0)

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
    solver.solve(b_host, m=M, gs=args.gs, tol=0.0, max_restarts=1, x_out=x_host, hist_cap=0)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.solve(b_host, m=M, gs=args.gs, tol=0.0, max_restarts=1, x_out=x_host, hist_cap=0)
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
    peak_tflops = 152 * FP64_FMA_PER_CLK_PER_SM * 2 * 2070.0e6 / 1e12
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    total_ms = sum(v["ms"] for v in prof.values())
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak_tflops, "traffic": None,
                "kernel": "k_dots (block multi-dot, Alg. 4.1 steps 5 and 14)",
                "peak_source": "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 FLOP x 2070 MHz (unit counts and max clock)",
                "hbm_gbs": bytes_per_launch / avg_s / 1e9, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": bytes_per_launch / avg_s / 1e9 / hbm_peak,
                "share_of_step": d["ms"] / total_ms if total_ms else None,
                "kernel_ms": {k: v["ms"] / args.steps for k, v in prof.items()},
                "sm_clock_mhz": sm_clock}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(args.gs), "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rate, dt = oracle_cycle_rate(A, b, M)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one full cycle ({M} Arnoldi columns) of the same workload, {dt:.1f} s"}
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
