#!/usr/bin/env python
"""Benchmark: solve the large GP system (n=32768, SE kernel, d=8, ell=0.5,
sn2=1e-3, one RHS) on one B300 and print one JSON line.

One step = one solve of A x = b from the device-resident FP64 matrix A by
the headline path; the metric is the factorization rate n^3/3 / step time
(GFLOP/s).  Beside it: the live roofline of the dominant kernel (CUDA events
around every launch of it inside the timed region), an end-to-end number
through the public API from pinned host buffers (points and right-hand side
in, solution out), the oracle timed on a bounded sample on the host cores,
and the SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n N]

With --gpus N > 1 (launched by torchrun) every rank solves its own
independent system (replicas; no data-path collective) and rank 0 prints the
aggregate.  --impl reference times the CPU oracle on the same workload
(bounded sample per step).
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
sys.path.insert(0, ROOT)

METRIC = "Cholesky GFLOP/s & CG GB/s, mixed vs FP64 at ≤1e-12 bwd err; served p50/p99 ms"
FP64_PEAK_GFLOPS = 1250.0   # nominal B300 FP64 (DFMA) rate, 148 SMs x ~2 FP64 FMA/clk/SM x 2 x clock
CPU_SAMPLE_N = 4096


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n_sample: int = CPU_SAMPLE_N):
    """The oracle (plain C, one thread) on the n_sample leading block of the
    same workload: SE matrix, textbook Cholesky, forward/back substitution."""
    import oracle
    from paper_2605_13209_b300 import inputs
    s = inputs.config2()
    X = s.X[:n_sample]
    b = s.B[:n_sample, 0]
    A = oracle.se_matrix(X, s.sf2, s.ell, s.sn2)
    t0 = time.perf_counter()
    L, info = oracle.cholesky(A)
    x = oracle.chol_solve(L, b)
    dt = time.perf_counter() - t0
    gflops = n_sample ** 3 / 3.0 / dt / 1e9
    return {"value": round(gflops, 3), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"or_cholesky + forward/back substitution on the n={n_sample} leading block of the "
                      f"n=32768 system (SE d=8, ell=0.5, sn2=1e-3), 1 thread, {dt:.2f} s",
            "seconds": round(dt, 3), "info": int(info)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2605_13209_b300 import inputs
    n = args.cpu_sample_n
    s = inputs.config2()
    A = oracle.se_matrix(s.X[:n], s.sf2, s.ell, s.sn2)
    b = s.B[:n, 0]

    def step():
        L, info = oracle.cholesky(A)
        return oracle.chol_solve(L, b)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = step()
    dt = (time.perf_counter() - t0) / args.steps
    value = n ** 3 / 3.0 / dt / 1e9
    bwd = oracle.backward_error(A, x, b)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "n=32768 SE GP system (d=8, ell=0.5, sn2=1e-3), one RHS; the oracle solves the "
                                   f"n={n} leading block per step", "n": 32768, "sample_n": n},
            "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": f"or_cholesky + forward/back substitution, n={n} leading block, 1 thread"},
            "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "check": {"backward_error": bwd}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--tile", type=int, default=512)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-n", type=int, default=CPU_SAMPLE_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2605_13209_b300 import gpchol, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    n, tile = args.n, args.tile
    sysm = inputs.config2(n) if rank == 0 else inputs.gp_system(n, 8, 0.5, 1e-3, nrhs=1, seed=2 + 1000 * rank)
    ctx = gpchol.Context(local)

    # device-resident inputs: A generated once by the A1 kernel
    Xd = torch.from_numpy(sysm.X).cuda()
    A0 = gpchol.se_matrix(Xd, sysm.sf2, sysm.ell, sysm.sn2, ctx=ctx)
    bd = gpchol.as_colmajor(torch.from_numpy(sysm.B[:, 0]).cuda())
    Aw = gpchol.colmajor(n, n)
    Xs = gpchol.colmajor(n, 1)
    torch.cuda.synchronize()

    def step():
        Aw.copy_(A0)
        gpchol.chol_factor(Aw, tile=tile, ctx=ctx)
        Xs.copy_(bd)
        gpchol.chol_solve(Aw, Xs, ctx=ctx)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    ctx.timing_enable(True)
    launches0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    gpu_launches = ctx.launch_count() - launches0
    tr_ms, tr_n, tr_work = ctx.timing_read(gpchol.PHASE_TRAILING)
    phase = {name: ctx.timing_read(ph) for name, ph in
             [("diag", gpchol.PHASE_DIAG), ("panel", gpchol.PHASE_PANEL), ("trailing", gpchol.PHASE_TRAILING),
              ("solve", gpchol.PHASE_SOLVE)]}
    ctx.timing_enable(False)
    ms_max = ms
    if dist is not None:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    flops = n ** 3 / 3.0
    value = world * flops / (ms_max / 1e3) / 1e9

    # result check (outside the timed region): backward error of the last solve
    x = Xs[:, 0]
    r = bd[:, 0] - torch.mv(A0, x)
    bwd = float(r.abs().max() / (A0.abs().sum(dim=1).max() * x.abs().max() + bd.abs().max()))

    # end to end: pinned host points + rhs in, host solution out
    Xh = torch.from_numpy(sysm.X).pin_memory()
    bh = torch.from_numpy(np.ascontiguousarray(sysm.B[:, 0])).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()

    def e2e_step():
        Xdev = Xh.cuda(non_blocking=True)
        gpchol.se_matrix(Xdev, sysm.sf2, sysm.ell, sysm.sn2, A=Aw, ctx=ctx)
        gpchol.chol_factor(Aw, tile=tile, ctx=ctx)
        Xs[:, 0].copy_(bh, non_blocking=True)
        gpchol.chol_solve(Aw, Xs, ctx=ctx)
        xh.copy_(Xs[:, 0], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_s = float("nan")
    if args.e2e_steps > 0:
        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * flops / e2e_s / 1e9

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    achieved = tr_work / (tr_ms / 1e3) / 1e9 if tr_ms > 0 else None
    roof = {"kernel": "gemm_nt_minus_kernel<true> (Algorithm 1 step 3, FP64 DFMA SYRK/GEMM)",
            "bound": "alu", "achieved": round(achieved, 2) if achieved else None, "peak": FP64_PEAK_GFLOPS,
            "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4) if achieved else None,
            "peak_source": "derived: nominal B300 FP64 rate (1.25 TFLOP/s; 148 SMs x 2 DFMA/clk x 2 flop x clock); "
                           "no FP64 figure in MEASURED_PEAKS.json",
            "launches": tr_n, "avg_launch_ms": round(tr_ms / max(tr_n, 1), 4),
            "flops_per_launch": tr_work / max(tr_n, 1), "traffic": None}
    cpu = None if args.no_cpu_baseline else cpu_baseline(args.cpu_sample_n)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"n={n} SE GP system (d=8, ell=0.5, sn2=1e-3), one RHS: FP64 blocked Cholesky "
                               f"(tile {tile}) + forward/back substitution, A device-resident",
                   "n": n, "tile": tile, "nrhs": 1, "path": "fp64",
                   "l2": "inputs larger than L2 (8.6 GB matrix re-copied each step)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": int(Xh.numel() * 8 + bh.numel() * 8),
                "d2h_bytes_per_step": int(xh.numel() * 8), "seconds_per_step": round(e2e_s, 4),
                "api": "gpchol.se_matrix + chol_factor + chol_solve from pinned host X, b"},
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "phases_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in phase.items()},
        "check": {"backward_error": bwd},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
