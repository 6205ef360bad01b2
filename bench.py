#!/usr/bin/env python
"""Benchmark on one B300: the large GP system (n=32768, SE kernel, d=8,
ell=0.5, sn2=1e-3, one RHS), solved from the device-resident FP64 matrix.

One step = one refined solve to backward error <= 1e-12: low-precision
Cholesky factor (FP64 diagonal tiles, FP32 panel, tensor-core trailing
update from a scaled binary16 head + tail of the panel (--prec split_f16,
the default; split_bf16 and bf16 selectable), tile 512) + FP64
preconditioned CG.  The metric is the
factorization-equivalent rate n^3/3 / step time (GFLOP/s).  Beside it, in
the same JSON line:
  fp64     the plain FP64 blocked Cholesky (tile 512) + substitution, timed once
  cg       CG GB/s: 100 iterations of Algorithm 1 (left) on the same matrix
  roofline the dominant kernel of the step, from CUDA events around every
           launch of it inside the timed region (gpch_timing_*)
  e2e      the same solve through the public API from pinned host buffers
           (points and right-hand side in, solution out)
  cpu_baseline  the CPU oracle on a bounded sample, on the host cores
  clocks   nvidia-smi samples taken during the timed region

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n N]

With --gpus N > 1 (torchrun) every rank solves its own independent system
(replicas, no data-path collective); rank 0 prints the aggregate.
--impl reference times the CPU oracle (the only reference there is) on a
bounded sample of the same workload.
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
FP64_PEAK_GFLOPS = 1250.0   # nominal B300 FP64 (DFMA): 148 SMs x 2 FMA/clk x 2 flop x clock
FP32_PEAK_GFLOPS = 148 * 128 * 2 * 2.032    # FFMA: 148 SMs x 128 lanes x 2 flop x 2.032 GHz
CPU_SAMPLE_N = 4096
CPU_ALLCORES_N = 2048
# DRAM bytes per algorithmic flop of syrk_tc_kernel's trailing updates
# (split-f16): 7.084 GB of dram__bytes_read.sum + dram__bytes_write.sum over
# all 74 update launches of one n = 16384 refined solve (long passes, short
# passes sharing their grids, next-tile updates) against their 3.818e12 flop.
SYRK_DRAM_BYTES_PER_FLOP = 1.856e-3


def ranks_max(v: float, dist=None, device: str = "cuda") -> float:
    """Largest v over the ranks of the default process group (v itself
    without one): a replicated step takes as long as its slowest rank."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job rate of `world` replicas that each did units_per_rank of
    work in at most `seconds` (the slowest rank's time): weak scaling."""
    return world * units_per_rank / seconds


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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                    power.append(float(p[3]))
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
                "samples": len(sm), "power_w_max": max(power)}


def _oracle_block_solve(n_sample: int) -> float:
    """One oracle solve of the n_sample leading block (seconds); run in a
    worker process of the all-cores leg."""
    import oracle
    from paper_2605_13209_b300 import inputs
    s = inputs.config2(n_sample)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    t0 = time.perf_counter()
    L, info = oracle.cholesky(A)
    oracle.chol_solve(L, s.B[:, 0])
    return time.perf_counter() - t0


def cpu_baseline(n_sample: int = CPU_SAMPLE_N, n_all: int = CPU_ALLCORES_N):
    """The oracle (plain C) on bounded samples of the same workload: SE
    matrix, textbook Cholesky, forward/back substitution.

    * all cores: one oracle solve of the n_all leading block per worker
      process, as many workers as host cores (at most 64), all at once;
      value = workers * n_all^3/3 / wall time;
    * one thread: one solve of the n_sample leading block."""
    import multiprocessing as mp
    cores = min(os.cpu_count() or 1, 64)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_block_solve, [256] * cores)          # workers up, oracle built
        t0 = time.perf_counter()
        per = pool.map(_oracle_block_solve, [n_all] * cores)
        wall = time.perf_counter() - t0
    all_value = cores * n_all ** 3 / 3.0 / wall / 1e9
    dt = _oracle_block_solve(n_sample)
    one = n_sample ** 3 / 3.0 / dt / 1e9
    return {"value": round(all_value, 3), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent oracle solves (or_cholesky + forward/back substitution), one per core, "
                      f"each of the n={n_all} leading block of the n=32768 system (SE d=8, ell=0.5, sn2=1e-3); "
                      f"wall {wall:.2f} s (slowest worker {max(per):.2f} s)",
            "host_cores": os.cpu_count(),
            "single_thread": {"value": round(one, 3), "unit": "GFLOP/s", "cores": 1, "seconds": round(dt, 3),
                              "sample": f"one oracle solve of the n={n_sample} leading block, 1 thread"}}


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
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "n=32768 SE GP system (d=8, ell=0.5, sn2=1e-3), one RHS; the CPU oracle solves "
                                   f"the n={n} leading block per step", "n": 32768, "sample_n": n},
            "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": f"or_cholesky + forward/back substitution, n={n} leading block, 1 thread"},
            "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "check": {"backward_error": oracle.backward_error(A, x, b)}}
    print(json.dumps(line), flush=True)
    return 0


CHECK_BLOCK_N = 4096


def oracle_check(sysm, x_mixed, x_fp64, L_block, x_emu=None, L_block_emu=None):
    """Errors of the benchmark's solutions, from the oracle on the host:
    the system matrix rebuilt by the oracle from the same points, the
    backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) with
    long-double residuals for the mixed solve and the FP64 solve, the
    forward error of the mixed x against the FP64 x, and the FP64 factor's
    relative error on its leading block (the leading block of L is the
    factor of the leading block of A), against the oracle's textbook
    Cholesky of that block."""
    import oracle
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    b = np.ascontiguousarray(sysm.B[:, 0])
    out = {"backward_error": oracle.backward_error(A, x_mixed, b), "by": "oracle (host, long-double residual)"}
    if x_fp64 is not None:
        out["backward_error_fp64"] = oracle.backward_error(A, x_fp64, b)
        out["forward_error_mixed_vs_fp64"] = oracle.forward_error(x_mixed, x_fp64)
    if x_emu is not None:
        out["backward_error_fp64_emulated_update"] = oracle.backward_error(A, x_emu, b)
    if L_block is not None:
        nb = L_block.shape[0]
        Lref, info = oracle.cholesky(A[:nb, :nb])
        out["fp64_factor_error_leading_block"] = oracle.factor_error(L_block, Lref)
        if L_block_emu is not None:
            out["fp64_emulated_factor_error_leading_block"] = oracle.factor_error(L_block_emu, Lref)
        out["factor_block_n"] = nb
    return out


def _batched_system_bwd(item):
    """Oracle backward error of system k of the batched workload (worker)."""
    import oracle
    from paper_2605_13209_b300 import inputs
    k, count, x = item
    sk = inputs.batch_spec(count=count, nmin=256, nmax=4096, seed=4).system(k, d=8)
    A = oracle.se_matrix(sk.X, sk.sf2, sk.ell, sk.sn2)
    return oracle.backward_error(A, x, sk.B[:, 0])


def batched_check(count, xs):
    """Largest oracle backward error over every system of the batch, the
    systems spread over the host cores (spawned workers)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 64)) as pool:
        errs = pool.map(_batched_system_bwd, [(k, count, x) for k, x in enumerate(xs)])
    return max(errs)


def roofline_of(phase_name, ms, launches, work, n, nrhs, pk):
    """Roofline entry for one timed phase: (achieved, peak, unit, bound)."""
    if ms <= 0 or launches == 0:
        return None
    per_launch_s = ms / 1e3 / launches
    hbm = pk.get("hbm_gbs", 6400.0)
    if phase_name == "mixed_trailing":
        tflops = work / launches / per_launch_s / 1e12
        tpeak = pk.get("bf16_tflops_sustained", 1400.0)
        return {"bound": "tensor", "achieved": round(tflops, 2), "peak": tpeak, "unit": "TFLOP/s",
                "frac": round(tflops / tpeak, 4), "peak_source": "measured (bf16_tflops_sustained)"}
    if phase_name == "solve":
        # two sweeps over the FP32 lower triangle per application
        gbs = 2.0 * n * n * 4 / 2 / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs / hbm, 4), "peak_source": "measured (hbm_gbs)"}
    if phase_name == "cg_matvec":
        gbs = work / launches / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs / hbm, 4), "peak_source": "measured (hbm_gbs)"}
    if phase_name == "panel":
        g = work / launches / per_launch_s / 1e9
        return {"bound": "alu", "achieved": round(g, 1), "peak": round(FP32_PEAK_GFLOPS, 1), "unit": "GFLOP/s",
                "frac": round(g / FP32_PEAK_GFLOPS, 4), "peak_source": "derived FP32 FFMA rate"}
    g = work / launches / per_launch_s / 1e9
    return {"bound": "alu", "achieved": round(g, 2), "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": round(g / FP64_PEAK_GFLOPS, 4), "peak_source": "derived nominal FP64 rate"}


def _cg_timed(ctx, A, B, X, variant, products, rtol, maxit, replace_every=50):
    """One CG solve from x = 0, timed with CUDA events on the current
    stream; returns (ms, result, matvec (ms, launches, bytes))."""
    import torch
    from paper_2605_13209_b300 import gpchol
    X.zero_()
    torch.cuda.synchronize()
    ctx.timing_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = gpchol.cg_solve(A, B, X, rtol=rtol, maxit=maxit, replace_every=replace_every, ctx=ctx,
                          raise_on_not_converged=False, variant=variant, products=products)
    e1.record()
    torch.cuda.synchronize()
    mv = ctx.timing_read(gpchol.PHASE_CG_MATVEC)
    ctx.timing_enable(False)
    return e0.elapsed_time(e1), res, mv


def _true_relres(A, B, X):
    """max over columns of ||b - A x|| / ||b|| with the stored operator
    (widened to FP64), on the device through torch (a check of the
    solution, outside every timed region)."""
    import torch
    R = B - A.double() @ X if A.dtype != torch.float64 else B - A @ X
    return float((R.norm(dim=0) / B.norm(dim=0)).max())


def cg_legs(args, ctx, A2, b2, n2, world, pk, max_over_ranks, rank):
    """CG measurements (Algorithm 1 left and its single-reduction form, FP64
    or double-float products):
      matrix2  the n = 32768 matrix, one RHS, args.cg_iters iterations of
               each form (fixed count: rate, matvec GB/s against HBM)
      config1  n = 2048 (33.5 MB, L2-resident), one RHS, solved to 1e-10
      config3  n = 65536, ell = 0.3, sn2 = 0.1, 16 RHS, FP64-stored
               (34.4 GB) and FP32-stored (17.2 GB) A, solved to 1e-10 with
               replacement every 50 iterations (double-float products, and
               FP64-accurate tensor-core products); the FP64-product rate
               over a few iterations beside it"""
    import torch
    from paper_2605_13209_b300 import gpchol, inputs
    hbm = pk.get("hbm_gbs", 6400.0)
    out = {}
    forms = [("classic", "fp64"), ("classic", "double_float"), ("single_reduction", "fp64"),
             ("single_reduction", "double_float")]
    X = gpchol.colmajor(n2, 1)
    m2 = {}
    for var, prod in forms:
        _cg_timed(ctx, A2, b2, X, var, prod, 0.0, 3, 0)
        ms, res, mv = _cg_timed(ctx, A2, b2, X, var, prod, 0.0, args.cg_iters, 0)
        ms = max_over_ranks(ms)
        mv_ms = mv[0] / max(mv[1], 1)
        m2[f"{var}/{prod}"] = {"ms_per_iteration": round(ms / args.cg_iters, 4),
                               "matvec_ms": round(mv_ms, 4),
                               "matvec_gbs": round(n2 * n2 * 8 / (mv_ms / 1e3) / 1e9, 1),
                               "matvec_frac_of_hbm": round(n2 * n2 * 8 / (mv_ms / 1e3) / 1e9 / hbm, 4)}
    m2["what"] = (f"n={n2} FP64 matrix (8.6 GB), one RHS, {args.cg_iters} iterations from x = 0 per form; "
                  "matvec GB/s = n^2 * 8 bytes / mean matvec launch time (CUDA events)")
    out["matrix_n32768"] = m2

    # config 1: n = 2048, L2-resident
    s1 = inputs.config1()
    A1 = gpchol.se_matrix(torch.from_numpy(s1.X).cuda(), s1.sf2, s1.ell, s1.sn2, ctx=ctx)
    b1 = gpchol.as_colmajor(torch.from_numpy(s1.B).cuda())
    X1 = gpchol.colmajor(2048, 1)
    c1 = {}
    for var, prod in forms:
        _cg_timed(ctx, A1, b1, X1, var, prod, 1e-10, 100000)
        ms, res, mv = _cg_timed(ctx, A1, b1, X1, var, prod, 1e-10, 100000)
        mv_ms = mv[0] / max(mv[1], 1)
        c1[f"{var}/{prod}"] = {"ms": round(ms, 3), "iterations": res.iterations, "converged": res.converged == 1,
                               "us_per_iteration": round(1e3 * ms / max(res.iterations, 1), 2),
                               "matvec_gbs_l2": round(2048 * 2048 * 8 / (mv_ms / 1e3) / 1e9, 1),
                               "true_relres": _true_relres(A1, b1, X1)}
    c1["what"] = ("n=2048 SE (ell=0.5, sn2=1e-2), one RHS, to relative residual 1e-10; the 33.5 MB matrix stays in "
                  "L2, so matvec GB/s is an L2 rate")
    out["config1"] = c1
    del A1

    # config 3: n = 65536, 16 RHS
    if args.cg3_n > 0:
        n3 = args.cg3_n
        s3 = inputs.config3(n3, 16) if rank == 0 else inputs.gp_system(n3, 8, 0.3, 1e-1, nrhs=16, seed=3 + 1000 * rank)
        A64 = gpchol.se_matrix(torch.from_numpy(s3.X).cuda(), s3.sf2, s3.ell, s3.sn2, ctx=ctx)
        A32 = gpchol.colmajor(n3, n3, dtype=torch.float32)
        A32.copy_(A64)                 # FP32 storage of the same operator (input preparation)
        B3 = gpchol.as_colmajor(torch.from_numpy(s3.B).cuda())
        X3 = gpchol.colmajor(n3, 16)
        c3 = {}
        for label, AA, el in (("fp64_stored", A64, 8), ("fp32_stored", A32, 4)):
            _cg_timed(ctx, AA, B3, X3, "classic", "double_float", 0.0, 2, 0)
            ms, res, mv = _cg_timed(ctx, AA, B3, X3, "classic", "double_float", 1e-10, 20000, 50)
            ms = max_over_ranks(ms)
            mv_ms = mv[0] / max(mv[1], 1)
            gbs = n3 * n3 * el / (mv_ms / 1e3) / 1e9
            ops = 4.0 * n3 * n3 * 16 / (mv_ms / 1e3) / 1e12
            c3[label] = {"ms": round(ms, 1), "iterations": res.iterations, "converged": res.converged,
                         "ms_per_iteration": round(ms / max(res.iterations, 1), 3),
                         "matvec_ms_mean": round(mv_ms, 3), "matvec_gbs": round(gbs, 1),
                         "matvec_frac_of_hbm": round(gbs / hbm, 4),
                         "products_tera_per_s": round(ops / 4.0, 3),
                         "true_relres_max": _true_relres(AA, B3, X3)}
            # FP64-accurate tensor-core products (the digit copy of A, 16 bytes
            # per entry, lives in a context of its own, released after)
            ctx_t = gpchol.Context(ctx.device)
            _cg_timed(ctx_t, AA, B3, X3, "classic", "tensor", 0.0, 2, 0)
            mst, rest, mvt = _cg_timed(ctx_t, AA, B3, X3, "classic", "tensor", 1e-10, 20000, 50)
            ctx_t.close()
            mst = max_over_ranks(mst)
            digit_bytes = 16 * ((n3 + 127) // 128 * 128) * ((n3 + 511) // 512 * 512)
            c3[label]["tensor_products"] = {
                "ms": round(mst, 1), "iterations": rest.iterations, "converged": rest.converged,
                "ms_per_iteration": round(mst / max(rest.iterations, 1), 3),
                "speedup_vs_double_float": round(ms / max(mst, 1e-9), 2),
                "digit_bytes_per_product": digit_bytes,
                "true_relres_max": _true_relres(AA, B3, X3)}
            tensor_phase = mvt   # matvec phase: the iteration's products and the true residuals, all tensor-core
            # FP64 products on the same operator: rate over a few iterations
            _cg_timed(ctx, AA, B3, X3, "classic", "fp64", 0.0, 1, 0)
            ms64, res64, mv64 = _cg_timed(ctx, AA, B3, X3, "classic", "fp64", 0.0, args.cg3_fp64_iters, 0)
            mv64_ms = mv64[0] / max(mv64[1], 1)
            c3[label]["fp64_products"] = {
                "iterations": args.cg3_fp64_iters, "ms_per_iteration": round(ms64 / args.cg3_fp64_iters, 3),
                "matvec_ms_mean": round(mv64_ms, 3),
                "frac_of_fp64_fma_rate": round(n3 * n3 * 16 / (mv64_ms / 1e3) / (FP64_PEAK_GFLOPS * 1e9 / 2), 4)}
            # the tensor-core product: every launch of the matvec phase (the
            # true residuals' products also keep weight class 7, a few more
            # MMAs on the same digit stream)
            t_ms = tensor_phase[0] / max(tensor_phase[1], 1)
            c3[label]["tensor_products"].update({
                "matvec_ms_mean": round(t_ms, 3),
                "digit_gbs": round(digit_bytes / (t_ms / 1e3) / 1e9, 1),
                "digit_frac_of_hbm": round(digit_bytes / (t_ms / 1e3) / 1e9 / hbm, 4),
                "fp64_matrix_equivalent_gbs": round(n3 * n3 * 8 / (t_ms / 1e3) / 1e9, 1)})
        c3["what"] = (f"n={n3} SE (ell=0.3, sn2=0.1), 16 RHS, classic CG with double-float products to relative "
                      "residual 1e-10 (replacement every 50 iterations, FP64 true residuals); FP32-stored A is the "
                      "FP32 rounding of the FP64 matrix; products_tera_per_s = n^2 * 16 / matvec time; "
                      "tensor_products: the same solve with FP64-accurate tensor-core products (8 base-128 digits "
                      "per entry, 28 digit pairs of weight class <= 6, exact per 512-entry pass; its true residuals keep "
                      "class 7 too), A's digits made once per solve")
        out["config3"] = c3
        del A64, A32, B3, X3
    return out


def serve_run(device, solo, rate, count, nmax):
    """One serving run: `count` requests of the seeded Poisson stream at
    `rate` per second, submitted at their arrival times, all waited for."""
    from paper_2605_13209_b300 import gpchol, inputs
    rs = inputs.request_stream(count=count, rate_per_s=rate, nmin=512, nmax=nmax)
    reqs = []
    for i in range(count):
        nq = int(rs.ns[i])
        reqs.append((inputs.points(nq, 8, int(rs.seeds[i])), inputs.rhs(nq, int(rs.nrhs[i]), int(rs.seeds[i]) + 1),
                     float(rs.ells[i]), float(rs.sn2s[i])))
    srv = gpchol.Server(device, hbm_budget=160 << 30, lanes=4, batch_max_count=32, batch_max_n=2048,
                        solo_prec=solo)
    t0 = time.perf_counter()
    tickets = []
    for i, (Xr, Br, ell, sn2) in enumerate(reqs):
        delay = t0 + float(rs.arrival_s[i]) - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(Xr, Br, 1.0, ell, sn2))
    worst, paths = 0.0, {1: 0, 2: 0, 3: 0}
    for t in tickets:
        _, r = srv.wait(t)
        worst = max(worst, r["backward_error"])
        paths[r["path"]] = paths.get(r["path"], 0) + 1
    st = srv.stats()
    srv.close()
    return {"requests": count, "p50_ms": round(st["p50_ms"], 2), "p99_ms": round(st["p99_ms"], 2),
            "max_ms": round(st["max_ms"], 2), "solves_per_s": round(st["solves_per_s"], 2),
            "completed": st["completed"], "failed": st["failed"], "batches": st["batches"],
            "batched_requests": st["batched_requests"], "solo_requests": paths.get(2, 0) + paths.get(3, 0),
            "peak_reserved_gb": round(st["peak_reserved_bytes"] / 2 ** 30, 2),
            "max_refined_backward_error": worst}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--tile", type=int, default=512)
    ap.add_argument("--prec", default="split_f16", choices=["split_f16", "split_bf16", "bf16"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cg-iters", type=int, default=100)
    ap.add_argument("--cg3-n", type=int, default=65536, help="n of the 16-RHS CG leg (0 = skip)")
    ap.add_argument("--cg3-fp64-iters", type=int, default=5)
    ap.add_argument("--cpu-sample-n", type=int, default=CPU_SAMPLE_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the oracle check of the solutions")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-nmax", type=int, default=16384)
    ap.add_argument("--serve-rates", default="50,100,150,200")
    ap.add_argument("--serve-fp64-requests", type=int, default=40)
    ap.add_argument("--serve-fp64-rates", default="1,3")
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

    def max_over_ranks(v: float) -> float:
        return ranks_max(v, dist, "cuda")

    n, tile = args.n, args.tile
    sysm = inputs.config2(n) if rank == 0 else inputs.gp_system(n, 8, 0.5, 1e-3, nrhs=1, seed=2 + 1000 * rank)
    ctx = gpchol.Context(local)
    pk = peaks()

    # device-resident inputs: A generated once by the A1 kernel
    Xd = torch.from_numpy(sysm.X).cuda()
    A0 = gpchol.se_matrix(Xd, sysm.sf2, sysm.ell, sysm.sn2, ctx=ctx)
    bd = gpchol.as_colmajor(torch.from_numpy(sysm.B[:, 0]).cuda())
    Xs = gpchol.colmajor(n, 1)
    torch.cuda.synchronize()
    flops = n ** 3 / 3.0
    last = {}

    def step():
        last["res"] = gpchol.solve_refined(A0, bd, Xs, prec=args.prec, tile=tile, bwd_tol=1e-12, maxit=500, ctx=ctx)

    # ---------------------------------------------------------- headline
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
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    gpu_launches = ctx.launch_count() - launches0
    names = {"diag": gpchol.PHASE_DIAG, "panel": gpchol.PHASE_PANEL, "mixed_trailing": gpchol.PHASE_MIXED_TRAILING,
             "solve": gpchol.PHASE_SOLVE, "cg_matvec": gpchol.PHASE_CG_MATVEC}
    phase = {k: ctx.timing_read(v) for k, v in names.items()}
    ctx.timing_enable(False)
    value = replica_rate(flops, ms / 1e3, world) / 1e9
    res = last["res"]

    # the timed steps' solution, checked against the oracle after all legs
    x_mixed = Xs[:, 0].cpu().numpy().copy()

    # dominant kernel of the step (syrk_tc_kernel: the largest share of the
    # ncu launch list of this workload) and its roofline
    dom = "mixed_trailing"
    roof = roofline_of(dom, *phase[dom], n, 1, pk)
    if roof is not None:
        work_per_launch = phase[dom][2] / max(phase[dom][1], 1)
        roof = {"kernel": "syrk_tc_kernel", **roof, "launches": phase[dom][1],
                "avg_launch_ms": round(phase[dom][0] / max(phase[dom][1], 1), 4),
                "traffic": (round(SYRK_DRAM_BYTES_PER_FLOP * work_per_launch)
                            if SYRK_DRAM_BYTES_PER_FLOP is not None and args.prec != "bf16" else None),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per flop over all syrk_tc_kernel "
                                  "update launches of one n = 16384 solve, times the average launch's work"}
    phases = {k: {"ms_per_step": round(v[0] / args.steps, 3), "launches_per_step": v[1] / args.steps,
                  "roofline": roofline_of(k, *v, n, 1, pk)} for k, v in phase.items()}

    # ---------------------------------------------------------- FP64 leg
    fp64 = None
    x_fp64 = L_block = x_emu = L_block_emu = None
    if not args.no_fp64:
        Aw = gpchol.colmajor(n, n)
        small = min(n, 2048)
        Aw[:small, :small].copy_(A0[:small, :small])
        gpchol.chol_factor(Aw[:small, :small], tile=tile if tile <= small else 256, ctx=ctx)   # warm kernels
        Aw.copy_(A0)
        torch.cuda.synchronize()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        gpchol.chol_factor(Aw, tile=tile, ctx=ctx)
        Xf = bd.clone()
        gpchol.chol_solve(Aw, Xf, ctx=ctx)
        f1.record()
        torch.cuda.synchronize()
        fms = max_over_ranks(f0.elapsed_time(f1))
        x_fp64 = Xf[:, 0].cpu().numpy().copy()
        nb = min(n, CHECK_BLOCK_N)
        L_block = np.tril(Aw[:nb, :nb].cpu().numpy())
        fp64 = {"ms_per_solve": round(fms, 2), "gflops": round(world * flops / (fms / 1e3) / 1e9, 2),
                "speedup_mixed_vs_fp64": round(fms / ms, 2), "steps": 1,
                "what": f"FP64 blocked Cholesky (tile {tile}) + forward/back substitution"}
        # the same with step 3 on the FP64-accurate tensor-core product
        Aw.copy_(A0)
        torch.cuda.synchronize()
        ctx.timing_enable(True)
        f0.record()
        gpchol.chol_factor(Aw, tile=tile, ctx=ctx, update="fp64_emulated")
        Xe = bd.clone()
        gpchol.chol_solve(Aw, Xe, ctx=ctx)
        f1.record()
        torch.cuda.synchronize()
        tr = ctx.timing_read(gpchol.PHASE_TRAILING)
        ctx.timing_enable(False)
        ems = max_over_ranks(f0.elapsed_time(f1))
        x_emu = Xe[:, 0].cpu().numpy().copy()
        L_block_emu = np.tril(Aw[:nb, :nb].cpu().numpy())
        fp64["emulated_update"] = {
            "ms_per_solve": round(ems, 2), "gflops": round(world * flops / (ems / 1e3) / 1e9, 2),
            "speedup_vs_fp64": round(fms / ems, 2),
            "update_ms": round(tr[0], 2), "update_tflops_fp64_equiv": round(tr[2] / (tr[0] / 1e3) / 1e12, 2),
            "what": "the same factor + solve with step 3 as FP64-accurate products on the bf16 tensor cores "
                    "(8 base-128 digits per entry, 28 digit pairs, exact class sums)"}
        del Aw

    # ---------------------------------------------------------- CG legs
    cg = None
    if args.cg_iters > 0:
        cg = cg_legs(args, ctx, A0, bd, n, world, pk, max_over_ranks, rank)

    # ---------------------------------------------------------- autotuner
    # tile choices of this GPU for the batched legs, the serving lanes and
    # the refined solve's tile 0 (the headline above names its tile)
    import tempfile
    t0 = time.perf_counter()
    tune = gpchol.autotune(os.path.join(tempfile.gettempdir(), "gpchol_tune.json"), nmax=32768, ctx=ctx)
    tune["seconds"] = round(time.perf_counter() - t0, 2)

    # ---------------------------------------------------------- batched leg
    batched = None
    xs_batched = xs_mixed = None
    if args.batch_count > 0:
        spec = inputs.batch_spec(count=args.batch_count, nmin=256, nmax=4096, seed=4)
        Ab, Bb, Bb0, Xp = [], [], [], []
        for k in range(args.batch_count):
            sk = spec.system(k, d=8) if rank == 0 else inputs.gp_system(int(spec.ns[k]), 8, float(spec.ells[k]),
                                                                         float(spec.sn2s[k]), seed=7 + 97 * k + rank)
            Xp.append((torch.from_numpy(sk.X).cuda(), sk.sf2, sk.ell, sk.sn2))
            Ab.append(gpchol.colmajor(sk.n, sk.n))
            Bb0.append(gpchol.as_colmajor(torch.from_numpy(sk.B).cuda()))
            Bb.append(gpchol.colmajor(sk.n, 1))

        def refill():
            for (xd, sf2, ell, sn2), a, b, b0 in zip(Xp, Ab, Bb, Bb0):
                gpchol.se_matrix(xd, sf2, ell, sn2, A=a, ctx=ctx)
                b.copy_(b0)

        bflops = float(sum(int(n) ** 3 for n in spec.ns)) / 3.0
        refill()
        gpchol.batched_solve(Ab, Bb, ctx=ctx)        # first call captures the graph
        times = []
        for _ in range(3):
            refill()
            torch.cuda.synchronize()
            ctx.timing_enable(True)
            gpchol.batched_solve(Ab, Bb, ctx=ctx)
            times.append(ctx.timing_read(gpchol.PHASE_BATCHED)[0])
            ctx.timing_enable(False)
        bms = max_over_ranks(min(times))
        xs_batched = [b[:, 0].cpu().numpy().copy() for b in Bb]
        batched = {"systems": args.batch_count, "n_range": [int(spec.ns.min()), int(spec.ns.max())],
                   "fp64": {"ms_per_batch": round(bms, 2), "gflops": round(world * bflops / (bms / 1e3) / 1e9, 2),
                            "frac_of_fp64_peak": round(bflops / (bms / 1e3) / 1e9 / FP64_PEAK_GFLOPS, 4),
                            "what": "FP64 blocked Cholesky (64-wide blocks) + substitution, one graph launch"}}
        # mixed: FP32 factors with FP64 diagonal leaves, FP64 iterative refinement to 1e-12
        refill()
        Xb = [gpchol.colmajor(b.shape[0], 1) for b in Bb]
        gpchol.batched_solve_mixed(Ab, Bb, Xb, bwd_tol=1e-12, maxit=30, ctx=ctx)   # captures the graphs
        mtimes, mres = [], None
        for _ in range(3):
            for x in Xb:
                x.zero_()
            torch.cuda.synchronize()
            ctx.timing_enable(True)
            mres = gpchol.batched_solve_mixed(Ab, Bb, Xb, bwd_tol=1e-12, maxit=30, ctx=ctx)
            mtimes.append(ctx.timing_read(gpchol.PHASE_BATCHED)[0])
            ctx.timing_enable(False)
        mms = max_over_ranks(min(mtimes))
        xs_mixed = [x[:, 0].cpu().numpy().copy() for x in Xb]
        batched["mixed"] = {"ms_per_batch": round(mms, 2), "gflops_equivalent": round(world * bflops / (mms / 1e3) / 1e9, 2),
                            "speedup_vs_fp64": round(bms / mms, 2), "refinement_iterations_max": mres.iterations,
                            "refinement_steps": mres.steps, "backward_error_lib": mres.backward_error_max,
                            "what": "FP32 factor (64-wide blocks, FP64 diagonal leaves) + FP64 iterative refinement "
                                    "to backward error 1e-12, one graph launch (+ replayed steps if needed)"}
        del Xb
        del Ab, Bb, Bb0, Xp

    # ---------------------------------------------------------- serving leg
    serving = None
    if args.serve_requests > 0 and rank == 0:
        serving = {}
        runs = [("mixed", args.prec, float(r), args.serve_requests) for r in args.serve_rates.split(",") if r]
        runs += [("fp64_only", "fp64", float(r), args.serve_fp64_requests)
                 for r in args.serve_fp64_rates.split(",") if r and args.serve_fp64_requests > 0]
        for label, solo, rate, count in runs:
            serving[f"{label}@{rate:g}/s"] = serve_run(local, solo, rate, count, args.serve_nmax)
        serving["what"] = (f"seeded Poisson streams, n log-uniform [512, {args.serve_nmax}], 1-8 RHS, ell ~ U[0.2, 1], "
                           "sn2 ~ U[1e-3, 1e-1]; 160 GB budget, 4 lanes; n <= 2048 grouped into batched FP64 launches "
                           f"(up to 32 per batch); larger requests solo: mixed = {args.prec} refined to backward error "
                           "1e-12, fp64_only = FP64 factor + solve; latency = completion - submission")

    # ---------------------------------------------------------- e2e
    Xh = torch.from_numpy(sysm.X).pin_memory()
    bh = torch.from_numpy(np.ascontiguousarray(sysm.B[:, 0])).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    Ae = A0   # the device buffer the SE matrix is regenerated into

    def e2e_step():
        Xdev = Xh.cuda(non_blocking=True)
        gpchol.se_matrix(Xdev, sysm.sf2, sysm.ell, sysm.sn2, A=Ae, ctx=ctx)
        bdev = gpchol.colmajor(n, 1)
        bdev[:, 0].copy_(bh, non_blocking=True)
        gpchol.solve_refined(Ae, bdev, Xs, prec=args.prec, tile=tile, bwd_tol=1e-12, maxit=500, ctx=ctx)
        xh.copy_(Xs[:, 0], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_s = float("nan")
    if args.e2e_steps > 0:
        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    check = oracle_check(sysm, x_mixed, x_fp64, L_block, x_emu, L_block_emu) if not args.no_check else None
    if batched is not None and xs_batched is not None and not args.no_check:
        batched["fp64"]["backward_error_max"] = batched_check(args.batch_count, xs_batched)
        batched["mixed"]["backward_error_max"] = batched_check(args.batch_count, xs_mixed)
        batched["backward_error_by"] = "oracle on every system (host, long-double residual)"
    if fp64 is not None and check is not None:
        fp64["backward_error"] = check["backward_error_fp64"]
    cpu = None if args.no_cpu_baseline else cpu_baseline(args.cpu_sample_n)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{args.prec}+f64_refine", "data": "synthetic",
        "config": {"workload": f"n={n} SE GP system (d=8, ell=0.5, sn2=1e-3), one RHS, A device-resident: "
                               f"{args.prec} mixed-precision Cholesky (tile {tile}) + FP64 PCG refinement to "
                               f"backward error 1e-12; value = n^3/3 per solve time",
                   "n": n, "tile": tile, "nrhs": 1, "prec": args.prec,
                   "l2": "inputs larger than L2 (8.6 GB FP64 matrix, 4.3 GB FP32 factor)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": round(world * flops / e2e_s / 1e9, 2) if e2e_s == e2e_s else None, "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(Xh.numel() * 8 + bh.numel() * 8),
                "d2h_bytes_per_step": int(xh.numel() * 8),
                "seconds_per_step": round(e2e_s, 4),
                "api": "gpchol.se_matrix + solve_refined from pinned host points X and b; x back to pinned host"},
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "refine": {"iterations": res.iterations, "factor_attempts": res.factor_attempts, "shift": res.shift,
                   "backward_error_lib": res.backward_error_max},
        "fp64": fp64,
        "cg": cg,
        "autotune": tune,
        "batched": batched,
        "serving": serving,
        "phases": phases,
        "check": check,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
