#!/usr/bin/env python
"""Benchmark of the DGDFT hot path on one GB300 (or N replicas under torchrun).

A step is one pass of the whole hot path over the 1024-element graphene-like
sheet (32 x 32 elements of 16x16x48 points, extended elements 32x32x48, 4096
atoms, 80-vector filter block, 72 eigenpairs, 64 ALBs): mixed-precision ALB
generation for every element followed by the interior-penalty DG assembly
(element + 4 face neighbours).  value = elements / step time.

The JSON line also carries: the roofline of the Chebyshev filter step (timed
live with CUDA events on its stream), the end-to-end number through the C-ABI
with host buffers, the FP64 GPU path on a sample of elements, the oracle timed
on the host cores (a baseline, not the target), SM clocks sampled during the
timed region and the number of kernel launches.

`--impl reference` times the oracle (the plain FP64 CPU restatement) instead.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ALB elements/sec, mixed vs FP64 at <=1e-6 Ha eigen error; % of roofline"
UNIT = "elements/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--degree", type=int, default=80)
    ap.add_argument("--max-iter", type=int, default=60)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--fp64-elements", type=int, default=16, help="elements in the FP64 GPU sample (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--elements", type=int, default=0, help="use only the first n elements (smoke runs)")
    ap.add_argument("--only-filter", action="store_true",
                    help="time only the FP32 Chebyshev filter (degree --degree) on random blocks (profiling)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None
        self.out = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(self.out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1])); mx.append(float(row[2])); pw.append(float(row[3]))
            except ValueError:
                continue
            for n, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


# -------------------------------------------------------------- oracle arm --
def _oracle_sample(args_tuple):
    """Time the oracle's own steps on one element: one H application on the filter block and one
    CholQR2 + Rayleigh-Ritz (the per-iteration work besides the filter)."""
    from oracle import local_operator as lo, chefsi as cf
    prob, params, k = args_tuple
    t0 = time.perf_counter()
    op = lo.LocalOperator(prob, k)
    X = cf.random_block(params.seed, k, int(params.n_blk[k]), op.N)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    Y = op.apply(X)
    t_h = time.perf_counter() - t0
    t0 = time.perf_counter()
    Q = cf.cholqr2(Y, op.dV)
    cf.rayleigh_ritz(op, Q)
    t_sub = time.perf_counter() - t0
    return t_setup, t_h, t_sub


def oracle_sample(wl, cores, iters_full, degree):
    """Oracle elements/s on the host cores, from timed oracle steps scaled to a full solve.

    Each of `cores` processes (one BLAS/FFT thread each) times, on its own element, one H
    application on the filter block (t_h) and one CholQR2 + Rayleigh-Ritz (t_sub, which contains
    one more H application).  A full solve is estimated as set-up + Lanczos (10 single-vector H
    applications) + start-up CholQR2/RR + iters_full x ((degree - 1) t_h + t_sub) + ALB truncation
    (neglected)."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"     # inherited by the spawned workers
    elems = list(range(min(cores, wl.problem.n_elem)))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(len(elems)) as pool:
        out = pool.map(_oracle_sample, [(wl.problem, wl.params, k) for k in elems])
    wall = time.perf_counter() - t0
    t_setup = statistics.mean(o[0] for o in out)
    t_h = statistics.mean(o[1] for o in out)
    t_sub = statistics.mean(o[2] for o in out)
    nb = float(wl.params.n_blk[0])
    t_full = t_setup + 10 * t_h / nb + t_sub + iters_full * ((degree - 1) * t_h + t_sub)
    value = len(elems) / t_full
    desc = (f"{len(elems)} elements in parallel (one process per core, 1 BLAS/FFT thread): oracle H x on the "
            f"{int(nb)}-vector block {t_h:.2f} s, CholQR2 + Rayleigh-Ritz {t_sub:.2f} s, set-up {t_setup:.2f} s; "
            f"full solve estimated as set-up + Lanczos + {iters_full} x ({degree - 1} H x + CholQR2/RR) = "
            f"{t_full:.0f} s per element per core; sample wall {wall:.1f} s")
    return value, desc, len(elems)


def run_reference(args, wl):
    cores = os.cpu_count() or 1
    iters_full = 9   # FP64 CheFSI passes of a 32x32x48 element at degree 80 to tol 1e-8 (GPU FP64 path, same algorithm)
    vals = []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc, used = oracle_sample(wl, cores, iters_full, args.degree)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wl.problem.n_elem / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args, wl):
    p, q = wl.problem, wl.params
    return {"workload": wl.name, "elements": int(p.n_elem), "atoms": int(p.n_atoms),
            "q_grid": "x".join(str(int(v)) for v in p.elem_Qn[0]),
            "e_grid": "x".join(str(int(v)) for v in p.elem_En[0]),
            "n_blk": int(q.n_blk[0]), "n_eig": int(q.n_eig[0]), "n_alb": int(q.n_alb[0]),
            "cheb_degree": args.degree, "tol": args.tol, "stencil": int(p.n_stencil), "alpha": wl.alpha,
            "precision": "mixed (FP32 filter/subspace, FP64 small solves + final FP64 Rayleigh-Ritz)",
            "l2": "working set >> L2 (blocks 16 GB per FP32 buffer): no flush needed"}


# ------------------------------------------------------------ multi-rank --
def max_over_ranks(ms, dist, device):
    """Slowest rank's step time (weak scaling: every rank runs its own replica of the workload)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, n_elem, ms):
    """Elements/s over all ranks: every rank solves n_elem elements in ms milliseconds at most."""
    return world * n_elem / (ms / 1000.0)


# -------------------------------------------------------------- native arm --
def run_native(args, wl, rank, world, local_rank):
    import torch
    from paper_2003_00407_gb300 import api, _abi
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ctx = api.Context(local_rank)
    p, q = wl.problem, wl.params
    M = p.n_elem
    stream = torch.cuda.current_stream()
    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step(host=False):
        res = api.alb_generate(ctx, p, q, precision=_abi.MIXED, cheb_degree=args.degree, tol=args.tol,
                               max_iter=args.max_iter, keep_eigvec=False, host_buffers=host)
        blocks = api.dg_assemble_host(ctx, p, q, res, wl.alpha) if host else api.dg_assemble(ctx, p, q, res,
                                                                                              wl.alpha)
        return res, blocks

    for _ in range(args.warmup):
        res, blocks = step()

    # ---- timed region ----
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0] or 0) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local_rank
    launches0 = ctx.lib.dgdft_kernel_launches()
    barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mid = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(gpu_index) as clk:
        start.record(stream)
        for i in range(args.steps):
            res = api.alb_generate(ctx, p, q, precision=_abi.MIXED, cheb_degree=args.degree, tol=args.tol,
                                   max_iter=args.max_iter, keep_eigvec=False)
            mid[i].record(stream)
            blocks = api.dg_assemble(ctx, p, q, res, wl.alpha)
            ends[i].record(stream)
        stop.record(stream)
        barrier()
    launches = ctx.lib.dgdft_kernel_launches() - launches0
    ms = max_over_ranks(start.elapsed_time(stop) / args.steps, dist, dev)
    t_alb = statistics.mean((start if i == 0 else ends[i - 1]).elapsed_time(mid[i]) for i in range(args.steps))
    t_dg = statistics.mean(mid[i].elapsed_time(ends[i]) for i in range(args.steps))
    iters = res.iters.cpu().numpy()
    status = res.status.cpu().numpy()
    value = whole_job_value(world, M, ms)

    # ---- roofline of the Chebyshev step (FP32 filter), timed live on this stream ----
    roof = filter_roofline(ctx, api, _abi, wl, torch, stream, res)

    # ---- end to end through the C-ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        barrier()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            resh, blocksh = step(host=True)
        barrier()
        t_e2e = (time.perf_counter() - t0) / max(1, args.steps)
        L = resh.L
        n_alb_pts = int(np.sum(q.n_alb * np.prod(p.elem_En, axis=1)))
        h2d = 8 * p.v_extra.size * 2 + 8 * M * L * L
        d2h = 8 * (3 * M * L + M * L * L + n_alb_pts) + 8 * M + 8 * M * p.n_stencil * L * L
        e2e = {"value": world * M / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- FP64 GPU path on a sample of elements ----
    fp64 = None
    if args.fp64_elements > 0:
        from workloads.configs import subset
        ns = min(args.fp64_elements, M)
        ws = subset(wl, range(ns))
        ws.problem.n_stencil = 1
        ws.problem.neighbors = np.arange(ns, dtype=np.int32)[:, None].copy()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r64 = api.alb_generate(ctx, ws.problem, ws.params, precision=_abi.FP64, cheb_degree=args.degree,
                               tol=args.tol, max_iter=args.max_iter, keep_eigvec=False)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = f0.elapsed_time(f1) / 1000.0
        t_dg_elem = t_dg / 1000.0 / M
        ev64 = r64.eigval.cpu().numpy()
        ev32 = res.eigval.cpu().numpy()
        n_eig = int(q.n_eig[0])
        diff = float(np.abs(ev64[:ns, :n_eig] - ev32[:ns, :n_eig]).max())
        fp64 = {"value": ns / (t64 + t_dg_elem * ns), "unit": UNIT,
                "sample": f"first {ns} elements, FP64 ALB generation timed + DG assembly time per element "
                          f"of the mixed run (the DG assembly is FP64 in both paths)",
                "alb_ms": 1000 * t64, "iterations_mean": float(np.mean(r64.iters.cpu().numpy())),
                "mixed_vs_fp64_max_eig_diff_ha": diff}
        # per filter pass and element: separates per-iteration speed from convergence
        fp64["ms_per_pass_per_element"] = 1000 * t64 / max(fp64["iterations_mean"], 1e-9) / ns

    out = None
    if rank == 0:
        cpu = None
        if not args.no_cpu and world == 1:   # the oracle baseline is timed at N = 1 only
            iters_full = int(round(fp64["iterations_mean"])) if fp64 else 9
            v, desc, used = oracle_sample(wl, os.cpu_count() or 1, iters_full, args.degree)
            cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc}
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config_dict(args, wl),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
               "clocks": clk.summary(), "fp64_gpu": fp64,
               "phase_ms": {"alb_generate": t_alb, "dg_assemble": t_dg},
               "iterations": {"mean": float(iters.mean()), "max": int(iters.max()),
                              "ms_per_pass_per_element": t_alb / max(float(iters.mean()), 1e-9) / M},
               "status_nonzero": int(np.count_nonzero(status))}
    ctx.close()
    return out


def filter_roofline(ctx, api, _abi, wl, torch, stream, res):
    """Per-degree time of the FP32 Chebyshev step over all elements and vectors, vs HBM bytes."""
    import copy
    p, q = wl.problem, wl.params
    M = p.n_elem
    N = np.prod(p.elem_Qn, axis=1).astype(np.int64)
    nb = q.n_blk.astype(np.int64)
    total = int(np.sum(nb * N))
    X = torch.randn(total, dtype=torch.float32, device="cuda")
    ev = res.eigval.cpu().numpy()
    bounds = np.stack([ev[:, 0], ev[:, int(nb[0]) - 1], np.full(M, 95.0)], axis=1)
    times = {}
    for m in (6, 16):
        api.chebyshev_filter(ctx, p, q, X, bounds, m, precision=_abi.MIXED)  # warm
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        api.chebyshev_filter(ctx, p, q, X, bounds, m, precision=_abi.MIXED)
        b.record(stream)
        torch.cuda.synchronize()
        times[m] = a.elapsed_time(b) / 1000.0
    t_step = (times[16] - times[6]) / 10.0
    # algorithmic bytes of one step: read Y_k, read Y_{k-1}, write Y_{k+1} (FP32) + V_eff once per element
    bytes_step = float(np.sum(12 * N * nb + 4 * N))
    peak = measured_peak()
    ach = bytes_step / t_step / 1e9
    del X
    # DRAM bytes of one full launch: dram__bytes_read.sum + dram__bytes_write.sum of the ncu capture in
    # profiles/k_cheb_fused_16elem_full.md (16 elements), scaled by the vectors processed (x 64); only for
    # the 1024-element sheet, which that capture samples
    traffic = 738.0e6 * (M / 16.0) if M == 1024 and int(np.max(N)) == 49152 else None
    return {"bound": "hbm", "achieved": ach, "peak": peak[0], "unit": "GB/s", "frac": ach / peak[0],
            "traffic": traffic, "kernel": "k_cheb_fused (one FP32 Chebyshev step over all vectors; one launch)",
            "step_ms": 1000 * t_step, "bytes_per_step": bytes_step, "peak_source": peak[1]}


def run_filter_only(args, wl):
    import torch
    from paper_2003_00407_gb300 import api, _abi
    ctx = api.Context(0)
    p, q = wl.problem, wl.params
    N = np.prod(p.elem_Qn, axis=1).astype(np.int64)
    nb = q.n_blk.astype(np.int64)
    X = torch.randn(int(np.sum(nb * N)), dtype=torch.float32, device="cuda")
    bounds = np.tile([-0.5, 1.0, 95.0], (p.n_elem, 1))
    stream = torch.cuda.current_stream()
    ts = []
    for i in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        api.chebyshev_filter(ctx, p, q, X, bounds, args.degree, precision=_abi.MIXED)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    by = float(np.sum(12 * N * nb + 4 * N)) * args.degree
    print(json.dumps({"mode": "filter-only", "elements": int(p.n_elem), "degree": args.degree, "ms": ms,
                      "GBps_algorithmic": by / ms / 1e6}), flush=True)
    ctx.close()


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    from workloads import make_config
    from workloads.configs import subset
    wl = make_config(args.config)
    if args.elements:
        wl = subset(wl, range(args.elements))
        wl.problem.n_stencil = 1
        wl.problem.neighbors = np.arange(args.elements, dtype=np.int32)[:, None].copy()
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return
    if args.only_filter:
        run_filter_only(args, wl)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_native(args, wl, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
