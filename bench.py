"""Benchmark: batched projection + inversion on the 4,096-curve workload.

One step = one pass of the query hot path over one batch: 1M projection and
1M inversion queries on 4,096 random curves (degree 2-7, 8-64 control points,
clamped non-uniform knots), decomposed into cubic Beziers at 1e-10 x diag.
Decomposition is preprocessing: timed once and reported separately.

Prints one JSON line (rank 0).  --impl reference times the CPU FP64 oracle on
the host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "projected pts/s, learned+mixed vs plain FP64, same GB300, at 1e-9 rel. dist"
TOL = 1e-10
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=0, help="grid samples per segment; 0 = autotune")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--curves", type=int, default=4096, help="curves in the workload")
    ap.add_argument("--queries", type=int, default=1_000_000, help="projection and inversion queries each")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- workload

def build_workload(seed, rank, n_curves=4096, n_queries=1_000_000):
    from paper_2504_11498_gb300 import synth
    cs, qs = synth.curve_set(seed=seed + 1000 * rank, n_curves=n_curves, n_proj=n_queries, n_inv=n_queries)
    return cs, qs


def cpu_oracle_rate(cs, qs, budget_s=12.0, max_q=40000):
    """Oracle (plain FP64, as it stands) on the host cores, bounded sample:
    equal numbers of projection and inversion queries."""
    from oracle import oracle as O
    n = 500
    elapsed, done = 0.0, 0
    threads = O.num_threads()
    C, _, _ = O.eval_curves(cs, qs.inv_curve[:max_q], qs.inv_t[:max_q])
    while elapsed < budget_s and done < max_q:
        k = min(n, max_q - done)
        t0 = time.perf_counter()
        O.project_curves(cs, qs.proj_curve[done:done + k], qs.proj_xyz[done:done + k], nthreads=threads)
        O.project_curves(cs, qs.inv_curve[done:done + k], C[done:done + k], nthreads=threads)
        elapsed += time.perf_counter() - t0
        done += k
        n = min(n * 2, 8000)
    return 2 * done / elapsed, threads, 2 * done, elapsed


# ------------------------------------------------------------------- main

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        cs, qs = build_workload(args.seed, 0, args.curves, args.queries)
        rates = []
        for _ in range(args.warmup):
            cpu_oracle_rate(cs, qs, budget_s=2.0, max_q=2000)
        t_all = 0.0
        for _ in range(args.steps):
            r, cores, nq, el = cpu_oracle_rate(cs, qs, budget_s=8.0, max_q=20000)
            rates.append(r)
            t_all += el
        v = float(np.median(rates))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pts/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": "curve_set_4096: 1M projection + 1M inversion queries",
                                                "tol_rel": TOL},
                "cpu_baseline": {"value": v, "unit": "pts/s", "cores": cores, "kind": "oracle",
                                 "sample": f"{nq} queries per step (half projection, half inversion)"},
                "e2e": {"value": v, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as dist
    from paper_2504_11498_gb300 import autotune, bspl, build

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cs, qs = build_workload(args.seed, rank, args.curves, args.queries)
    dc = bspl.DeviceCurves(cs, dev)

    # decomposition (preprocessing, timed separately)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    segs = bspl.decompose(dc, TOL)
    torch.cuda.synchronize()
    decomp_ms = 1e3 * (time.perf_counter() - t0)

    pc = torch.as_tensor(qs.proj_curve, device=dev)
    pq = torch.as_tensor(qs.proj_xyz, device=dev)
    ic = torch.as_tensor(qs.inv_curve, device=dev)
    iq = bspl.bspl_eval_curves(dc, ic, torch.as_tensor(qs.inv_t, device=dev))
    n_step = pc.numel() + ic.numel()
    bufs_p = bspl.QueryBuffers(segs, pc.numel(), dev)
    bufs_i = bspl.QueryBuffers(segs, ic.numel(), dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # launch configuration per precision, chosen by the autotuner (untimed)
    cfg = {p: (autotune.tune_curves(segs, pc, pq, p) if args.samples == 0 else dict(samples=args.samples))
           for p in (bspl.MIXED, bspl.FP64)}

    def step(prec, counters=None):
        o = bspl.make_options(prec=prec, counters=counters, **cfg[prec])
        bspl.bspl_project_curves(segs, pc, pq, o, bufs_p)
        bspl.bspl_invert_curves(segs, ic, iq, o, bufs_i)

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            a.record(stream)
            step(prec)
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return float(np.mean(ms)), ms

    # algorithmic work from the device counters (one extra, untimed pass)
    def counted(prec):
        cnt = torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=dev)
        step(prec, cnt)
        torch.cuda.synchronize()
        return dict(zip(bspl.COUNTER_NAMES, cnt.cpu().tolist()))

    # the query kernel alone: inputs pre-grouped by curve on the host, no
    # sorting inside the call, events around each kernel launch
    op = np.argsort(qs.proj_curve, kind="stable")
    oi = np.argsort(qs.inv_curve, kind="stable")
    spc, spq = pc[torch.as_tensor(op, device=dev)], pq[torch.as_tensor(op, device=dev)]
    sic, siq = ic[torch.as_tensor(oi, device=dev)], iq[torch.as_tensor(oi, device=dev)]

    def kernel_ms(prec, steps):
        o = bspl.make_options(prec=prec, sort_queries=0, **cfg[prec])
        for _ in range(2):
            bspl.bspl_project_curves(segs, spc, spq, o, bufs_p)
            bspl.bspl_invert_curves(segs, sic, siq, o, bufs_i)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            bspl.bspl_project_curves(segs, spc, spq, o, bufs_p)
            ev[1].record(stream)
            flush.fill_(1.0)
            ev[2].record(stream)
            bspl.bspl_invert_curves(segs, sic, siq, o, bufs_i)
            ev[3].record(stream)
            torch.cuda.synchronize()
            tot += ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])
        return tot / steps  # both launches of one step

    # clocks are sampled across the timed loops (mixed, then plain)
    clocks = ClockSampler(local)
    clocks.start()
    ms_mixed, ms_list = timed(bspl.MIXED, args.steps, args.warmup)
    ms_plain, _ = timed(bspl.FP64, max(2, args.steps // 3), 2)
    clk = clocks.stop()
    c_mixed = counted(bspl.MIXED)
    c_plain = counted(bspl.FP64)
    kms_mixed = kernel_ms(bspl.MIXED, max(3, args.steps // 2))
    kms_plain = kernel_ms(bspl.FP64, 2)

    # end to end through the public API with host buffers (pinned)
    h_pc = pc.cpu().pin_memory()
    h_pq = pq.cpu().pin_memory()
    h_ic = ic.cpu().pin_memory()
    h_iq = iq.cpu().pin_memory()
    h_out = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in
             (bufs_p.param, bufs_p.dist, bufs_p.status, bufs_i.param, bufs_i.dist, bufs_i.status)]
    d_in = [torch.empty_like(x, device=dev) for x in (h_pc, h_pq, h_ic, h_iq)]

    def e2e_step():
        for d, h in zip(d_in, (h_pc, h_pq, h_ic, h_iq)):
            d.copy_(h, non_blocking=True)
        o = bspl.make_options(prec=bspl.MIXED, **cfg[bspl.MIXED])
        bspl.bspl_project_curves(segs, d_in[0], d_in[1], o, bufs_p)
        bspl.bspl_invert_curves(segs, d_in[2], d_in[3], o, bufs_i)
        for h, d in zip(h_out, (bufs_p.param, bufs_p.dist, bufs_p.status, bufs_i.param, bufs_i.dist,
                                bufs_i.status)):
            h.copy_(d, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    k_e2e = max(3, args.steps // 2)
    for _ in range(k_e2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / k_e2e
    h2d = sum(x.numel() * x.element_size() for x in (h_pc, h_pq, h_ic, h_iq))
    d2h = sum(x.numel() * x.element_size() for x in h_out)

    # max over ranks
    vals = torch.tensor([ms_mixed, ms_plain, ms_e2e], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    ms_mixed, ms_plain, ms_e2e = vals.tolist()
    total_q = n_step * world
    value = total_q / (ms_mixed * 1e-3)

    # roofline of the query kernels: FP32 + FP64 arithmetic against measured
    # FMA-chain peaks (FP32-equivalent TFLOP/s)
    p32 = bspl.measure_fma_peak(False)
    p64 = bspl.measure_fma_peak(True)
    S = cfg[bspl.MIXED]["samples"]

    def flops(c, mixed):
        # per-unit figures: 12 flops per box test, 15 per grid sample, 45 per
        # Newton iteration; units counted by the kernel
        cull = 12 * (c["grp_tested"] + c["seg_tested"])
        grid = 15 * S * c["candidates"]
        if mixed:
            return cull + grid + 45 * c["newton32_iters"], 45 * c["newton64_iters"]
        return 0, cull + grid + 45 * c["newton64_iters"]

    f32m, f64m = flops(c_mixed, True)
    S = cfg[bspl.FP64]["samples"]
    f32p, f64p = flops(c_plain, False)
    S = cfg[bspl.MIXED]["samples"]
    t_m, t_p = kms_mixed * 1e-3, kms_plain * 1e-3
    eq_m = (f32m + f64m * p32 / p64) / t_m
    eq_p = (f32p + f64p * p32 / p64) / t_p
    roofline = {"bound": "alu", "achieved": eq_m / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                "frac": eq_m / p32, "traffic": None,
                "note": "query kernel (k_query_curves, 2 launches per step); FP32-equivalent rate "
                        "(FP32 flops + FP64 flops x P32/P64) / kernel time; peaks measured by an FMA-chain "
                        "microbenchmark on this GPU (MEASURED_PEAKS.json has no FP32/FP64 ALU peak)",
                "kernel_ms_per_step": kms_mixed, "flops_fp32": f32m, "flops_fp64": f64m,
                "fp32_peak_tflops": p32 / 1e12, "fp64_peak_tflops": p64 / 1e12,
                "plain_fp64": {"achieved_fp64_tflops": f64p / t_p / 1e12, "frac": eq_p / p32}}

    out = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64 (mixed: FP32 search, FP64 finish)", "data": "synthetic",
           "config": {"workload": f"curve_set_{args.curves}: {args.queries} projection + {args.queries} inversion "
                                  "queries per GPU",
                      "tol_rel": TOL, "launch": {"mixed": cfg[bspl.MIXED], "fp64": cfg[bspl.FP64]},
                      "prec": "mixed", "l2": "512 MB flush between timed steps",
                      "segments": int(segs.total), "decompose_ms": decomp_ms},
           "plain_fp64": {"value": total_q / t_p, "ms_per_step": ms_plain},
           "speedup_mixed_vs_plain": ms_plain / ms_mixed,
           "e2e": {"value": total_q / (ms_e2e * 1e-3), "unit": "pts/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": 12, "roofline": roofline, "clocks": clk,
           "counters_mixed": c_mixed}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, nq, el = cpu_oracle_rate(cs, qs)
        out["cpu_baseline"] = {"value": r, "unit": "pts/s", "cores": cores, "kind": "oracle",
                               "sample": f"{nq} queries of the same workload (half projection, half inversion), "
                                         f"{el:.1f} s"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
