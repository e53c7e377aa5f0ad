"""Benchmark: batched point projection / inversion on B-spline curves and
surfaces (learned seed + FP32/BF16 bulk + FP64 finish vs plain FP64).

Default (--workload c4): one step = 16M projection queries on the 4,096-curve
set (degree 2-7, 8-64 control points, clamped non-uniform knots) decomposed
into cubic Beziers at 1e-10 x diag, through the learned-seed path; the 1M
projection + 1M inversion batch on the same curves (c2) is measured in the
same run and reported beside it.  --workload c3 / c5: the 1,024-surface set
and the ragged curve + surface batch.  Decomposition and the seed network's
training are preprocessing: timed once and reported separately.

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
SURF_TOL = 1e-4  # surfaces: decomposed at the paper's alpha, last Newton steps on the original patch
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) of one k_cull_cands launch on the 16M-query
# workload, from the ncu capture summarised in
# profiles/k_cull_cands_dram_curve_set_4096_16M.md
CULL_TRAFFIC_PER_LAUNCH = 1_545_019_136 + 1_797_668_352


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
    ap.add_argument("--workload", default="c4", choices=["c2", "c4", "c3", "c5", "p", "nurbs"],
                    help="c4 (default): 16M projection queries on the 4,096-curve set (learned seed), with the "
                         "c2 batch measured beside it; c2: 1M projection + 1M inversion queries; "
                         "c3: 1,024 surfaces, 4M + 4M queries; c5: 65,536 cubic curves + 8,192 bicubic "
                         "surfaces, 64M Zipf-skewed queries; p: the paper-shaped 18-curve suite; nurbs: 4,096 "
                         "rational curves, 1M projection + 1M inversion queries, refined on the original curves")
    ap.add_argument("--surfaces", type=int, default=1024, help="c3: surfaces in the workload")
    ap.add_argument("--surface-queries", type=int, default=4_000_000,
                    help="c3: projection and inversion queries each")
    ap.add_argument("--train-curves", type=int, default=2048, help="curves of the seed network's training set")
    ap.add_argument("--train-queries", type=int, default=3_500_000, help="their projection and inversion queries")
    ap.add_argument("--train-pairs", type=int, default=10_000_000, help="training pairs at most")
    ap.add_argument("--train-epochs", type=int, default=3)
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
            # the timed region starts once nvidia-smi is sampling (its start-up
            # holds the driver for a moment)
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
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

def build_workload(seed, rank, n_curves=4096, n_queries=1_000_000, n_inv=None):
    from paper_2504_11498_gb300 import synth
    cs, qs = synth.curve_set(seed=seed + 1000 * rank, n_curves=n_curves, n_proj=n_queries,
                             n_inv=n_queries if n_inv is None else n_inv)
    return cs, qs


def cpu_oracle_rate(cs, qs, budget_s=15.0, max_q=1_000_000, threads=0):
    """Oracle (plain FP64, as it stands) on the host cores (all of them, or
    `threads`), bounded sample of the workload: its projection queries and,
    when it has them, as many inversion queries."""
    from oracle import oracle as O
    n = 500 if threads != 1 else 50
    elapsed, done = 0.0, 0
    threads = threads or O.num_threads()
    inv = len(qs.inv_curve) > 0
    max_q = min(max_q, len(qs.proj_curve))
    if inv:
        max_q = min(max_q, len(qs.inv_curve))
        C, _, _ = O.eval_curves(cs, qs.inv_curve[:max_q], qs.inv_t[:max_q])
    while elapsed < budget_s and done < max_q:
        k = min(n, max_q - done)
        t0 = time.perf_counter()
        O.project_curves(cs, qs.proj_curve[done:done + k], qs.proj_xyz[done:done + k], nthreads=threads)
        if inv:
            O.project_curves(cs, qs.inv_curve[done:done + k], C[done:done + k], nthreads=threads)
        elapsed += time.perf_counter() - t0
        done += k
        n = min(n * 2, 8000)
    per = 2 if inv else 1
    return per * done / elapsed, threads, per * done, elapsed


def combine_over_ranks(times_ms, n_per_rank, world, dist=None, device="cpu"):
    """Weak scaling over independent replicas: each time is the maximum
    over ranks (the slowest replica bounds the job), the units processed are
    the per-rank units times the number of ranks."""
    import torch
    vals = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    return vals.tolist(), n_per_rank * world


# ------------------------------------------------------------ learned seed

def train_seed(args, rank, dev, rational=False):
    """Trains the seed network on (segment, query, t*) pairs of a second
    curve set of the same recipe (seed 12; rational=True: the NURBS recipe):
    pairs from the learned path's own culling, labels from the FP64 solver,
    hand-written training kernels.  Returns the network and a summary
    (untimed preprocessing)."""
    import torch
    from paper_2504_11498_gb300 import bspl, synth
    t0 = time.perf_counter()
    make = synth.nurbs_curve_set if rational else synth.curve_set
    cs, qs = make(seed=12 + 1000 * rank, n_curves=args.train_curves, n_proj=args.train_queries,
                  n_inv=args.train_queries)
    dc = bspl.DeviceCurves(cs, dev)
    segs = bspl.decompose(dc, TOL)
    inv = bspl.bspl_eval_curves(dc, torch.as_tensor(qs.inv_curve, device=dev),
                                torch.as_tensor(qs.inv_t, device=dev))
    qc = torch.cat([torch.as_tensor(qs.proj_curve, device=dev), torch.as_tensor(qs.inv_curve, device=dev)])
    q = torch.cat([torch.as_tensor(qs.proj_xyz, device=dev), inv])
    pq, ps, found = bspl.bspl_mlp_collect_pairs(segs, qc, q, cap=args.train_pairs)
    written = pq.numel()
    X = bspl.bspl_mlp_features(segs, pq, ps, q)
    y = bspl.bspl_mlp_labels(segs, pq, ps, q)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    mlp = bspl.Mlp(synth.mlp_init(7), dev)
    loss = mlp.train(X, y, epochs=args.train_epochs, batch=8192, lr=2e-3, seed=5).cpu().numpy()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    if bspl.mlp_check() != bspl.OK:
        raise SystemExit("a tensor-core wait timed out during training")
    del X, y, pq, ps, q, qc, inv, segs, dc
    return mlp, {"pairs": int(written), "pairs_found": int(found), "epochs": args.train_epochs, "batch": 8192,
                 "curves": args.train_curves, "data_ms": 1e3 * (t1 - t0), "train_ms": 1e3 * (t2 - t1),
                 "loss_first_epoch": float(loss[0]), "loss_last_epoch": float(loss[-1])}


def train_surface_seed(kind, rank, dev, n_queries=600_000, max_pairs=6_000_000, epochs=3):
    """Trains the surface seed network on (query, patch) pairs of a second
    surface set of the workload's recipe (c3: the random surfaces, seed 13;
    c5: the ragged batch's bicubic surfaces, seed 15): pairs from the learned
    surface path's own culling, labels = the pair's bicubic minimiser,
    hand-written training kernels.  Untimed preprocessing."""
    import torch
    from paper_2504_11498_gb300 import bspl, synth
    t0 = time.perf_counter()
    if kind == "c3":
        ss, sq = synth.surface_set(seed=13 + 1000 * rank, n_surf=256, n_proj=n_queries, n_inv=1)
    else:
        cs_, ss, qc_, qs_, rng_ = synth.ragged_mix(seed=15 + 1000 * rank, n_curves=16, n_surf=2048,
                                                   n_queries=2 * n_queries)
        _, sq = synth.ragged_queries(cs_, ss, qc_, qs_, rng_)
    dsf = bspl.DeviceSurfaces(ss, dev)
    segs = bspl.decompose(dsf, SURF_TOL)
    ps = torch.as_tensor(sq.proj_surf, device=dev)
    q = bspl.bspl_eval_surfaces(dsf, ps, torch.as_tensor(sq.proj_uv, device=dev)) + \
        torch.as_tensor(sq.proj_dir, device=dev) * torch.as_tensor(sq.proj_r, device=dev)[:, None]
    pq, pp, found = bspl.bspl_smlp_collect_pairs(segs, ps, q, cap=max_pairs)
    X = bspl.bspl_smlp_features(segs, pq, pp, q)
    y = bspl.bspl_smlp_labels(segs, pq, pp, q)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    n = X.shape[0]
    ntr = int(0.9 * n)
    mlp = bspl.Mlp(synth.smlp_init(8), dev, kind=bspl.MLP_SURFACE)
    loss = mlp.train(X[:ntr].contiguous(), y[:ntr].contiguous(), epochs=epochs, batch=8192, lr=2e-3,
                     seed=5).cpu().numpy()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    held = (mlp.forward(X[ntr:].contiguous()) - y[ntr:]).abs().mean().item()
    centre = (0.5 - y[ntr:]).abs().mean().item()
    if bspl.mlp_check() != bspl.OK:
        raise SystemExit("a tensor-core wait timed out during training")
    return mlp, {"pairs": int(n), "pairs_found": int(found), "epochs": epochs, "batch": 8192,
                 "surfaces": int(ss.n), "data_ms": 1e3 * (t1 - t0), "train_ms": 1e3 * (t2 - t1),
                 "loss_first_epoch": float(loss[0]), "loss_last_epoch": float(loss[-1]),
                 "heldout_seed_abs_err": held, "heldout_patch_centre_abs_err": centre}


# ------------------------------------------------------------------- main

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.workload in ("c3", "c5"):
        return run_surface_workloads(args, rank, world, local)
    if args.workload == "p":
        return run_paper_suite(args, rank, world, local)
    if args.workload == "nurbs":
        return run_nurbs(args, rank, world, local)
    # c4 (default): 16M projection queries on the 4,096-curve set, the
    # learned-seed configuration, with the c2 batch (1M + 1M) measured beside
    # it; c2: the 1M + 1M batch alone
    n_proj = 16_000_000 if args.workload == "c4" else args.queries
    n_inv = 0 if args.workload == "c4" else args.queries
    label = {"c4": f"curve_set_{args.curves}: {n_proj} projection queries per GPU (learned seed)",
             "c2": f"curve_set_{args.curves}: {n_proj} projection + {n_inv} inversion queries per GPU"}[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return
        cs, qs = build_workload(args.seed, 0, args.curves, n_proj, n_inv)
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
                "data": "synthetic", "config": {"workload": label, "tol_rel": TOL},
                "cpu_baseline": {"value": v, "unit": "pts/s", "cores": cores, "kind": "oracle",
                                 "sample": f"{nq} queries of the workload per step"},
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
    stream = torch.cuda.current_stream()
    cs, qs = build_workload(args.seed, rank, args.curves, n_proj, n_inv)
    dc = bspl.DeviceCurves(cs, dev)

    # decomposition (preprocessing, timed separately)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    segs = bspl.decompose(dc, TOL)
    torch.cuda.synchronize()
    decomp_ms = 1e3 * (time.perf_counter() - t0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    mlp, train = train_seed(args, rank, dev)
    p32 = bspl.measure_fma_peak(False)
    p64 = bspl.measure_fma_peak(True)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    bf16_peak = peaks["bf16_tflops"] * 1e12
    clocks = ClockSampler(local)
    clocks.start()
    head = measure_curves(args, world, dist, dev, stream, flush, segs, dc, qs, mlp, full=True,
                          peaks=(p32, p64, bf16_peak))
    beside = None
    if args.workload == "c4":
        _, q2 = build_workload(args.seed, rank, args.curves, args.queries, args.queries)
        beside = measure_curves(args, world, dist, dev, stream, flush, segs, dc, q2, mlp, full=False,
                                peaks=(p32, p64, bf16_peak))
    clk = clocks.stop()
    if bspl.mlp_check() != bspl.OK:
        raise SystemExit("a tensor-core wait timed out")

    train.update(head.pop("seed_quality"))
    out = {"metric": METRIC, "value": head["value"], "unit": "pts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16+f32+f64 (BF16 tensor-core seed, FP32 search, FP64 finish)",
           "data": "synthetic",
           "config": {"workload": label, "tol_rel": TOL, "prec": "learned_mixed", "launch": head.pop("launch"),
                      "l2": "512 MB flush between timed steps (inputs and tables also exceed L2)",
                      "segments": int(segs.total), "decompose_ms": decomp_ms, "seed_network": train}}
    out.update(head)
    out["clocks"] = clk
    if beside is not None:
        beside.pop("seed_quality", None)
        beside.pop("launch", None)
        out["c2_curve_set_1M_proj_1M_inv"] = beside
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, nq, el = cpu_oracle_rate(cs, qs)
        r1, _, nq1, el1 = cpu_oracle_rate(cs, qs, budget_s=5.0, threads=1)
        out["cpu_baseline"] = {"value": r, "unit": "pts/s", "cores": cores, "kind": "oracle",
                               "sample": f"{nq} queries of the same workload, {el:.1f} s",
                               "one_core": {"value": r1, "sample": f"{nq1} queries, {el1:.1f} s"}}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def measure_curves(args, world, dist, dev, stream, flush, segs, dc, qs, mlp, full, peaks):
    """One curve workload: the learned step (captured once as a CUDA graph by
    the library and replayed) against the plain FP64 path, accuracy against
    plain on every query, and (full) the ablations, counters, stage times,
    rooflines and the end-to-end number."""
    import torch
    from paper_2504_11498_gb300 import autotune, bspl
    p32, p64, bf16_peak = peaks
    pc = torch.as_tensor(qs.proj_curve, device=dev)
    pq = torch.as_tensor(qs.proj_xyz, device=dev)
    ic = torch.as_tensor(qs.inv_curve, device=dev)
    iq = bspl.bspl_eval_curves(dc, ic, torch.as_tensor(qs.inv_t, device=dev)) if ic.numel() else \
        torch.empty((0, 3), dtype=torch.float64, device=dev)
    has_inv = ic.numel() > 0
    n_step = pc.numel() + ic.numel()
    bufs_p = bspl.QueryBuffers(segs, pc.numel(), dev, learned=True)
    bufs_i = bspl.QueryBuffers(segs, max(ic.numel(), 1), dev, learned=True) if has_inv else None

    # the seed network's error on this workload's own seeded pairs, against
    # the midpoint seed
    seed_q = {}
    sp, ss_, found = bspl.bspl_mlp_collect_pairs(segs, pc, pq, cap=1_000_000)
    ystar = bspl.bspl_mlp_labels(segs, sp, ss_, pq)
    pred = mlp.forward(bspl.bspl_mlp_features(segs, sp, ss_, pq))
    seed_q["heldout_seed_abs_err"] = float((pred - ystar).abs().mean().item())
    seed_q["heldout_midpoint_abs_err"] = float((0.5 - ystar).abs().mean().item())
    del sp, ss_, ystar, pred

    # launch configuration per precision, chosen by the autotuner (untimed)
    cfg = {p: (autotune.tune_curves(segs, pc, pq, p) if args.samples == 0 else dict(samples=args.samples))
           for p in (bspl.MIXED, bspl.FP64)}
    cfg[bspl.LEARNED_MIXED] = (autotune.tune_curves(segs, pc, pq, bspl.LEARNED_MIXED, mlp=mlp)
                               if args.samples == 0 else {"occupancy": 0})
    cfg[bspl.CLIP_MIXED] = {k: v for k, v in cfg[bspl.LEARNED_MIXED].items() if k == "occupancy"}
    use_mlp = [mlp]

    def opts(prec, **kw):
        return bspl.make_options(prec=prec, mlp=use_mlp[0] if prec == bspl.LEARNED_MIXED else None, **cfg[prec],
                                 **kw)

    def step(prec, **kw):
        o = opts(prec, **kw)
        bspl.bspl_project_curves(segs, pc, pq, o, bufs_p)
        if has_inv:
            bspl.bspl_invert_curves(segs, ic, iq, o, bufs_i)

    def timed(run, steps, warmup):
        for _ in range(warmup):
            run()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            a.record(stream)
            run()
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    # the learned step captured once as a CUDA graph by the library (static
    # buffers), then replayed: what a serving loop does
    for _ in range(2):
        step(bspl.LEARNED_MIXED)
    torch.cuda.synchronize()
    with bspl.Graph() as graph:
        step(bspl.LEARNED_MIXED)
    torch.cuda.synchronize()
    ms_learned = timed(lambda: graph.replay(stream), args.steps, args.warmup)
    res = {}
    if full:
        ms_direct = timed(lambda: step(bspl.LEARNED_MIXED), args.steps, args.warmup)
        use_mlp[0] = None  # the same pipeline without its network (midpoint seed)
        ms_no_net = timed(lambda: step(bspl.LEARNED_MIXED), args.steps, args.warmup)
        use_mlp[0] = mlp
        ms_mixed = timed(lambda: step(bspl.MIXED), args.steps, args.warmup)
        ms_clip = timed(lambda: step(bspl.CLIP_MIXED), args.steps, args.warmup)
    ms_plain = timed(lambda: step(bspl.FP64), max(2, args.steps // 3), 2)

    # accuracy of the timed paths against the plain FP64 path on every query,
    # and of the learned path against the oracle on a sample
    diag_p = segs.diag[pc.long()]
    diag_i = segs.diag[ic.long()] if has_inv else None
    step(bspl.FP64)
    ref = (bufs_p.dist.clone(), bufs_i.dist.clone() if has_inv else None)
    acc = {}
    for name, prec in (("learned_mixed", bspl.LEARNED_MIXED),) + \
            ((("mixed", bspl.MIXED), ("clip_search", bspl.CLIP_MIXED)) if full else ()):
        step(prec)
        rel = (bufs_p.dist - ref[0]).abs() / diag_p
        if has_inv:
            rel = torch.cat([rel, (bufs_i.dist - ref[1]).abs() / diag_i])
        acc[name] = {"max_rel_dist_diff_vs_plain_fp64": float(rel.max().item()),
                     "queries_over_1e-9": int((rel > 1e-9).sum().item()),
                     "fallback_rate": float(((bufs_p.status & bspl.Q_FALLBACK) != 0).float().mean().item())}

    out = {"value": world * n_step / (ms_learned * 1e-3), "ms_per_step": ms_learned,
           "gpu_launches": int(graph.n_kernels),
           "graph": "learned step captured once by bspl_graph_begin/end (include/bspl_graph.h) and replayed; "
                    "gpu_launches = its kernel nodes",
           "plain_fp64": {"value": world * n_step / (ms_plain * 1e-3), "ms_per_step": ms_plain},
           "speedup_learned_vs_plain": ms_plain / ms_learned, "accuracy": acc, "seed_quality": seed_q,
           "launch": {str(k): v for k, v in cfg.items()}}
    if not full:
        return out

    def counted(prec):
        cnt = torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=dev)
        step(prec, counters=cnt)
        torch.cuda.synchronize()
        return dict(zip(bspl.COUNTER_NAMES, cnt.cpu().tolist()))

    c_learned, c_mixed, c_plain = counted(bspl.LEARNED_MIXED), counted(bspl.MIXED), counted(bspl.FP64)
    c_clip = counted(bspl.CLIP_MIXED)
    use_mlp[0] = None
    c_no_net = counted(bspl.LEARNED_MIXED)
    use_mlp[0] = mlp

    # per-stage device time of the learned path (events recorded by the
    # library at its stage boundaries, every call of a step summed)
    def stage_ms(steps):
        tot = np.zeros(bspl.NSTAGE_EVENTS - 1)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(bspl.NSTAGE_EVENTS)] for _ in range(2)]
        for _ in range(steps):
            flush.fill_(1.0)
            bspl.bspl_project_curves(segs, pc, pq, opts(bspl.LEARNED_MIXED, stage_events=evs[0]), bufs_p)
            if has_inv:
                flush.fill_(1.0)
                bspl.bspl_invert_curves(segs, ic, iq, opts(bspl.LEARNED_MIXED, stage_events=evs[1]), bufs_i)
            torch.cuda.synchronize()
            for e in evs[:2 if has_inv else 1]:
                tot += [e[k].elapsed_time(e[k + 1]) for k in range(bspl.NSTAGE_EVENTS - 1)]
        return dict(zip(bspl.STAGE_NAMES, (tot / steps).tolist()))

    st_ms = stage_ms(max(3, args.steps // 2))
    # the same stages without the network (seed u = 1/2): what the seed saves
    # downstream, against what it costs
    use_mlp[0] = None
    st_ms_nonet = stage_ms(max(3, args.steps // 2))
    use_mlp[0] = mlp
    n_calls = 2 if has_inv else 1

    # end to end through the public API with pinned host buffers: inputs into
    # the graph's static buffers, replay, results back
    h_in = [x.cpu().pin_memory() for x in ((pc, pq, ic, iq) if has_inv else (pc, pq))]
    outs = [bufs_p.param, bufs_p.dist, bufs_p.status] + \
        ([bufs_i.param, bufs_i.dist, bufs_i.status] if has_inv else [])
    h_out = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in outs]
    dins = (pc, pq, ic, iq) if has_inv else (pc, pq)

    def e2e_step():
        for d, h in zip(dins, h_in):
            d.copy_(h, non_blocking=True)
        graph.replay(stream)
        for h, d in zip(h_out, outs):
            h.copy_(d, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_e2e = max(3, args.steps // 2)
    e0.record(stream)
    for _ in range(k_e2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / k_e2e
    h2d = sum(x.numel() * x.element_size() for x in h_in)
    d2h = sum(x.numel() * x.element_size() for x in h_out)

    # max over ranks; every rank processed its own n_step queries
    (ms_learned, ms_direct, ms_no_net, ms_mixed, ms_clip, ms_plain, ms_e2e), total_q = combine_over_ranks(
        [ms_learned, ms_direct, ms_no_net, ms_mixed, ms_clip, ms_plain, ms_e2e], n_step, world,
        dist if world > 1 else None, dev)

    # rooflines.  ALU work from device counters with per-unit figures: 12
    # flops per box test, 110 per pair classification (E in Bernstein form
    # with its rounding bound), 15 per grid sample, 45 per Newton iteration;
    # the seed network 2 (16*128 + 2*128*128 + 128) = 69,888 flops per row.
    rows = c_learned["classified"]  # every pair the culling classified; the seeded ones run the network
    seeded = int(train_rows(segs, pc, pq, ic, iq, has_inv))
    box_flops = 12 * (c_learned["grp_tested"] + c_learned["seg_tested"])
    cls_flops = 110 * rows
    cull_flops = box_flops + cls_flops
    t_cull = max(st_ms["cull"], 1e-6) * 1e-3
    t_cls = max(st_ms["classify"], 1e-6) * 1e-3
    mlp_flops = 69888 * seeded
    t_seed = max(st_ms["seed"], 1e-6) * 1e-3
    dominant = max(st_ms, key=st_ms.get)
    mlp_line = {"bound": "tensor", "achieved": mlp_flops / t_seed / 1e12, "peak": bf16_peak / 1e12,
                "unit": "TFLOP/s", "frac": mlp_flops / t_seed / bf16_peak, "rows_per_step": seeded,
                "ms_per_step": st_ms["seed"], "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}
    cull_line = {"bound": "alu", "achieved": box_flops / t_cull / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                 "frac": box_flops / t_cull / p32, "ms_per_step": st_ms["cull"],
                 "peak_source": "FP32 FMA-chain microbenchmark on this GPU (of measured)"}
    cls_line = {"bound": "alu", "achieved": cls_flops / t_cls / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                "frac": cls_flops / t_cls / p32, "ms_per_step": st_ms["classify"], "pairs_per_step": rows}
    roofline = dict(cull_line if dominant != "seed" else mlp_line)
    roofline.update({"kernel": "k_cull_cands" if dominant != "seed" else "k_mlp_fused",
                     "traffic": (CULL_TRAFFIC_PER_LAUNCH * n_calls
                                 if dominant == "cull" and CULL_TRAFFIC_PER_LAUNCH is not None
                                 and args.workload == "c4" and full else None),
                     "traffic_unit": f"DRAM bytes per step ({n_calls} launch(es), full-size ncu capture)",
                     "stages_ms_per_step": st_ms, "dominant_stage": dominant, "mlp_seed_kernel": mlp_line,
                     "classify_kernel": cls_line})
    f32_step = cull_flops + 45 * c_learned["newton32_iters"]
    f64_step = 60 * c_learned["newton"] + 45 * max(0, c_learned["newton64_iters"] - 2 * c_learned["newton"])
    t_step = ms_learned * 1e-3
    roofline["step"] = {"frac": f32_step / t_step / p32 + f64_step / t_step / p64 + mlp_flops / t_step / bf16_peak,
                        "fp32_flops": f32_step, "fp64_flops": f64_step, "bf16_flops": mlp_flops,
                        "note": "sum of the three pipes' fractions over the timed step (ms_per_step)"}
    # the plain FP64 path: FP64 flops from its counters over the FP64 FMA
    # peak (box tests, S grid samples per candidate segment, Newton
    # iterations), over its whole timed step
    S64 = cfg[bspl.FP64]["samples"]
    f64_plain = 12 * (c_plain["grp_tested"] + c_plain["seg_tested"]) + 15 * S64 * c_plain["candidates"] + \
        45 * c_plain["newton64_iters"]
    roofline["plain_fp64"] = {"kernel": "k_query_curves<double>", "bound": "alu",
                              "achieved": f64_plain / (ms_plain * 1e-3) / 1e12, "peak": p64 / 1e12,
                              "unit": "TFLOP/s (FP64)", "frac": f64_plain / (ms_plain * 1e-3) / p64,
                              "fp64_flops": f64_plain, "ms_per_step": ms_plain,
                              "peak_source": "FP64 FMA-chain microbenchmark on this GPU (of measured)"}
    S = cfg[bspl.MIXED]["samples"]
    f32m = 12 * (c_mixed["grp_tested"] + c_mixed["seg_tested"]) + 15 * S * c_mixed["candidates"] + \
        45 * c_mixed["newton32_iters"]
    f64m = 45 * c_mixed["newton64_iters"]
    roofline["mixed_grid"] = {"kernel": "k_query_curves<float>", "bound": "alu",
                              "achieved": (f32m + f64m * p32 / p64) / (ms_mixed * 1e-3) / 1e12, "peak": p32 / 1e12,
                              "unit": "TFLOP/s (FP32-equivalent)",
                              "frac": (f32m + f64m * p32 / p64) / (ms_mixed * 1e-3) / p32, "ms_per_step": ms_mixed}
    out.update({"value": total_q / (ms_learned * 1e-3), "ms_per_step": ms_learned,
                "learned_direct": {"value": total_q / (ms_direct * 1e-3), "ms_per_step": ms_direct},
                "learned_without_network": {"value": total_q / (ms_no_net * 1e-3), "ms_per_step": ms_no_net,
                                            "stages_ms_per_step": st_ms_nonet,
                                            "network_at_bf16_peak_ms": mlp_flops / bf16_peak * 1e3,
                                            "note": "same pipeline, seed u = 1/2 instead of the network; "
                                                    "network_at_bf16_peak_ms: the seed stage's cost if it ran "
                                                    "at the measured BF16 peak"},
                "mixed_grid": {"value": total_q / (ms_mixed * 1e-3), "ms_per_step": ms_mixed},
                "clip_search": {"value": total_q / (ms_clip * 1e-3), "ms_per_step": ms_clip,
                                "note": "the learned path's culling and certification with the paper's search "
                                        "(closed-form roots of E', elimination, Bezier clipping) in place of "
                                        "the network and the FP32 isolation"},
                "plain_fp64": {"value": total_q / (ms_plain * 1e-3), "ms_per_step": ms_plain},
                "speedup_learned_vs_plain": ms_plain / ms_learned, "speedup_mixed_vs_plain": ms_plain / ms_mixed,
                "e2e": {"value": total_q / (ms_e2e * 1e-3), "unit": "pts/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "roofline": roofline, "peaks_measured": {"fp32_tflops": p32 / 1e12, "fp64_tflops": p64 / 1e12},
                "counters": {"learned_mixed": c_learned, "learned_without_network": c_no_net, "mixed": c_mixed,
                             "clip_search": c_clip, "plain_fp64": c_plain}})
    return out


def train_rows(segs, pc, pq, ic, iq, has_inv):
    """Seeded pairs (rows through the network) of one learned step."""
    from paper_2504_11498_gb300 import bspl
    n = bspl.bspl_mlp_collect_pairs(segs, pc, pq, cap=0)[2]
    if has_inv:
        n += bspl.bspl_mlp_collect_pairs(segs, ic, iq, cap=0)[2]
    return n


# ------------------------------------------------------ paper-shaped suite

PAPER_ALPHA = 1e-4  # the paper's decomposition tolerance
P_SIZES = (10_000, 50_000, 100_000)


def run_paper_suite(args, rank, world, local):
    """--workload p: one curve per paper model (a-r: the models' degrees,
    knot-vector lengths and control-point counts, 2D models at z = 0),
    each decomposed on its own at the paper's alpha = 1e-4 (timed: the
    paper counts it in its totals), then 1e4, 5e4 and 1e5 projection queries
    per model, each call followed by the refinement on the original curve
    (bspl_refine_curves), through the learned path (network trained on the
    curve-set recipe), the mixed grid path and the plain FP64 path.  value =
    learned pts/s over the 18 models at 1e5 queries each."""
    from paper_2504_11498_gb300 import synth
    label = "paper_suite_18: one curve per model a-r (2D at z = 0), 1e4/5e4/1e5 projection queries per model"
    cs, qs = synth.paper_suite(seed=17 + 1000 * rank, n_proj=P_SIZES[-1], n_inv=0)
    if args.impl == "reference":
        if rank != 0:
            return
        rates, t_all = [], 0.0
        for _ in range(args.warmup):
            cpu_oracle_rate(cs, qs, budget_s=2.0, max_q=2000)
        for _ in range(args.steps):
            r, cores, nq, el = cpu_oracle_rate(cs, qs, budget_s=8.0, max_q=20000)
            rates.append(r)
            t_all += el
        v = float(np.median(rates))
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "pts/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": label, "tol_rel": PAPER_ALPHA},
                          "cpu_baseline": {"value": v, "unit": "pts/s", "cores": cores, "kind": "oracle",
                                           "sample": f"{nq} queries of the suite per step"},
                          "e2e": {"value": v, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    import torch
    import torch.distributed as dist
    from paper_2504_11498_gb300 import bspl, build
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    mlp, train = train_seed(args, rank, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    n_max = P_SIZES[-1]
    per_model, tot = {}, {"learned": 0.0, "mixed": 0.0, "plain": 0.0, "e2e": 0.0}
    worst, over, launches = 0.0, 0, None
    for m, (name, dim, p, klen, ncp) in enumerate(synth.PAPER_MODELS):
        sub = cs.subset([m])
        dcm = bspl.DeviceCurves(sub, dev)
        for _ in range(2):  # the first call on a new shape pays one-time setup
            bspl.decompose(dcm, PAPER_ALPHA)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        segs = bspl.decompose(dcm, PAPER_ALPHA)
        torch.cuda.synchronize()
        dec_ms = 1e3 * (time.perf_counter() - t0)
        sel = slice(m * n_max, (m + 1) * n_max)
        qc_all = torch.zeros(n_max, dtype=torch.int32, device=dev)
        q_all = torch.as_tensor(qs.proj_xyz[sel], device=dev)
        row = {"dim": dim, "degree": p, "knots": klen, "cps": ncp, "segments": int(segs.total),
               "decompose_ms": dec_ms}
        paths = (("learned", bspl.LEARNED_MIXED, mlp), ("mixed", bspl.MIXED, None), ("plain", bspl.FP64, None))
        res = {}
        for n in P_SIZES:
            qc, q = qc_all[:n], q_all[:n]
            for key, prec, net in paths:
                bufs = bspl.QueryBuffers(segs, n, dev, learned=prec == bspl.LEARNED_MIXED)
                o = bspl.make_options(prec=prec, mlp=net)

                def call():
                    r = bspl.bspl_project_curves(segs, qc, q, o, bufs)
                    bspl.bspl_refine_curves(dcm, qc, q, r)

                for _ in range(max(3, args.warmup)):
                    call()
                torch.cuda.synchronize()
                # the call (projection + refinement) captured once as a CUDA
                # graph and replayed, as a serving loop does; direct calls
                # beside it (their host-side launch cost shows at 1e4 queries)
                with bspl.Graph() as g:
                    call()
                torch.cuda.synchronize()

                def timed(run):
                    for _ in range(2):
                        run()
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(args.steps)]
                    torch.cuda.synchronize()
                    for a, b in ev:
                        flush.fill_(1.0)  # L2 flush between timed calls (outside the events)
                        a.record(stream)
                        run()
                        b.record(stream)
                    torch.cuda.synchronize()
                    return float(np.mean([a.elapsed_time(b) for a, b in ev]))

                ms = timed(lambda: g.replay(stream))
                row.setdefault(f"{key}_ms", {})[str(n)] = ms
                row.setdefault(f"{key}_direct_ms", {})[str(n)] = timed(call)
                if n == n_max:
                    tot[key] += ms
                    res[key] = bufs.dist.clone()
                    if key == "learned":
                        launches = g.n_kernels
        # end to end at 1e5: pinned host queries in, results out
        h_in = torch.as_tensor(qs.proj_xyz[sel].copy()).pin_memory()
        h_qc = torch.zeros(n_max, dtype=torch.int32).pin_memory()
        bufs = bspl.QueryBuffers(segs, n_max, dev, learned=True)
        h_out = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in (bufs.param, bufs.dist, bufs.status)]
        o = bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp)
        r = bspl.bspl_project_curves(segs, qc_all, q_all, o, bufs)
        bspl.bspl_refine_curves(dcm, qc_all, q_all, r)
        torch.cuda.synchronize()
        with bspl.Graph() as g_e2e:
            r = bspl.bspl_project_curves(segs, qc_all, q_all, o, bufs)
            bspl.bspl_refine_curves(dcm, qc_all, q_all, r)
        torch.cuda.synchronize()

        def e2e():
            qc_all.copy_(h_qc, non_blocking=True)
            q_all.copy_(h_in, non_blocking=True)
            g_e2e.replay(stream)
            for h, d in zip(h_out, (bufs.param, bufs.dist, bufs.status)):
                h.copy_(d, non_blocking=True)

        for _ in range(3):
            e2e()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            e2e()
            b.record(stream)
        torch.cuda.synchronize()
        tot["e2e"] += float(np.mean([a.elapsed_time(b) for a, b in ev]))
        diag = float(segs.diag[0].item())
        rel = ((res["learned"] - res["plain"]).abs() / diag)
        worst = max(worst, float(rel.max().item()))
        over += int((rel > 1e-9).sum().item())
        row["total_ms_1e4_learned"] = dec_ms + row["learned_ms"][str(P_SIZES[0])]
        per_model[name] = row
    clk = clocks.stop()
    if bspl.mlp_check() != bspl.OK:
        raise SystemExit("a tensor-core wait timed out")
    n_all = len(synth.PAPER_MODELS) * n_max
    (t_l, t_m, t_p, t_e), total_q = combine_over_ranks([tot["learned"], tot["mixed"], tot["plain"], tot["e2e"]],
                                                       n_all, world, dist if world > 1 else None, dev)
    out = {"metric": METRIC, "value": total_q / (t_l * 1e-3), "unit": "pts/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_l, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16+f32+f64 (BF16 tensor-core seed, FP32 search, FP64 finish and refinement)",
           "data": "synthetic",
           "config": {"workload": label, "tol_rel": PAPER_ALPHA, "refine": "bspl_refine_curves after every call",
                      "step": "18 calls (one per model) of 1e5 projection queries + refinement, each "
                              "captured once as a CUDA graph and replayed (direct-call times beside it)",
                      "l2": "512 MB flush between timed calls", "seed_network": train},
           "mixed_grid": {"value": total_q / (t_m * 1e-3), "ms_per_step": t_m},
           "plain_fp64": {"value": total_q / (t_p * 1e-3), "ms_per_step": t_p},
           "speedup_learned_vs_plain": t_p / t_l,
           "accuracy": {"learned_vs_plain_fp64_refined": {"max_rel_dist_diff": worst, "queries_over_1e-9": over}},
           "e2e": {"value": total_q / (t_e * 1e-3), "unit": "pts/s",
                   "h2d_bytes_per_step": n_all * 28, "d2h_bytes_per_step": n_all * 17},
           "gpu_launches": int(launches) * len(synth.PAPER_MODELS),
           "per_model": per_model, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, nq, el = cpu_oracle_rate(cs, qs)
        out["cpu_baseline"] = {"value": r, "unit": "pts/s", "cores": cores, "kind": "oracle",
                               "sample": f"{nq} projection queries of the suite, {el:.1f} s"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------ rational curves

def refine_flops(evals, rational=True):
    """Algorithmic FP64 flops of the refinement from its evaluation counts
    per degree p (an FMA counts 2): entries 0..31 evaluate C, C', C'' (the
    triangular basis recursion 2p^2 + 4p, the sums over the span's
    homogeneous points 2 * 4 * (3p) (3 coordinates for a non-rational
    curve), the quotient rule 27), entries 32..63 C and C' alone (the sums
    2 * 4 * (2p + 1), the quotient rule 14); the squared distance and the
    Newton quantities 30 per evaluation."""
    nc = 4 if rational else 3
    full = sum(int(n) * (2 * p * p + 4 * p + 6 * nc * p + (27 if rational else 0) + 30)
               for p, n in enumerate(evals[:32]))
    part = sum(int(n) * (2 * p * p + 4 * p + 2 * nc * (2 * p + 1) + (14 if rational else 0) + 30)
               for p, n in enumerate(evals[32:64]))
    return float(full + part)


def run_nurbs(args, rank, world, local):
    """--workload nurbs: 4,096 rational curves (the curve-set recipe with
    per-control-point weights log-uniform in [1/2, 2]) decomposed at 1e-10 x
    diag into certified cubics (timed once, preprocessing).  One step = 1M
    projection + 1M inversion queries through the learned path (seed network
    trained on pairs of a second NURBS set of the same recipe), each call
    followed by the rational Newton refinement on the original curves, the
    step captured once as a CUDA graph and replayed; the same step through
    the mixed grid path and the plain FP64 path beside it.  value = learned
    pts/s (projections + inversions) per step."""
    from paper_2504_11498_gb300 import synth
    n_q = args.queries
    label = f"nurbs_curve_set_4096: {n_q} projection + {n_q} inversion queries per GPU, refined on the original curves"
    cs, qs = synth.nurbs_curve_set(seed=4 + 1000 * rank, n_proj=n_q, n_inv=n_q)
    if args.impl == "reference":
        if rank != 0:
            return
        rates, t_all = [], 0.0
        for _ in range(args.warmup):
            cpu_oracle_rate(cs, qs, budget_s=2.0, max_q=2000)
        for _ in range(args.steps):
            r, cores, nq, el = cpu_oracle_rate(cs, qs, budget_s=8.0, max_q=20000)
            rates.append(r)
            t_all += el
        v = float(np.median(rates))
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "pts/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": label, "tol_rel": TOL},
                          "cpu_baseline": {"value": v, "unit": "pts/s", "cores": cores, "kind": "oracle",
                                           "sample": f"{nq} queries of the workload per step"},
                          "e2e": {"value": v, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    import torch
    import torch.distributed as dist
    from paper_2504_11498_gb300 import bspl, build
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    mlp, train = train_seed(args, rank, dev, rational=True)
    dc = bspl.DeviceCurves(cs, dev)
    for _ in range(2):
        bspl.decompose(dc, TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    segs = bspl.decompose(dc, TOL)
    torch.cuda.synchronize()
    dec_ms = 1e3 * (time.perf_counter() - t0)
    pc, pq = torch.as_tensor(qs.proj_curve, device=dev), torch.as_tensor(qs.proj_xyz, device=dev)
    ic = torch.as_tensor(qs.inv_curve, device=dev)
    iq = bspl.bspl_eval_curves(dc, ic, torch.as_tensor(qs.inv_t, device=dev))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(run, prep=None):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            if prep is not None:
                prep()
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            a.record(stream)
            run()
            b.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    paths = (("learned", bspl.LEARNED_MIXED, mlp), ("mixed", bspl.MIXED, None), ("plain", bspl.FP64, None))
    ms, res, graphs, bufs_of = {}, {}, {}, {}
    rws = bspl.refine_workspace(dc, n_q, dev)  # the refinement groups its queries by curve
    clocks = ClockSampler(local)
    clocks.start()
    for key, prec, net in paths:
        learned = prec == bspl.LEARNED_MIXED
        bp = bspl.QueryBuffers(segs, n_q, dev, learned=learned)
        bi = bspl.QueryBuffers(segs, n_q, dev, learned=learned)
        o = bspl.make_options(prec=prec, mlp=net)

        def step(bp=bp, bi=bi, o=o):
            r = bspl.bspl_project_curves(segs, pc, pq, o, bp)
            bspl.bspl_refine_curves(dc, pc, pq, r, ws=rws)
            r = bspl.bspl_invert_curves(segs, ic, iq, o, bi)
            bspl.bspl_refine_curves(dc, ic, iq, r, invert=True, diag=segs.diag, ws=rws)

        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        with bspl.Graph() as g:
            step()
        for _ in range(2):
            g.replay(stream)
        ms[key] = timed(lambda: g.replay(stream))
        graphs[key], bufs_of[key] = g, (bp, bi, o)
        res[key] = (bp.dist.clone(), bi.dist.clone())
    # the refinement alone (learned path's results before refinement restored
    # before each timed pair of refinement launches), and its evaluation counts
    bp, bi, o = bufs_of["learned"]
    bspl.bspl_project_curves(segs, pc, pq, o, bp)
    bspl.bspl_invert_curves(segs, ic, iq, o, bi)
    saved = [x.clone() for x in (bp.param, bp.dist, bp.status, bi.param, bi.dist, bi.status)]

    def restore():
        for x, y in zip((bp.param, bp.dist, bp.status, bi.param, bi.dist, bi.status), saved):
            x.copy_(y)

    def refine_pair(evals=None):
        bspl.bspl_refine_curves(dc, pc, pq, bp, evals=evals, ws=rws)
        bspl.bspl_refine_curves(dc, ic, iq, bi, invert=True, diag=segs.diag, evals=evals, ws=rws)

    restore()
    refine_pair()
    refine_ms = timed(refine_pair, prep=restore)
    evals = torch.zeros(bspl.REFINE_EVALS, dtype=torch.int64, device=dev)
    restore()
    refine_pair(evals)
    torch.cuda.synchronize()
    ev_counts = evals.cpu().numpy().tolist()
    # end to end: pinned host queries in, results out, around the learned graph
    h_in = [torch.as_tensor(x).pin_memory() for x in (qs.proj_curve, qs.proj_xyz, qs.inv_curve)]
    h_iq = iq.cpu().pin_memory()
    h_out = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
             for x in (bp.param, bp.dist, bp.status, bi.param, bi.dist, bi.status)]
    g = graphs["learned"]

    def e2e():
        for d, h in zip((pc, pq, ic, iq), h_in + [h_iq]):
            d.copy_(h, non_blocking=True)
        g.replay(stream)
        for h, d in zip(h_out, (bp.param, bp.dist, bp.status, bi.param, bi.dist, bi.status)):
            h.copy_(d, non_blocking=True)

    for _ in range(3):
        e2e()
    e2e_ms = timed(e2e)
    clk = clocks.stop()
    if bspl.mlp_check() != bspl.OK:
        raise SystemExit("a tensor-core wait timed out")
    diag = segs.diag.double()
    worst, over = 0.0, 0
    for a, b, idx in ((res["learned"][0], res["plain"][0], pc), (res["learned"][1], res["plain"][1], ic)):
        rel = (a - b).abs() / diag[idx.long()]
        worst = max(worst, float(rel.max().item()))
        over += int((rel > 1e-9).sum().item())
    dist_i = res["learned"][1] / diag[ic.long()]
    off_curve = int((dist_i > 1e-9).sum().item())
    (t_l, t_m, t_p, t_r, t_e), total_q = combine_over_ranks(
        [ms["learned"], ms["mixed"], ms["plain"], refine_ms, e2e_ms], 2 * n_q, world, dist if world > 1 else None,
        dev)
    p64 = bspl.measure_fma_peak(True)
    flops = refine_flops(ev_counts)
    achieved = flops / (t_r * 1e-3)
    roofline = {"kernel": "k_refine_curves<4> (rational Newton, FP64)", "bound": "alu",
                "achieved": achieved / 1e12, "peak": p64 / 1e12, "unit": "TFLOP/s", "frac": achieved / p64,
                "peak_kind": "FP64 FMA-chain peak measured by bspl.measure_fma_peak on this GPU",
                "traffic": None, "flops_per_step": flops, "evaluations_per_step": int(sum(ev_counts)),
                "share_of_learned_step": t_r / t_l}
    out = {"metric": METRIC, "value": total_q / (t_l * 1e-3), "unit": "pts/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_l, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16+f32+f64 (BF16 tensor-core seed, FP32 search, FP64 finish and rational refinement)",
           "data": "synthetic",
           "config": {"workload": label, "tol_rel": TOL, "weights": "log-uniform in [1/2, 2]",
                      "step": "learned projection + refinement, learned inversion + refinement, one CUDA graph",
                      "l2": "512 MB flush between timed steps", "seed_network": train,
                      "segments": int(segs.total), "decompose_ms": dec_ms},
           "mixed_grid": {"value": total_q / (t_m * 1e-3), "ms_per_step": t_m},
           "plain_fp64": {"value": total_q / (t_p * 1e-3), "ms_per_step": t_p},
           "speedup_learned_vs_plain": t_p / t_l,
           "refine": {"ms_per_step": t_r,
                      "evaluations_by_degree": {str(p): int(n) for p, n in enumerate(ev_counts[:32]) if n},
                      "trial_evaluations_by_degree": {str(p): int(n) for p, n in enumerate(ev_counts[32:64]) if n}},
           "accuracy": {"learned_vs_plain_fp64_refined": {"max_rel_dist_diff": worst, "queries_over_1e-9": over},
                        "inversions_over_1e-9": off_curve},
           "e2e": {"value": total_q / (t_e * 1e-3), "unit": "pts/s",
                   "h2d_bytes_per_step": n_q * (4 + 24 + 4 + 24), "d2h_bytes_per_step": 2 * n_q * 17},
           "gpu_launches": int(graphs["learned"].n_kernels), "roofline": roofline, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, nq, el = cpu_oracle_rate(cs, qs)
        out["cpu_baseline"] = {"value": r, "unit": "pts/s", "cores": cores, "kind": "oracle",
                               "sample": f"{nq} queries of the workload (half projection, half inversion), "
                                         f"{el:.1f} s"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------- surfaces and ragged batch

def build_surface_workload(kind, rank, n_surf=1024, n_q=4_000_000):
    """c3: the 1,024-surface set, 4M projection + 4M inversion queries
    (smaller with --surfaces / --surface-queries).
    c5: 65,536 cubic curves + 8,192 bicubic surfaces, 64M queries (32M per
    spline kind, half projection, half inversion), Zipf(1.1) over splines."""
    from paper_2504_11498_gb300 import synth
    if kind == "c3":
        ss, sq = synth.surface_set(seed=3 + 1000 * rank, n_surf=n_surf, n_proj=n_q, n_inv=n_q)
        return None, None, ss, sq
    cs, ss, qc, qs, rng = synth.ragged_mix(seed=5 + 1000 * rank)
    cq, sq = synth.ragged_queries(cs, ss, qc, qs, rng)
    return cs, cq, ss, sq


def cpu_oracle_surface_rate(cs, cq, ss, sq, budget_s=15.0, threads=0):
    """Oracle on the host cores, bounded sample: surface projection and
    inversion queries (and, for the ragged batch, as many curve queries)."""
    from oracle import oracle as O
    threads = threads or O.num_threads()
    m = 4000
    S = O.eval_surfaces(ss, sq.inv_surf[:m], sq.inv_uv[:m])[0]
    B = O.eval_surfaces(ss, sq.proj_surf[:m], sq.proj_uv[:m])[0]
    Pq = B + sq.proj_dir[:m] * sq.proj_r[:m, None]
    if cq is not None:
        C = O.eval_curves(cs, cq.inv_curve[:m], cq.inv_t[:m])[0]
    done, el, n = 0, 0.0, 50
    while el < budget_s and done < m:
        k = min(n, m - done)
        t0 = time.perf_counter()
        O.project_surfaces(ss, sq.proj_surf[done:done + k], Pq[done:done + k], nthreads=threads)
        O.project_surfaces(ss, sq.inv_surf[done:done + k], S[done:done + k], nthreads=threads)
        if cq is not None:
            O.project_curves(cs, cq.proj_curve[done:done + k], cq.proj_xyz[done:done + k], nthreads=threads)
            O.project_curves(cs, cq.inv_curve[done:done + k], C[done:done + k], nthreads=threads)
        el += time.perf_counter() - t0
        done += k
        n = min(2 * n, 1000)
    per = 2 if cq is None else 4
    return per * done / el, threads, per * done, el


def run_surface_workloads(args, rank, world, local):
    """The surface set (c3) and the ragged batch (c5).  A step: every query
    of the batch once.  Surfaces run the mixed path (FP32 grid seed and
    Newton, last steps in FP64 on the original patch); the ragged batch's
    curves run the learned path.  Both are set against the plain FP64 path
    on the same queries."""
    label = {"c3": f"surface_set_{args.surfaces}: {args.surface_queries} projection + {args.surface_queries} "
                   "inversion queries (bi-degree 2..5)",
             "c5": "ragged_mix: 65,536 cubic curves + 8,192 bicubic surfaces, 64M queries (Zipf 1.1), "
                   "half projection, half inversion per spline kind"}[args.workload]
    if args.impl == "reference":
        if rank != 0:
            return
        cs, cq, ss, sq = build_surface_workload(args.workload, 0, args.surfaces, args.surface_queries)
        rates, t_all = [], 0.0
        for _ in range(args.warmup):
            cpu_oracle_surface_rate(cs, cq, ss, sq, budget_s=1.0)
        for _ in range(args.steps):
            r, cores, nq, el = cpu_oracle_surface_rate(cs, cq, ss, sq, budget_s=6.0)
            rates.append(r)
            t_all += el
        v = float(np.median(rates))
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "pts/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": label},
                          "cpu_baseline": {"value": v, "unit": "pts/s", "cores": cores, "kind": "oracle",
                                           "sample": f"{nq} queries per step"},
                          "e2e": {"value": v, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    import torch.distributed as dist
    from paper_2504_11498_gb300 import bspl, build

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    cs, cq, ss, sq = build_surface_workload(args.workload, rank, args.surfaces, args.surface_queries)
    has_c = cs is not None

    def T(x, dt):
        return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dsf = bspl.DeviceSurfaces(ss, dev)
    ssegs = bspl.decompose(dsf, SURF_TOL)
    torch.cuda.synchronize()
    dec_s = 1e3 * (time.perf_counter() - t0)
    ps = T(sq.proj_surf, torch.int32)
    sp = bspl.bspl_eval_surfaces(dsf, ps, T(sq.proj_uv, torch.float64)) + \
        T(sq.proj_dir, torch.float64) * T(sq.proj_r, torch.float64)[:, None]
    isf = T(sq.inv_surf, torch.int32)
    si = bspl.bspl_eval_surfaces(dsf, isf, T(sq.inv_uv, torch.float64))
    calls = [("surf_proj", bspl.bspl_project_surfaces, ssegs, ps, sp),
             ("surf_inv", bspl.bspl_invert_surfaces, ssegs, isf, si)]
    mlp, dec_c, train = None, None, None
    if has_c:
        t0 = time.perf_counter()
        dc = bspl.DeviceCurves(cs, dev)
        csegs = bspl.decompose(dc, TOL)
        torch.cuda.synchronize()
        dec_c = 1e3 * (time.perf_counter() - t0)
        pc, ic = T(cq.proj_curve, torch.int32), T(cq.inv_curve, torch.int32)
        cpq = T(cq.proj_xyz, torch.float64)
        ciq = bspl.bspl_eval_curves(dc, ic, T(cq.inv_t, torch.float64))
        calls = [("curve_proj", bspl.bspl_project_curves, csegs, pc, cpq),
                 ("curve_inv", bspl.bspl_invert_curves, csegs, ic, ciq)] + calls
        mlp, train = train_seed(args, rank, dev)
    smlp, strain = train_surface_seed(args.workload, rank, dev)
    bufs = {name: bspl.QueryBuffers(sg, qi.numel(), dev, learned=True) for name, _, sg, qi, _ in calls}
    n_step = sum(qi.numel() for _, _, _, qi, _ in calls)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # launch configuration per call and precision, chosen by the autotuner
    # (untimed; curves: occupancy and FP32 steps, surfaces: sample tile and
    # FP32 steps)
    from paper_2504_11498_gb300 import autotune
    tuned = {}
    for name, fn, sg, qi, qx in calls:
        for fast in (True, False):
            if name.startswith("curve"):
                prec = bspl.LEARNED_MIXED if fast else bspl.FP64
                tuned[(name, fast)] = autotune.tune_curves(sg, qi, qx, prec, mlp=mlp if fast else None)
            else:
                tuned[(name, fast)] = (autotune.tune_surfaces(sg, qi, qx, bspl.LEARNED_MIXED, mlp=smlp) if fast
                                       else autotune.tune_surfaces(sg, qi, qx, bspl.FP64))
    surf_mode = [bspl.LEARNED_MIXED, smlp]  # the surfaces' fast path (switched for the ablations)

    def opts(name, fast, **kw):
        cfg_ = dict(tuned[(name, fast)], **kw)
        if not fast:
            return bspl.make_options(prec=bspl.FP64, **cfg_)
        if name.startswith("curve"):
            return bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp, **cfg_)
        return bspl.make_options(prec=surf_mode[0], mlp=surf_mode[1], **cfg_)

    def step(fast, only=None, **kw):
        for name, fn, sg, qi, qx in calls:
            if only is None or name == only:
                fn(sg, qi, qx, opts(name, fast, **kw), bufs[name])

    def timed(fast, steps, warmup, only=None):
        for _ in range(warmup):
            step(fast, only)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            step(fast, only)
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    # the fast step captured once as a CUDA graph by the library, replayed
    step(True)
    torch.cuda.synchronize()
    with bspl.Graph() as graph:
        step(True)
    torch.cuda.synchronize()

    def timed_graph(steps, warmup):
        for _ in range(warmup):
            graph.replay(stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            graph.replay(stream)
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    clocks = ClockSampler(local)
    clocks.start()
    ms_fast = timed_graph(args.steps, args.warmup)
    ms_plain = timed(False, max(2, args.steps // 3), 2)
    per_call = {name: timed(True, max(2, args.steps // 2), 1, only=name) for name, *_ in calls}
    # the surfaces through the grid-seeded mixed path, and through the
    # learned path without its network (seed = patch centre)
    surf_names = [name for name, *_ in calls if name.startswith("surf")]
    surf_mode[:] = [bspl.MIXED, None]
    ms_surf_grid = sum(timed(True, max(2, args.steps // 2), 1, only=nm) for nm in surf_names)
    surf_mode[:] = [bspl.LEARNED_MIXED, None]
    ms_surf_nonet = sum(timed(True, max(2, args.steps // 2), 1, only=nm) for nm in surf_names)
    surf_mode[:] = [bspl.LEARNED_MIXED, smlp]
    ms_surf_learned = sum(per_call[nm] for nm in surf_names)
    clk = clocks.stop()
    if bspl.mlp_check() != bspl.OK:
        raise SystemExit("a tensor-core wait timed out")

    # accuracy of the timed path against the plain FP64 path, every query
    step(False)
    ref = {name: bufs[name].dist.clone() for name in bufs}
    step(True)
    acc = {}
    for name, _, sg, qi, _ in calls:
        rel = (bufs[name].dist - ref[name]).abs() / sg.diag[qi.long()]
        acc[name] = {"max_rel_dist_diff_vs_plain_fp64": float(rel.max().item()),
                     "queries_over_1e-9": int((rel > 1e-9).sum().item())}

    cnt = {}
    for name, *_ in calls:
        c = torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=dev)
        step(True, only=name, counters=c)
        torch.cuda.synchronize()
        cnt[name] = dict(zip(bspl.COUNTER_NAMES, c.cpu().tolist()))

    # end to end through the public API: inputs from pinned host memory,
    # results back, every step
    h_in = {name: (qi.cpu().pin_memory(), qx.cpu().pin_memory()) for name, _, _, qi, qx in calls}
    h_out = {name: [torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
                    for x in (bufs[name].param, bufs[name].dist, bufs[name].status)] for name in bufs}

    def e2e_step():
        for name, _, _, qi, qx in calls:
            qi.copy_(h_in[name][0], non_blocking=True)
            qx.copy_(h_in[name][1], non_blocking=True)
        graph.replay(stream)
        for name in bufs:
            for h, d in zip(h_out[name], (bufs[name].param, bufs[name].dist, bufs[name].status)):
                h.copy_(d, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_e2e = max(2, args.steps // 3)
    e0.record(stream)
    for _ in range(k_e2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / k_e2e
    h2d = sum(a.numel() * a.element_size() + b.numel() * b.element_size() for a, b in h_in.values())
    d2h = sum(x.numel() * x.element_size() for v in h_out.values() for x in v)

    (ms_fast, ms_plain, ms_e2e), total_q = combine_over_ranks([ms_fast, ms_plain, ms_e2e], n_step, world,
                                                              dist if world > 1 else None, dev)

    # roofline of the dominant call.  Surfaces (mixed): 12 FP32 flops per
    # group or patch box test, 95 per bicubic grid sample (power-form Horner
    # in u and v for 3 coordinates, then the squared distance), GU x GV = 32
    # samples per surviving patch; Newton iterations are not counted, so the
    # figure is a lower bound.  Curves (learned): as in the curve bench.
    p32 = bspl.measure_fma_peak(False)
    dominant = max(per_call, key=per_call.get)
    c = cnt[dominant]
    if dominant.startswith("surf"):
        flops = 12 * (c["grp_tested"] + c["seg_tested"]) + 95 * 32 * c["candidates"]
        kern = "k_query_surfaces<float,8,4,true>"
    else:
        flops = 12 * (c["grp_tested"] + c["seg_tested"]) + 110 * c["classified"] + 45 * c["newton32_iters"]
        kern = "learned curve path (k_cull_pairs + pair kernels)"
    t_dom = per_call[dominant] * 1e-3
    roofline = {"bound": "alu", "achieved": flops / t_dom / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                "frac": flops / t_dom / p32, "traffic": None, "kernel": kern, "call": dominant,
                "ms_per_step": per_call[dominant], "calls_ms_per_step": per_call,
                "peak_source": "FP32 FMA-chain microbenchmark on this GPU (of measured)",
                "note": "counted FP32 flops only (Newton iterations of the surface kernel uncounted): a lower bound"}

    cfg = {"workload": label, "tol_rel_curves": TOL, "tol_rel_surfaces": SURF_TOL, "surface_seed_network": strain,
           "launch": {f"{k[0]}|{'fast' if k[1] else 'plain'}": v for k, v in tuned.items()},
           "schedule": "queries grouped heaviest spline first; persistent work-stealing launches",
           "prec": "surfaces learned_mixed" + (", curves learned_mixed" if has_c else ""),
           "l2": "512 MB flush between timed steps", "patches": int(ssegs.total), "decompose_surfaces_ms": dec_s}
    if has_c:
        cfg.update({"segments": int(csegs.total), "decompose_curves_ms": dec_c, "seed_network": train})
    out = {"metric": METRIC, "value": total_q / (ms_fast * 1e-3), "unit": "pts/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_fast, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16+f32+f64 (BF16 tensor-core seeds, FP32 search, FP64 finish)",
           "data": "synthetic", "config": cfg,
           "plain_fp64": {"value": total_q / (ms_plain * 1e-3), "ms_per_step": ms_plain},
           "speedup_vs_plain": ms_plain / ms_fast, "accuracy": acc,
           "surfaces_ms_per_step": {"learned_mixed": ms_surf_learned, "learned_without_network": ms_surf_nonet,
                                    "mixed_grid": ms_surf_grid,
                                    "note": "surface calls only, each timed alone (not the graph replay)"},
           "e2e": {"value": total_q / (ms_e2e * 1e-3), "unit": "pts/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": int(graph.n_kernels),
           "graph": "fast step captured once by bspl_graph_begin/end and replayed; gpu_launches = its kernel nodes",
           "roofline": roofline, "clocks": clk, "counters": cnt}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, nq, el = cpu_oracle_surface_rate(cs, cq, ss, sq)
        out["cpu_baseline"] = {"value": r, "unit": "pts/s", "cores": cores, "kind": "oracle",
                               "sample": f"{nq} queries of the same workload, {el:.1f} s"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
