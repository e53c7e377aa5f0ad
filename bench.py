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
SURF_TOL = 1e-4  # surfaces: decomposed at the paper's alpha, last Newton steps on the original patch
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
    ap.add_argument("--workload", default="c2", choices=["c2", "c4", "c3", "c5"],
                    help="c2: 1M projection + 1M inversion queries; c4: 16M projection queries, same curves; "
                         "c3: 1,024 surfaces, 4M + 4M queries; c5: 65,536 cubic curves + 8,192 bicubic "
                         "surfaces, 64M Zipf-skewed queries")
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

def train_seed(args, rank, dev):
    """Trains the seed network on (segment, query, t*) pairs of a second
    curve set of the same recipe (seed 12): pairs from the learned path's own
    culling, labels from the FP64 solver, hand-written training kernels.
    Returns the network and a summary (untimed preprocessing)."""
    import torch
    from paper_2504_11498_gb300 import bspl, synth
    t0 = time.perf_counter()
    cs, qs = synth.curve_set(seed=12 + 1000 * rank, n_curves=args.train_curves, n_proj=args.train_queries,
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


# ------------------------------------------------------------------- main

def main():
    args = parse()
    n_inv = None
    if args.workload == "c4":  # the learned-seed configuration: projection queries only
        args.queries = 16_000_000 if args.queries == 1_000_000 else args.queries
        n_inv = 0
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.workload in ("c3", "c5"):
        return run_surface_workloads(args, rank, world, local)

    if args.impl == "reference":
        if rank != 0:
            return
        cs, qs = build_workload(args.seed, 0, args.curves, args.queries, n_inv)
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
    stream = torch.cuda.current_stream()
    cs, qs = build_workload(args.seed, rank, args.curves, args.queries, n_inv)
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
    bufs_p = bspl.QueryBuffers(segs, pc.numel(), dev, learned=True)
    bufs_i = bspl.QueryBuffers(segs, ic.numel(), dev, learned=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # the learned seed, trained before anything is timed; its error on this
    # workload's own seeded pairs, against the midpoint seed
    mlp, train = train_seed(args, rank, dev)
    rows = 0
    for qcur, qpts in ((pc, pq), (ic, iq)):
        sp, ss, found = bspl.bspl_mlp_collect_pairs(segs, qcur, qpts, cap=1_000_000)
        rows += found
        if qcur is pc:
            ystar = bspl.bspl_mlp_labels(segs, sp, ss, qpts)
            pred = mlp.forward(bspl.bspl_mlp_features(segs, sp, ss, qpts))
            train["heldout_seed_abs_err"] = float((pred - ystar).abs().mean().item())
            train["heldout_midpoint_abs_err"] = float((0.5 - ystar).abs().mean().item())
    train["eval_seed_rows_per_step"] = int(rows)

    # launch configuration per precision, chosen by the autotuner (untimed)
    cfg = {p: (autotune.tune_curves(segs, pc, pq, p) if args.samples == 0 else dict(samples=args.samples))
           for p in (bspl.MIXED, bspl.FP64)}
    cfg[bspl.LEARNED_MIXED] = (autotune.tune_curves(segs, pc, pq, bspl.LEARNED_MIXED, mlp=mlp)
                               if args.samples == 0 else {"occupancy": 0})

    def opts(prec, **kw):
        return bspl.make_options(prec=prec, mlp=mlp if prec == bspl.LEARNED_MIXED else None, **cfg[prec], **kw)

    def step(prec, **kw):
        o = opts(prec, **kw)
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
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    def counted(prec):
        cnt = torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=dev)
        step(prec, counters=cnt)
        torch.cuda.synchronize()
        return dict(zip(bspl.COUNTER_NAMES, cnt.cpu().tolist()))

    # the learned step captured once as a CUDA graph (static buffers), then
    # replayed: what a serving loop does
    def capture(prec):
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(2):
                step(prec)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step(prec)
        torch.cuda.synchronize()
        return g

    graph = capture(bspl.LEARNED_MIXED)

    def timed_graph(steps, warmup):
        for _ in range(warmup):
            graph.replay()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            graph.replay()
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    # clocks are sampled across the timed loops
    clocks = ClockSampler(local)
    clocks.start()
    ms_learned = timed_graph(args.steps, args.warmup)
    ms_learned_direct = timed(bspl.LEARNED_MIXED, args.steps, args.warmup)
    # the same pipeline without its network (midpoint seed): what the network
    # costs and saves in time
    mlp_keep = mlp
    mlp = None
    ms_no_net = timed(bspl.LEARNED_MIXED, args.steps, args.warmup)
    mlp = mlp_keep
    ms_mixed = timed(bspl.MIXED, args.steps, args.warmup)
    ms_plain = timed(bspl.FP64, max(2, args.steps // 3), 2)
    clk = clocks.stop()
    if bspl.mlp_check() != bspl.OK:
        raise SystemExit("a tensor-core wait timed out")

    # accuracy of the timed paths against the plain FP64 path, every query
    acc = {}
    diag_p = segs.diag[pc.long()]
    diag_i = segs.diag[ic.long()]
    step(bspl.FP64)
    ref = (bufs_p.dist.clone(), bufs_i.dist.clone())
    for name, prec in (("learned_mixed", bspl.LEARNED_MIXED), ("mixed", bspl.MIXED)):
        step(prec)
        rel = torch.cat([(bufs_p.dist - ref[0]).abs() / diag_p, (bufs_i.dist - ref[1]).abs() / diag_i])
        acc[name] = {"max_rel_dist_diff_vs_plain_fp64": float(rel.max().item()),
                     "queries_over_1e-9": int((rel > 1e-9).sum().item())}

    c_learned = counted(bspl.LEARNED_MIXED)
    c_mixed = counted(bspl.MIXED)
    c_plain = counted(bspl.FP64)

    # per-stage device time of the learned path (events recorded by the
    # library at its stage boundaries, both calls of a step summed)
    def stage_ms(steps):
        tot = np.zeros(bspl.NSTAGE_EVENTS - 1)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(bspl.NSTAGE_EVENTS)] for _ in range(2)]
        for _ in range(steps):
            flush.fill_(1.0)
            bspl.bspl_project_curves(segs, pc, pq, opts(bspl.LEARNED_MIXED, stage_events=evs[0]), bufs_p)
            flush.fill_(1.0)
            bspl.bspl_invert_curves(segs, ic, iq, opts(bspl.LEARNED_MIXED, stage_events=evs[1]), bufs_i)
            torch.cuda.synchronize()
            for e in evs:
                tot += [e[k].elapsed_time(e[k + 1]) for k in range(bspl.NSTAGE_EVENTS - 1)]
        return dict(zip(bspl.STAGE_NAMES, (tot / steps).tolist()))

    st_ms = stage_ms(max(3, args.steps // 2))

    # the grid kernel alone (mixed), pre-grouped inputs, events around launches
    op = torch.as_tensor(np.argsort(qs.proj_curve, kind="stable"), device=dev)
    oi = torch.as_tensor(np.argsort(qs.inv_curve, kind="stable"), device=dev)
    spc, spq, sic, siq = pc[op], pq[op], ic[oi], iq[oi]

    def kernel_ms(prec, steps):
        o = bspl.make_options(prec=prec, sort_queries=0, **cfg[prec])
        tot = 0.0
        for it in range(steps + 2):
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
            if it >= 2:
                tot += ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])
        return tot / steps

    kms_mixed = kernel_ms(bspl.MIXED, max(3, args.steps // 2))

    # end to end through the public API with pinned host buffers
    h_in = [x.cpu().pin_memory() for x in (pc, pq, ic, iq)]
    h_out = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in
             (bufs_p.param, bufs_p.dist, bufs_p.status, bufs_i.param, bufs_i.dist, bufs_i.status)]

    def e2e_step():
        # inputs into the graph's static buffers, replay, results back
        for d, h in zip((pc, pq, ic, iq), h_in):
            d.copy_(h, non_blocking=True)
        graph.replay()
        for h, d in zip(h_out, (bufs_p.param, bufs_p.dist, bufs_p.status, bufs_i.param, bufs_i.dist,
                                bufs_i.status)):
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
    (ms_learned, ms_mixed, ms_plain, ms_e2e), total_q = combine_over_ranks(
        [ms_learned, ms_mixed, ms_plain, ms_e2e], n_step, world, dist if world > 1 else None, dev)

    # rooflines.  ALU work from device counters with per-unit figures: 12
    # FP32 flops per box test, 110 per pair classification (E in Bernstein
    # form with its rounding bound), 15 per grid sample, 45 per Newton
    # iteration; the MLP 2 (16*128 + 2*128*128 + 128) = 69,888 flops per row.
    p32 = bspl.measure_fma_peak(False)
    p64 = bspl.measure_fma_peak(True)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    bf16_peak = peaks["bf16_tflops"] * 1e12
    cull_flops = 12 * (c_learned["grp_tested"] + c_learned["seg_tested"]) + 110 * c_learned["candidates"]
    t_cull = st_ms["cull"] * 1e-3
    rows = train["eval_seed_rows_per_step"]
    mlp_flops = 69888 * rows
    t_seed = st_ms["seed"] * 1e-3
    dominant = max(st_ms, key=st_ms.get)
    mlp_line = {"bound": "tensor", "achieved": mlp_flops / t_seed / 1e12, "peak": bf16_peak / 1e12,
                "unit": "TFLOP/s", "frac": mlp_flops / t_seed / bf16_peak, "rows_per_step": rows,
                "ms_per_step": st_ms["seed"], "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}
    cull_line = {"bound": "alu", "achieved": cull_flops / t_cull / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                 "frac": cull_flops / t_cull / p32, "ms_per_step": st_ms["cull"],
                 "peak_source": "FP32 FMA-chain microbenchmark on this GPU (of measured)"}
    roofline = dict(cull_line if dominant == "cull" else (mlp_line if dominant == "seed" else cull_line))
    # DRAM bytes of the dominant kernel per step: ncu capture of the same
    # kernel on the 1,024-curve, 250k + 250k-query case (247.6 MB per
    # launch), scaled by the units processed (4x queries and tables) and the
    # two launches of a step
    n_calls = 2 if ic.numel() > 0 else 1
    traffic = n_calls * 4 * 247.56e6 * (pc.numel() / 1_000_000) if dominant == "cull" else None
    roofline.update({"kernel": "k_cull_pairs" if roofline["bound"] == "alu" else "k_mlp_fused",
                     "traffic": traffic, "traffic_unit": f"bytes per step ({n_calls} launch(es))",
                     "stages_ms_per_step": st_ms, "dominant_stage": dominant,
                     "mlp_seed_kernel": mlp_line})

    # the whole learned step: counted FP32 flops / FP32 peak + FP64 flops /
    # FP64 peak + MLP flops / BF16 peak, per second of the timed step
    f32_step = cull_flops + 45 * c_learned["newton32_iters"]
    f64_step = 60 * c_learned["newton"] + 45 * max(0, c_learned["newton64_iters"] - 2 * c_learned["newton"])
    t_step = ms_learned * 1e-3
    roofline["step"] = {"frac": f32_step / t_step / p32 + f64_step / t_step / p64 + mlp_flops / t_step / bf16_peak,
                        "fp32_flops": f32_step, "fp64_flops": f64_step, "bf16_flops": mlp_flops,
                        "note": "sum of the three pipes' fractions over the timed step (ms_per_step)"}

    S = cfg[bspl.MIXED]["samples"]
    f32m = 12 * (c_mixed["grp_tested"] + c_mixed["seg_tested"]) + 15 * S * c_mixed["candidates"] + \
        45 * c_mixed["newton32_iters"]
    f64m = 45 * c_mixed["newton64_iters"]
    eq_m = (f32m + f64m * p32 / p64) / (kms_mixed * 1e-3)
    roofline["mixed_grid_kernel"] = {"kernel": "k_query_curves<float>", "bound": "alu", "achieved": eq_m / 1e12,
                                     "peak": p32 / 1e12, "unit": "TFLOP/s (FP32-equivalent)", "frac": eq_m / p32,
                                     "ms_per_step": kms_mixed, "fp64_peak_tflops": p64 / 1e12}

    out = {"metric": METRIC, "value": total_q / (ms_learned * 1e-3), "unit": "pts/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_learned, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16+f32+f64 (BF16 tensor-core seed, FP32 search, FP64 finish)", "data": "synthetic",
           "config": {"workload": f"curve_set_{args.curves}: {pc.numel()} projection + {ic.numel()} inversion "
                                  "queries per GPU",
                      "tol_rel": TOL, "prec": "learned_mixed", "launch": {str(k): v for k, v in cfg.items()},
                      "l2": "512 MB flush between timed steps", "segments": int(segs.total),
                      "decompose_ms": decomp_ms, "seed_network": train},
           "graph": "learned step captured once as a CUDA graph and replayed",
           "learned_direct": {"value": total_q / (ms_learned_direct * 1e-3), "ms_per_step": ms_learned_direct},
           "learned_without_network": {"value": total_q / (ms_no_net * 1e-3), "ms_per_step": ms_no_net,
                                       "note": "same pipeline, seed u = 1/2 instead of the network"},
           "mixed_grid": {"value": total_q / (ms_mixed * 1e-3), "ms_per_step": ms_mixed},
           "plain_fp64": {"value": total_q / (ms_plain * 1e-3), "ms_per_step": ms_plain},
           "speedup_learned_vs_plain": ms_plain / ms_learned, "speedup_mixed_vs_plain": ms_plain / ms_mixed,
           "accuracy": acc,
           "e2e": {"value": total_q / (ms_e2e * 1e-3), "unit": "pts/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": 26, "roofline": roofline, "clocks": clk,
           "counters": {"learned_mixed": c_learned, "mixed": c_mixed, "plain_fp64": c_plain}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, nq, el = cpu_oracle_rate(cs, qs)
        r1, _, nq1, el1 = cpu_oracle_rate(cs, qs, budget_s=5.0, threads=1)
        out["cpu_baseline"] = {"value": r, "unit": "pts/s", "cores": cores, "kind": "oracle",
                               "sample": f"{nq} queries of the same workload (half projection, half inversion), "
                                         f"{el:.1f} s",
                               "one_core": {"value": r1, "sample": f"{nq1} queries, {el1:.1f} s"}}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------- surfaces and ragged batch

def build_surface_workload(kind, rank):
    """c3: the 1,024-surface set, 4M projection + 4M inversion queries.
    c5: 65,536 cubic curves + 8,192 bicubic surfaces, 64M queries (32M per
    spline kind, half projection, half inversion), Zipf(1.1) over splines."""
    from paper_2504_11498_gb300 import synth
    if kind == "c3":
        ss, sq = synth.surface_set(seed=3 + 1000 * rank)
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
    label = {"c3": "surface_set_1024: 4M projection + 4M inversion queries (bi-degree 2..5)",
             "c5": "ragged_mix: 65,536 cubic curves + 8,192 bicubic surfaces, 64M queries (Zipf 1.1), "
                   "half projection, half inversion per spline kind"}[args.workload]
    if args.impl == "reference":
        if rank != 0:
            return
        cs, cq, ss, sq = build_surface_workload(args.workload, 0)
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
    cs, cq, ss, sq = build_surface_workload(args.workload, rank)
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
    bufs = {name: bspl.QueryBuffers(sg, qi.numel(), dev, learned=name.startswith("curve"))
            for name, _, sg, qi, _ in calls}
    n_step = sum(qi.numel() for _, _, _, qi, _ in calls)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def opts(name, fast, **kw):
        if not fast:
            return bspl.make_options(prec=bspl.FP64, **kw)
        if name.startswith("curve"):
            return bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp, **kw)
        return bspl.make_options(prec=bspl.MIXED, **kw)

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

    clocks = ClockSampler(local)
    clocks.start()
    ms_fast = timed(True, args.steps, args.warmup)
    ms_plain = timed(False, max(2, args.steps // 3), 2)
    per_call = {name: timed(True, max(2, args.steps // 2), 1, only=name) for name, *_ in calls}
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
        step(True)
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
        flops = 12 * (c["grp_tested"] + c["seg_tested"]) + 110 * c["candidates"] + 45 * c["newton32_iters"]
        kern = "learned curve path (k_cull_pairs + pair kernels)"
    t_dom = per_call[dominant] * 1e-3
    roofline = {"bound": "alu", "achieved": flops / t_dom / 1e12, "peak": p32 / 1e12, "unit": "TFLOP/s",
                "frac": flops / t_dom / p32, "traffic": None, "kernel": kern, "call": dominant,
                "ms_per_step": per_call[dominant], "calls_ms_per_step": per_call,
                "peak_source": "FP32 FMA-chain microbenchmark on this GPU (of measured)",
                "note": "counted FP32 flops only (Newton iterations of the surface kernel uncounted): a lower bound"}

    cfg = {"workload": label, "tol_rel_curves": TOL, "tol_rel_surfaces": SURF_TOL,
           "prec": "surfaces mixed" + (", curves learned_mixed" if has_c else ""),
           "l2": "512 MB flush between timed steps", "patches": int(ssegs.total), "decompose_surfaces_ms": dec_s}
    if has_c:
        cfg.update({"segments": int(csegs.total), "decompose_curves_ms": dec_c, "seed_network": train})
    # per call: counting sort (histogram, scan, scatter; the scan is one
    # launch up to 2,048 splines, three above) and the query kernel; the
    # learned curve call 13
    launches = {"c3": 2 * 4, "c5": 2 * 6 + 2 * 13}[args.workload]
    out = {"metric": METRIC, "value": total_q / (ms_fast * 1e-3), "unit": "pts/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_fast, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64 (FP32 search, FP64 finish)" + ("; curves bf16+f32+f64" if has_c else ""),
           "data": "synthetic", "config": cfg,
           "plain_fp64": {"value": total_q / (ms_plain * 1e-3), "ms_per_step": ms_plain},
           "speedup_vs_plain": ms_plain / ms_fast, "accuracy": acc,
           "e2e": {"value": total_q / (ms_e2e * 1e-3), "unit": "pts/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": launches, "roofline": roofline, "clocks": clk, "counters": cnt}
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
