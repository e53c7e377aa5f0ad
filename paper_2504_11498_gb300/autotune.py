"""Autotuner for the query kernels' launch configuration.

Times every candidate configuration on a bounded sample of the caller's
queries, picks the fastest and caches the choice on disk, keyed by GPU name,
spline kind, precision and the workload's exact shape (splines, pieces and
batch size).  Candidates: curves -- grid samples per segment (the sample
tile of a warp step: 32 / S segments), register/occupancy variant and the
FP32 Newton step count; the learned path -- the culling kernel's occupancy
variant and the FP32 step count; surfaces -- the sample tile per patch (8 x 4
or 4 x 4) and the FP32 step count.  A warp always serves 32 queries (one
per lane in the culling), and the work-stealing launches always fill the GPU
(SMs x resident blocks).  Every candidate computes the same result to the
stated tolerance; only the speed differs.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import bspl

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CURVE_CANDIDATES = [dict(samples=s, occupancy=o, fp32_steps=f) for s in (16, 32) for o in (0, 1, 2) for f in (4, 6)]
SURFACE_CANDIDATES = [dict(samples=s, fp32_steps=f) for s in (16, 32) for f in (6, 8)]
_lock = threading.Lock()


def _key(segs, prec, n_q):
    name = torch.cuda.get_device_name()
    kind = "surfaces" if segs.is_surface else "curves"
    return f"{name}|{kind}|prec{prec}|n{int(segs.n)}|seg{int(segs.total)}|q{int(n_q)}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


LEARNED_CANDIDATES = [dict(occupancy=o, fp32_steps=f) for o in (0, 1, 2) for f in (3, 4, 6)]


def time_config(segs, q_idx, q_xyz, prec, cfg, reps=3, invert=False, mlp=None):
    """Mean device time (ms) of one query call with configuration cfg."""
    if segs.is_surface:
        fn = bspl.bspl_invert_surfaces if invert else bspl.bspl_project_surfaces
    else:
        fn = bspl.bspl_invert_curves if invert else bspl.bspl_project_curves
    learned = prec == bspl.LEARNED_MIXED
    bufs = bspl.QueryBuffers(segs, q_idx.numel(), q_xyz.device, learned=learned)
    opts = bspl.make_options(prec=prec, mlp=mlp if learned else None, **cfg)
    fn(segs, q_idx, q_xyz, opts, bufs)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        fn(segs, q_idx, q_xyz, opts, bufs)
    ev[1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps


def tune_curves(segs, q_idx, q_xyz, prec, max_sample=262144, use_cache=True, candidates=None, mlp=None):
    """Best launch configuration for this workload (cached): {samples,
    occupancy} for the grid paths, {occupancy} for the learned path."""
    key = _key(segs, prec, q_idx.numel())
    with _lock:
        db = _load() if use_cache else {}
        if key in db:
            return dict(db[key]["config"])
    n = min(q_idx.numel(), max_sample)
    sel = torch.randperm(q_idx.numel(), device=q_idx.device)[:n]
    qi, qx = q_idx[sel].contiguous(), q_xyz[sel].contiguous()
    results = []
    if candidates is None:
        candidates = LEARNED_CANDIDATES if prec == bspl.LEARNED_MIXED else CURVE_CANDIDATES
    for cfg in candidates:
        results.append((time_config(segs, qi, qx, prec, cfg, mlp=mlp), cfg))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    with _lock:
        db = _load()
        db[key] = {"config": best, "ms": [[r[0], r[1]] for r in results]}
        _store(db)
    return dict(best)


def tune_surfaces(segs, q_idx, q_xyz, prec, max_sample=131072, use_cache=True, candidates=None, mlp=None):
    """Best {samples, fp32_steps} for surface queries of this workload (cached)."""
    return tune_curves(segs, q_idx, q_xyz, prec, max_sample=max_sample, use_cache=use_cache,
                       candidates=candidates or SURFACE_CANDIDATES, mlp=mlp)
