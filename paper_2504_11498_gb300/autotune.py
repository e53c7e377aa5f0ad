"""Autotuner for the query kernels' launch configuration.

Times every candidate configuration (grid samples per segment, register /
occupancy variant) on a bounded sample of the caller's queries, picks the
fastest and caches the choice on disk, keyed by GPU name, precision and the
workload's shape (splines, segments and batch size, each rounded to a power
of two).  Every candidate computes the same result to the stated tolerance;
only the speed differs.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import bspl

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CURVE_CANDIDATES = [dict(samples=s, occupancy=o) for s in (16, 32) for o in (0, 1, 2)]
_lock = threading.Lock()


def _bucket(x: int) -> int:
    return 1 << max(0, int(x) - 1).bit_length()


def _key(segs, prec, n_q):
    name = torch.cuda.get_device_name()
    return f"{name}|curves|prec{prec}|n{_bucket(segs.n)}|seg{_bucket(segs.total)}|q{_bucket(n_q)}"


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


LEARNED_CANDIDATES = [dict(occupancy=o) for o in (0, 1, 2)]


def time_config(segs, q_idx, q_xyz, prec, cfg, reps=3, invert=False, mlp=None):
    """Mean device time (ms) of one query call with configuration cfg."""
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
