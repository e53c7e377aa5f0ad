"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
synthetic workload (weak scaling, no data-path collective), combine their
step times by a max over ranks and count the units of all ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    cs, qs = bench.build_workload(2, rank, n_curves=8, n_queries=100)
    times = [1.0 + rank, 5.0 - rank]
    (t0, t1), total = bench.combine_over_ranks(times, 200, world, dist)
    out[rank] = (t0, t1, total, float(qs.proj_xyz.sum()), int(cs.n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    r0, r1 = out[0], out[1]
    # both ranks report the slowest rank's times and the job's units
    assert r0[:3] == r1[:3] == (2.0, 5.0, 400)
    # each rank generated its own workload
    assert r0[3] != r1[3] and r0[4] == r1[4] == 8


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    (t,), total = bench.combine_over_ranks([3.5], 10, 1)
    assert t == 3.5 and total == 10
