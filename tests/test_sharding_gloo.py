"""Sharding across ranks (CPU, gloo, world size 2).

Samples are keyed by id, so ranks that take disjoint id ranges and sum their
class counts reproduce the single-range counts exactly.  This is the N > 1
path of bench.py (each rank its own id range); the sums here use the oracle.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, k, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import graphgen as gg
    import oracle as O
    import bench
    g = gg.chung_lu(1500, 10.0, 2.3, 120.0, 4)
    og = O.prepare(g.off, g.col)
    h6 = O.sample_3paths(og, k, 9, rank * k).astype(np.int64)
    h4 = O.sample_centered(og, k, 9, rank * k).astype(np.int64)
    t = torch.from_numpy(np.concatenate([h6, h4]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    mx = bench.reduce_max(float(rank + 1), world, "cpu")
    if rank == 0:
        out.put((t.numpy().tolist(), mx))
    dist.destroy_process_group()


def test_two_rank_shards_sum_to_the_whole_range():
    import graphgen as gg
    import oracle as O
    k = 20000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, k, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.chung_lu(1500, 10.0, 2.3, 120.0, 4)
    og = O.prepare(g.off, g.col)
    want = np.concatenate([O.sample_3paths(og, 2 * k, 9), O.sample_centered(og, 2 * k, 9)])
    assert got == want.astype(np.int64).tolist()
    assert mx == 2.0
