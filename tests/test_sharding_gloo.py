"""Sharding across ranks (CPU, gloo, world size 2).

Samples are keyed by id, so ranks that take contiguous id ranges and sum their
class counts reproduce the single-range counts exactly.  Each rank here takes
its range from ``shard.shard_range`` and sums with ``shard.combine_histograms``
-- the functions bench.py's torchrun branch calls on the GPU (there over NCCL)
-- with the oracle standing in for the per-rank sampling; the combined
histograms must equal the oracle's over the whole range, and rank 0's
estimates from them the oracle's estimates of the whole job.
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


def _graph():
    import graphgen as gg
    return gg.chung_lu(1500, 10.0, 2.3, 120.0, 4)


def _worker(rank, world, port, k3, kc, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    import bench
    from paper_1411_4942_gb300 import shard
    og = O.prepare(*(lambda g: (g.off, g.col))(_graph()))
    f3, n3 = shard.shard_range(k3, rank, world)
    fc, nc = shard.shard_range(kc, rank, world)
    hist = torch.zeros(16, dtype=torch.int64)
    hist[shard.HIST6] = torch.from_numpy(O.sample_3paths(og, n3, 9, f3).astype(np.int64))
    hist[shard.HIST4] = torch.from_numpy(O.sample_centered(og, nc, 9, fc).astype(np.int64))
    shard.combine_histograms(hist)
    mx = bench.reduce_max(float(rank + 1), world, "cpu")
    if rank == 0:
        out.put((hist.numpy().tolist(), mx))
    dist.destroy_process_group()


def test_shard_ranges_partition_the_ids():
    from paper_1411_4942_gb300 import shard
    for k in (0, 1, 7, 1000, 2 ** 27 + 3):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_range(k, r, world) for r in range(world)]
            assert parts[0][0] == 0
            assert all(a[0] + a[1] == b[0] for a, b in zip(parts, parts[1:]))
            assert sum(c for _, c in parts) == k
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def test_combine_without_process_group_is_identity():
    from paper_1411_4942_gb300 import shard
    h = torch.arange(16, dtype=torch.int64)
    assert shard.combine_histograms(h) is h
    assert h.tolist() == list(range(16))
    with pytest.raises(TypeError):
        shard.combine_histograms(torch.zeros(16, dtype=torch.int32))


def test_two_rank_shards_sum_to_the_whole_range():
    import oracle as O
    from paper_1411_4942_gb300 import shard
    k3, kc = 20001, 10001  # odd: the ranks' ranges differ in size
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, k3, kc, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = _graph()
    og = O.prepare(g.off, g.col)
    h6, h4 = O.sample_3paths(og, k3, 9), O.sample_centered(og, kc, 9)
    assert got[shard.HIST6] == h6.astype(np.int64).tolist()
    assert got[shard.HIST4] == h4.astype(np.int64).tolist()
    assert mx == 2.0
    # rank 0's estimates from the combined words are those of the whole job
    c6 = np.array(got[shard.HIST6], dtype=np.uint64)
    c4 = np.array(got[shard.HIST4], dtype=np.uint64)
    _, est, _, _ = O.estimate(og.W, og.Lambda, og.N1, c6, k3, c4, kc)
    _, want, _, _ = O.estimate(og.W, og.Lambda, og.N1, h6, k3, h4, kc)
    assert est.tolist() == want.tolist()
