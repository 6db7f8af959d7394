"""Sharding of the sampling path over several ranks (one GPU each).

The samples of Alg. 1 and Alg. 3 are independent draws (Claim 3.1; the proof
of Theorem 3.4 treats them as i.i.d.), and the library derives every draw
from (seed, sample id) alone.  So a job of k samples splits into contiguous
id ranges, one per rank, each rank sampling its range on its own replica of
the graph, and the class counts of the whole job are the integer sums of the
ranks' counts: one all-reduce of the 10 histogram words (6 of Alg. 2's
classes, 4 of Alg. 4's), exact because it is an integer sum.

``combine_histograms`` is that all-reduce.  It runs on whatever backend the
process group has: NCCL over CUDA tensors on GPUs, gloo over CPU tensors in
the CPU tests.  The histograms are uint64 in the library and int64 in torch;
two's-complement addition gives the same bits as unsigned addition, so the
sum is exact for every count below 2^64.
"""
from __future__ import annotations

# layout of one rank's histogram words in a 16-word tensor: Alg. 2's six
# classes at 0..5, Alg. 4's four at 8..11 (the library's two outputs)
HIST6 = slice(0, 6)
HIST4 = slice(8, 12)


def shard_range(k: int, rank: int, world: int) -> tuple[int, int]:
    """Sample ids [first, first + count) of `rank` when ids [0, k) are split
    into `world` contiguous ranges whose sizes differ by at most one."""
    if world <= 0 or not 0 <= rank < world or k < 0:
        raise ValueError(f"bad shard: k={k} rank={rank} world={world}")
    base, extra = divmod(k, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def combine_histograms(hist, group=None):
    """Sums `hist` (a torch int64 tensor of histogram words, on the device the
    process group's backend serves) over all ranks of `group`, in place, and
    returns it.  With one rank (or no process group) it returns `hist`
    unchanged."""
    import torch
    import torch.distributed as dist

    if hist.dtype != torch.int64:
        raise TypeError("histogram words are int64 (the uint64 counts' bits)")
    if not dist.is_available() or not dist.is_initialized():
        return hist
    if dist.get_world_size(group) == 1:
        return hist
    dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    return hist
