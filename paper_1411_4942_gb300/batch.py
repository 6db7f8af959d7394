"""Batched sampling over many loaded graphs in one persistent launch.

A batch is a list of requests (graph, sampler, k, seed, first id); it is cut
into work items of at most `chunk` sample ids, written to a device queue, and
run by ps_batch_sample_prepared: resident blocks take items from the queue
and add each item's class counts to its request's histogram slot.  Because
draws are keyed by (seed, sample id), every request's histogram equals the
one the plain per-graph calls produce.  Launches can be captured in a CUDA
graph and replayed.  The autotuner picks the launch (block size, samples per
thread, samples per item, resident blocks per SM) and, per graph-size bucket,
the hub-bitmap rows (how many, and from which degree) by timing candidates;
results never depend on the choice.
"""
from __future__ import annotations

import dataclasses
import itertools
import time

import numpy as np

from . import pathsample as ps

SAMPLER_3PATH, SAMPLER_CENTRED = 0, 1


@dataclasses.dataclass
class Request:
    graph: int          # index into the GraphSet
    sampler: int        # 0: Alg. 1 (3-path), 1: Alg. 3 (centred)
    k: int
    seed: int
    first_id: int = 0
    slot: int = -1      # histogram slot (6 uint64); assigned by plan_items when -1


# graphs with at least this many edges can have their large requests taken
# in draw order (their records and rows no longer stay in L2)
ORDERED_MIN_EDGES = 1 << 20
NEVER = 1 << 62


@dataclasses.dataclass
class LaunchConfig:
    block_size: int = 256
    chunk: int = 1 << 16
    blocks_per_sm: int = 0
    samples_per_thread: int = 1
    # requests of at least this many samples on graphs of >= ORDERED_MIN_EDGES
    # edges run through the draw-ordered samplers inside the same step (same
    # counts); the queue kernel takes the rest
    ordered_min_k: int = NEVER

    def tuning(self) -> ps.PsTuning:
        return ps.make_tuning(block_size=self.block_size, blocks_per_sm=self.blocks_per_sm,
                              samples_per_thread=self.samples_per_thread)


class GraphSet:
    """Loaded graphs plus their descriptor table on the device."""

    def __init__(self, graphs, stream=None):
        import torch
        self.graphs = list(graphs)
        self.device = self.graphs[0].device
        nb = ps.ps_batch_table_bytes(len(self.graphs))
        self.table = torch.empty(nb, dtype=torch.uint8, device=self.device)
        rc = ps.ps_batch_prepare([g.handle for g in self.graphs], self.table.data_ptr(), stream)
        ps._check(rc, "ps_batch_prepare")

    def __len__(self):
        return len(self.graphs)

    @property
    def workspace_bytes(self) -> int:
        return sum(int(g.workspace.numel()) for g in self.graphs)


def order_by_graph(items: np.ndarray) -> np.ndarray:
    """Items grouped by graph, graphs with the most work first.  Resident
    blocks take items in this order, so at any moment they share one graph's
    working set (which then stays in L2) and the small graphs form the tail."""
    if items.size == 0:
        return items
    g = items["graph"].astype(np.int64)
    work = np.bincount(g, weights=items["count"].astype(np.float64))
    return items[np.lexsort((items["first_id"], items["sampler"], g, -work[g]))]


def plan_items(requests, chunk: int) -> tuple[np.ndarray, int]:
    """Work items for the requests (grouped by graph), and the number of slots."""
    slots = 0
    for r in requests:
        if r.slot < 0:
            r.slot = slots
        slots = max(slots, r.slot + 1)
    recs = []
    for r in requests:
        done = 0
        while done < r.k:
            c = min(chunk, r.k - done)
            recs.append((r.first_id + done, r.seed, c, r.graph, r.slot, r.sampler))
            done += c
    items = np.array(recs, dtype=ps.WORK_DTYPE) if recs else np.zeros(0, dtype=ps.WORK_DTYPE)
    return order_by_graph(items), slots


class BatchRunner:
    """Device buffers for one batch and its launch (eager or CUDA graph)."""

    def __init__(self, gset: GraphSet, requests, cfg: LaunchConfig, stream=None):
        import torch
        self.gset, self.cfg = gset, cfg
        self.stream = stream
        requests = list(requests)
        plan_items(requests, cfg.chunk)  # assigns slots
        self.ordered = [r for r in requests if r.k >= cfg.ordered_min_k and
                        int(gset.graphs[r.graph].stats.m) >= ORDERED_MIN_EDGES]
        big = {id(r) for r in self.ordered}
        items, self.slots = plan_items([r for r in requests if id(r) not in big], cfg.chunk)
        self.slots = max([self.slots] + [r.slot + 1 for r in self.ordered])
        self.n_items = int(items.shape[0])
        dev = gset.device
        self.d_items = torch.from_numpy(items.view(np.uint8).copy()).to(dev)
        self.d_hist = torch.zeros(6 * max(self.slots, 1), dtype=torch.int64, device=dev)
        self.d_counter = torch.zeros(2, dtype=torch.int32, device=dev)
        self.tuning = cfg.tuning()
        self.graph = None
        # scratch of the draw-ordered calls: one chunk of the largest of them
        self.d_order = None
        if self.ordered:
            k_max = min(max(r.k for r in self.ordered), 1 << 24)
            self.d_order = torch.empty(ps.ps_ordered_scratch_bytes(k_max), dtype=torch.uint8, device=dev)

    def launch(self, zero: bool = True):
        if zero:
            self.d_hist.zero_()
        if self.n_items:
            rc = ps.ps_batch_sample_prepared(self.gset.table.data_ptr(), len(self.gset),
                                             self.d_items.data_ptr(), self.n_items,
                                             self.d_hist.data_ptr(), self.d_counter.data_ptr(),
                                             self.tuning, self.stream)
            ps._check(rc, "ps_batch_sample_prepared")
        for r in self.ordered:
            fn = ps.ps_sample_3paths_ordered if r.sampler == SAMPLER_3PATH else ps.ps_sample_centered_ordered
            rc = fn(self.gset.graphs[r.graph].handle, r.k, r.seed, r.first_id, self.d_hist.data_ptr() + 48 * r.slot,
                    self.d_order.data_ptr(), self.d_order.numel(), self.stream)
            ps._check(rc, "draw-ordered sample", (ps.PS_OK, ps.PS_NO_PATHS))

    def capture(self):
        """Record zeroing + the batched launch in a CUDA graph."""
        import torch
        s = torch.cuda.Stream(self.gset.device)
        s.wait_stream(torch.cuda.current_stream(self.gset.device))
        with torch.cuda.stream(s):
            self.launch()  # warm-up outside capture (occupancy query, lazy loading)
        torch.cuda.current_stream(self.gset.device).wait_stream(s)
        torch.cuda.synchronize(self.gset.device)
        g = torch.cuda.CUDAGraph()
        saved = self.stream
        self.stream = None  # capture on torch's current (capturing) stream
        with torch.cuda.graph(g):
            self.launch()
        self.stream = saved
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def histograms(self) -> np.ndarray:
        """The slots' histograms after the last launch; raises if that launch
        skipped items (a graph whose adjacency variant differs from the one
        the descriptor table records: its samples would be missing)."""
        import torch
        both = torch.cat([self.d_hist, self.d_counter.to(torch.int64)]).cpu().numpy()
        check_skipped(int(both[-1]))
        return both[:-2].reshape(-1, 6).astype(np.uint64)


def check_skipped(skipped: int):
    """The batched kernel counts the items it skipped (counter word 1);
    any skipped item means histograms that do not sum to their k."""
    if skipped:
        raise RuntimeError(f"the batched launch skipped {skipped} work items: the descriptor "
                           "table's adjacency variant does not match a graph's")


def run_plain(gset: GraphSet, requests, stream=None):
    """The same requests as ordinary per-graph calls (two launches per graph)."""
    import torch
    slots = max(r.slot for r in requests) + 1
    hist = torch.zeros(6 * slots, dtype=torch.int64, device=gset.device)
    for r in requests:
        g = gset.graphs[r.graph]
        fn = ps.ps_sample_3paths if r.sampler == SAMPLER_3PATH else ps.ps_sample_centered
        rc = fn(g.handle, r.k, r.seed, r.first_id, hist.data_ptr() + 48 * r.slot, stream)
        ps._check(rc, "plain sample", (ps.PS_OK, ps.PS_NO_PATHS))
    return hist


def time_device(fn, reps: int = 3, warmup: int = 1) -> float:
    """Best-of-reps milliseconds of fn() measured with CUDA events."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


class Autotuner:
    """Chooses launch parameters by timing candidates on (a slice of) the
    real batch; caches the choice per device and graph-size bucket."""

    # hub-bitmap settings tried per graph-size bucket: (rows, smallest degree);
    # rows -1 = none, (0, 0) = the library's defaults (up to 8192 rows within
    # 48 bytes per edge, degree >= 64)
    HUB_CHOICES = ((-1, 0), (0, 0), (1024, 64), (1024, 16), (4096, 16))
    # graph-size buckets by edges: below 2^17, below 2^20, the rest
    SIZE_EDGES = (1 << 17, 1 << 20)
    # smallest request taken in draw order (on graphs of >= ORDERED_MIN_EDGES)
    ORDERED_MIN_K = (NEVER, 1 << 21, 1 << 19)

    def __init__(self, block_sizes=(128, 256, 512), chunks=(1 << 12, 1 << 13, 1 << 14, 1 << 16, 1 << 18),
                 blocks_per_sm=(0,), samples_per_thread=(1, 2)):
        self.candidates = [LaunchConfig(b, c, p, t) for b, c, p, t in
                           itertools.product(block_sizes, chunks, blocks_per_sm, samples_per_thread)]
        self.cache: dict = {}
        self.hub_choice: dict = {}   # size bucket -> (rows, smallest degree)
        self.log: list = []

    @classmethod
    def size_bucket(cls, m: int) -> int:
        return sum(m >= e for e in cls.SIZE_EDGES)

    def graph_tuning(self, m: int) -> ps.PsTuning:
        """The load-time tuning of a graph with m edges: its size bucket's hub
        rows (the library's defaults before tune_hubs)."""
        rows, deg = self.hub_choice.get(self.size_bucket(m), (0, 0))
        return ps.make_tuning(hub_count=rows, hub_min_degree=deg)

    def tune_hubs(self, hosts, k: int = 1 << 20, seed: int = 1):
        """Hub rows per size bucket: the largest graph of each bucket is loaded
        with every HUB_CHOICES setting and both samplers timed on it."""
        reps = {}
        for h in hosts:
            b = self.size_bucket(h.m)
            if b not in reps or h.m > reps[b].m:
                reps[b] = h
        for b, h in sorted(reps.items()):
            best, best_ms = None, float("inf")
            for rows, deg in self.HUB_CHOICES:
                G = ps.Graph(h.off, h.col, tuning=ps.make_tuning(hub_count=rows, hub_min_degree=deg))

                def both():
                    hist = G.new_hist()
                    G.sample_3paths(k, seed, 0, hist)
                    G.sample_centered(k, seed, 0, hist)
                ms = time_device(both, reps=2)
                self.log.append({"size_bucket": b, "edges": int(h.m), "hub_rows": rows,
                                 "hub_min_degree": deg, "hubs": int(G.stats.hubs), "ms": ms})
                G.close()
                if ms < best_ms:
                    best, best_ms = (rows, deg), ms
            self.hub_choice[b] = best
        return dict(self.hub_choice)

    @staticmethod
    def bucket(gset: GraphSet) -> tuple:
        import torch
        edges = sum(int(g.stats.m) for g in gset.graphs)
        return (torch.cuda.get_device_name(gset.device), len(gset), int(np.log2(max(edges, 1))))

    def tune_launch(self, gset: GraphSet, requests, budget_samples: int = 1 << 26) -> LaunchConfig:
        key = self.bucket(gset)
        if key in self.cache:
            return self.cache[key]
        # a proportional slice of every request keeps the mix of graphs and samplers
        total = sum(r.k for r in requests)
        frac = min(1.0, budget_samples / max(total, 1))
        trial = [dataclasses.replace(r, k=max(1, int(r.k * frac)), slot=i)
                 for i, r in enumerate(requests)]
        best, best_ms = None, float("inf")
        for cfg in self.candidates:
            runner = BatchRunner(gset, trial, cfg)
            ms = time_device(runner.launch, reps=2)
            self.log.append({"cfg": dataclasses.asdict(cfg), "ms": ms})
            if ms < best_ms:
                best, best_ms = cfg, ms
        # which requests go in draw order: timed on the whole batch
        best_ms = float("inf")
        for min_k in self.ORDERED_MIN_K:
            cfg = dataclasses.replace(best, ordered_min_k=min_k)
            runner = BatchRunner(gset, [dataclasses.replace(r) for r in requests], cfg)
            ms = time_device(runner.launch, reps=2)
            self.log.append({"cfg": dataclasses.asdict(cfg), "ms": ms, "whole_batch": True})
            if ms < best_ms:
                choice, best_ms = cfg, ms
        self.cache[key] = choice
        return choice

    def tune_graph_variant(self, off, col, k: int = 1 << 20, seed: int = 1,
                           hub_counts=(256, 1024)) -> ps.PsTuning:
        """Adjacency variant (and hub-bitmap row count for the search variant)
        for graphs like this one, by timing both samplers."""
        choices = [ps.make_tuning(adjacency=ps.ADJ_HASH), ps.make_tuning(adjacency=ps.ADJ_VTAB)]
        choices += [ps.make_tuning(adjacency=ps.ADJ_SEARCH, hub_count=h) for h in hub_counts]
        best, best_ms = None, float("inf")
        for t in choices:
            G = ps.Graph(off, col, tuning=t)

            def both():
                h = G.new_hist()
                G.sample_3paths(k, seed, 0, h)
                G.sample_centered(k, seed, 0, h)
            ms = time_device(both, reps=2)
            self.log.append({"adjacency": int(t.adjacency), "hub_count": int(t.hub_count), "ms": ms})
            G.close()
            if ms < best_ms:
                best, best_ms = t, ms
        return best


def random_requests(rs: np.random.Generator, n_graphs: int, log2_k=(16, 22), both=True):
    """One 3-path and one centred request per graph, k = 2^U{log2_k}, own seeds."""
    reqs = []
    for gi in range(n_graphs):
        k = 1 << int(rs.integers(log2_k[0], log2_k[1] + 1))
        seed = int(rs.integers(1, 2 ** 63))
        reqs.append(Request(gi, SAMPLER_3PATH, k, seed))
        if both:
            reqs.append(Request(gi, SAMPLER_CENTRED, k, seed))
    for i, r in enumerate(reqs):
        r.slot = i
    return reqs


def now() -> float:
    return time.perf_counter()
