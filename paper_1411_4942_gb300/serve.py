"""Serving: estimate requests against device-resident graphs, continuously batched.

Requests (graph, k, seed) arrive over time.  The server keeps graphs loaded
(CSR, edge table, prefixes, adjacency structure) inside a device-memory
budget, admits a request once its graph is resident and two histogram slots
are free, and runs iterations: each iteration hands out up to
`iteration_samples` sample ids per sampler, oldest admitted request first (at
most `quantum` to one request), groups the work items by graph so the
resident blocks share a graph's working set, and launches them all in one
batched kernel.  Iterations alternate between streams, so a
request that arrives while earlier work is on the GPU joins the next
iteration and its kernel runs alongside.  A request finishes when the last
iteration holding its samples finishes; its histograms are then read back
and turned into estimates.  Draws are keyed by (seed, sample id), so every
result equals that of the same request run alone.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import pathsample as ps
from .batch import LaunchConfig, SAMPLER_3PATH, SAMPLER_CENTRED, check_skipped, order_by_graph


@dataclasses.dataclass
class EstimateRequest:
    rid: int
    graph: str
    k: int
    seed: int
    arrival: float = 0.0      # seconds after the start of the stream


@dataclasses.dataclass
class Result:
    rid: int
    est: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    hist6: np.ndarray
    hist4: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class GraphPool:
    """Loaded graphs within a byte budget; idle graphs are evicted least
    recently used first when a new one needs room."""

    def __init__(self, sources: dict, budget_bytes: int, max_graphs: int = 256, tuning=None,
                 device=None):
        import torch
        self.sources = sources              # key -> (off, col) host arrays
        self.budget = int(budget_bytes)
        self.tuning = tuning
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.max_graphs = max_graphs
        self.loaded: dict = {}              # key -> ps.Graph
        self.index: dict = {}               # key -> descriptor-table index
        self.refs = collections.Counter()
        self.last_use: dict = {}
        self.free_idx = list(range(max_graphs))[::-1]
        self.used_bytes = 0
        self.loads = 0
        self.evictions = 0
        self.table = torch.empty(ps.ps_batch_table_bytes(max_graphs), dtype=torch.uint8,
                                 device=self.device)
        self._table_dirty = False

    def bytes_for(self, key) -> int:
        off, col = self.sources[key]
        return ps.ps_graph_workspace_bytes(len(off) - 1, len(col), self.tuning)

    def acquire(self, key):
        """Table index of a resident graph (loading it if it fits), else None."""
        if key in self.loaded:
            self.refs[key] += 1
            self.last_use[key] = time.perf_counter()
            return self.index[key]
        need = self.bytes_for(key)
        if need > self.budget:
            raise ValueError(f"graph {key} alone exceeds the device budget")
        while self.used_bytes + need > self.budget or not self.free_idx:
            idle = [k for k in self.loaded if self.refs[k] == 0]
            if not idle:
                return None
            self.evict(min(idle, key=lambda k: self.last_use.get(k, 0.0)))
        off, col = self.sources[key]
        g = ps.Graph(off, col, tuning=self.tuning, device=self.device)
        self.loaded[key] = g
        self.index[key] = self.free_idx.pop()
        self.used_bytes += int(g.workspace.numel())
        self.refs[key] += 1
        self.last_use[key] = time.perf_counter()
        self.loads += 1
        self._table_dirty = True
        return self.index[key]

    def release(self, key):
        self.refs[key] -= 1
        self.last_use[key] = time.perf_counter()

    def evict(self, key):
        g = self.loaded.pop(key)
        self.free_idx.append(self.index.pop(key))
        self.used_bytes -= int(g.workspace.numel())
        g.close()
        self.evictions += 1

    def sync_table(self, stream=None):
        """Write the descriptors of the resident graphs (unused entries repeat
        a resident graph; no item ever names them)."""
        if not self._table_dirty or not self.loaded:
            return
        handles = [None] * self.max_graphs
        any_handle = next(iter(self.loaded.values())).handle
        for key, idx in self.index.items():
            handles[idx] = self.loaded[key].handle
        handles = [h if h is not None else any_handle for h in handles]
        ps._check(ps.ps_batch_prepare(handles, self.table.data_ptr(), stream), "ps_batch_prepare")
        self._table_dirty = False



@dataclasses.dataclass
class _Active:
    req: EstimateRequest
    gidx: int
    slot: int                 # slots 2*slot (3-path) and 2*slot+1 (centred)
    admitted: float
    issued: int = 0           # sample ids issued per sampler
    outstanding: int = 0      # iterations in flight holding its samples


class Server:
    def __init__(self, pool: GraphPool, quantum: int = 1 << 22, max_active: int = 1024,
                 streams: int = 2, cfg: LaunchConfig | None = None, delta: float = 0.01,
                 iteration_samples: int = 1 << 25):
        import torch
        self.pool = pool
        self.quantum = int(quantum)
        # per-iteration cap (sample ids per sampler), filled oldest request first
        self.iteration_samples = int(iteration_samples)
        self.max_active = int(max_active)
        self.cfg = cfg or LaunchConfig(block_size=256, chunk=1 << 16)
        self.delta = delta
        dev = pool.device
        self.streams = [torch.cuda.Stream(dev) for _ in range(streams)]
        self.d_hist = torch.zeros(12 * self.max_active, dtype=torch.int64, device=dev)
        self.counters = [torch.zeros(2, dtype=torch.int32, device=dev) for _ in self.streams]
        # items the batched kernel skipped, summed per launch stream (each
        # stream adds its own launch's count after the kernel)
        self.skipped = torch.zeros(len(self.streams), dtype=torch.int64, device=dev)
        self.free_slots = list(range(self.max_active))[::-1]
        self.tuning = self.cfg.tuning()
        self.iterations = 0
        self.items_launched = 0

    def warmup(self):
        """Runs each device operation of an iteration once, untimed: the first
        use of a torch operation in a process loads its kernels, which took
        seconds on a fresh host and stalled the first requests behind it."""
        import torch
        self._zero_slots([0])
        sel = torch.tensor([0], dtype=torch.int64, device=self.pool.device)
        torch.cat([self.d_hist.view(self.max_active, 12).index_select(0, sel).flatten(),
                   self.skipped]).cpu()
        self.skipped[0:1] += self.counters[0][1:2]
        torch.from_numpy(np.zeros(16, dtype=np.uint8)).pin_memory().to(self.pool.device, non_blocking=True)
        torch.cuda.Event().record(self.streams[0])
        torch.cuda.synchronize(self.pool.device)

    def _zero_slots(self, slots):
        """Clears reused histogram slots on the current stream; every launch
        stream waits on that stream before its kernel."""
        import torch
        idx = torch.tensor(slots, dtype=torch.int64, device=self.pool.device)
        self.d_hist.view(self.max_active, 12).index_fill_(0, idx, 0)

    def _launch(self, si, items: np.ndarray):
        import torch
        s = self.streams[si]
        s.wait_stream(torch.cuda.current_stream(self.pool.device))
        with torch.cuda.stream(s):
            host = torch.from_numpy(items.view(np.uint8)).pin_memory()
            d_items = host.to(self.pool.device, non_blocking=True)
            rc = ps.ps_batch_sample_prepared(self.pool.table.data_ptr(), self.pool.max_graphs,
                                             d_items.data_ptr(), int(items.shape[0]),
                                             self.d_hist.data_ptr(), self.counters[si].data_ptr(),
                                             self.tuning, s)
            ps._check(rc, "ps_batch_sample_prepared")
            self.skipped[si:si + 1] += self.counters[si][1:2]
            ev = torch.cuda.Event()
            ev.record(s)
        self.iterations += 1
        self.items_launched += int(items.shape[0])
        return ev, (host, d_items)

    def run(self, requests, realtime: bool = True, idle_sleep: float = 50e-6):
        """Serve `requests`.  realtime=True replays their arrival times;
        False treats every request as arrived at the start (throughput).
        Returns (results, report); latencies are wall-clock seconds."""
        import torch
        self.warmup()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active: dict = {}
        inflight = collections.deque()      # (event, rids, keepalive)
        results = []
        t0 = time.perf_counter()
        turn = 0
        total_samples = 0
        while pending or waiting or active or inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.popleft())
            # admission: graph resident within the budget and a free slot pair
            admitted = []
            while waiting and self.free_slots:
                req = waiting[0]
                gidx = self.pool.acquire(req.graph)
                if gidx is None:
                    break
                waiting.popleft()
                slot = self.free_slots.pop()
                admitted.append(slot)
                active[req.rid] = _Active(req, gidx, slot, now if realtime else 0.0)
            if admitted:
                self._zero_slots(admitted)
            # retire finished iterations
            while inflight and inflight[0][0].query():
                _, rids, _ = inflight.popleft()
                done = []
                for rid in rids:
                    a = active[rid]
                    a.outstanding -= 1
                    if a.outstanding == 0 and a.issued >= a.req.k:
                        done.append(a)
                if done:
                    hist = self.d_hist.view(self.max_active, 12)
                    sel = torch.tensor([a.slot for a in done], dtype=torch.int64,
                                       device=self.pool.device)
                    both = torch.cat([hist.index_select(0, sel).flatten(), self.skipped]).cpu().numpy()
                    check_skipped(int(both[-len(self.streams):].sum()))
                    rows = both[:-len(self.streams)].reshape(-1, 12).astype(np.uint64)
                    t_fin = time.perf_counter() - t0
                    for a, row in zip(done, rows):
                        g = self.pool.loaded[a.req.graph]
                        h6, h4 = row[:6], row[6:10]
                        rc, est, lo, hi = ps.ps_estimate(g.stats, h6, a.req.k, h4, a.req.k, self.delta)
                        arrival = a.req.arrival if realtime else 0.0
                        results.append(Result(a.req.rid, est, lo, hi, h6, h4, arrival,
                                              a.admitted, t_fin))
                        del active[a.req.rid]
                        self.free_slots.append(a.slot)
                        self.pool.release(a.req.graph)
            # launch the next iteration
            work = [a for a in active.values() if a.issued < a.req.k]
            if work and len(inflight) < len(self.streams):
                self.pool.sync_table()
                recs = []
                rids = []
                budget = self.iteration_samples
                for a in work:  # admission order: the oldest requests first
                    if budget <= 0:
                        break
                    n_new = min(self.quantum, a.req.k - a.issued, budget)
                    budget -= n_new
                    for sampler in (SAMPLER_3PATH, SAMPLER_CENTRED):
                        done_ = 0
                        while done_ < n_new:
                            c = min(self.cfg.chunk, n_new - done_)
                            recs.append((a.issued + done_, a.req.seed, c, a.gidx,
                                         2 * a.slot + sampler, sampler))
                            done_ += c
                    a.issued += n_new
                    a.outstanding += 1
                    total_samples += 2 * n_new
                    rids.append(a.req.rid)
                items = order_by_graph(np.array(recs, dtype=ps.WORK_DTYPE))
                ev, keep = self._launch(turn % len(self.streams), items)
                turn += 1
                inflight.append((ev, rids, keep))
                continue
            if inflight:
                if not pending or pending[0].arrival > now + idle_sleep:
                    time.sleep(idle_sleep)
            elif pending:
                gap = pending[0].arrival - now
                if gap > 0:
                    time.sleep(min(gap, 1e-3))
        check_skipped(int(self.skipped.sum().item()))
        makespan = (max(r.finished for r in results)) if results else 0.0
        lat = np.array([r.latency for r in results]) if results else np.zeros(1)
        report = {
            "requests": len(results), "samples": total_samples, "makespan_s": makespan,
            "samples_per_s": total_samples / makespan if makespan > 0 else None,
            "estimates_per_s": len(results) / makespan if makespan > 0 else None,
            "latency_p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "latency_p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "latency_max_ms": 1e3 * float(lat.max()),
            "iterations": self.iterations, "items": self.items_launched,
            "graph_loads": self.pool.loads, "graph_evictions": self.pool.evictions,
            "resident_bytes": self.pool.used_bytes,
        }
        return results, report


def poisson_requests(rs: np.random.Generator, graph_keys, n: int, rate: float,
                     log2_k=(14, 22)) -> list:
    """n requests with exponential inter-arrival gaps (mean 1/rate), a
    uniformly chosen graph, k = 2^U{log2_k} and their own seeds."""
    gaps = rs.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    out = []
    for i in range(n):
        out.append(EstimateRequest(i, graph_keys[int(rs.integers(0, len(graph_keys)))],
                                   1 << int(rs.integers(log2_k[0], log2_k[1] + 1)),
                                   int(rs.integers(1, 2 ** 63)), float(t[i])))
    return out


def run_sequential(pool: GraphPool, requests, delta: float = 0.01):
    """Baseline: each request alone with plain calls, one after another."""
    import torch
    results = []
    t0 = time.perf_counter()
    hist = torch.zeros(16, dtype=torch.int64, device=pool.device)
    samples = 0
    for req in requests:
        pool.acquire(req.graph)
        g = pool.loaded[req.graph]
        hist.zero_()
        ps._check(ps.ps_sample_3paths(g.handle, req.k, req.seed, 0, hist.data_ptr()), "3paths",
                  (ps.PS_OK, ps.PS_NO_PATHS))
        ps._check(ps.ps_sample_centered(g.handle, req.k, req.seed, 0, hist.data_ptr() + 64),
                  "centred", (ps.PS_OK, ps.PS_NO_PATHS))
        h = hist.cpu().numpy().astype(np.uint64)
        rc, est, lo, hi = ps.ps_estimate(g.stats, h[:6], req.k, h[8:12], req.k, delta)
        pool.release(req.graph)
        samples += 2 * req.k
        results.append((req.rid, h[:6].copy(), h[8:12].copy(), est))
    dt = time.perf_counter() - t0
    return results, {"samples_per_s": samples / dt, "seconds": dt, "estimates_per_s": len(requests) / dt}
