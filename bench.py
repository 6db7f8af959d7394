#!/usr/bin/env python3
"""Benchmark of the path-sampling hot path on GB300.

One step = the whole path over one synthetic graph resident in HBM:
validation + degree-order relabel + sorted rows + edge table (ps_load_csr),
tau / lambda prefixes + guide tables + hub bitmaps (ps_tau_prefix), k3
samples of Alg. 1 and kc samples of Alg. 3 taken in edge-draw order
(ps_sample_3paths_ordered / ps_sample_centered_ordered: the same counts as
ps_sample_3paths / ps_sample_centered), the histograms read back and the
estimates with error bars (ps_estimate).  value = (k3 + kc) samples per
second of step time, timed with CUDA events on the launching stream, L2
flushed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Under torchrun each rank runs the same workload on its own GPU with its own
range of sample ids (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3-path samples/s (plain vs batched/served) at bit-exact histograms; HBM roofline %"
UNIT = "samples/s"
SECTOR = 32
# Algorithmic bytes per sample (the paper's O(1) cost model of Theorem 3.5,
# one 32-byte sector per random access): 3-path = edge draw, edge record,
# both endpoint offsets, the two neighbour reads and three adjacency lookups
BYTES_3PATH = 9 * SECTOR
# samples per chunk of the draw-ordered samplers
ORDER_CHUNK = 1 << 24


def workloads():
    import graphgen as gg
    return {
        "rmat20": dict(
            make=gg.rmat20, k3=1 << 24, kc=1 << 24, seed=11,
            desc=("R-MAT scale 20, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), graph seed "
                  "11, symmetrised and deduplicated; k=2^24 3-path + 2^24 centred samples, "
                  "Philox seed 11")),
        "chung_lu_5k": dict(
            make=gg.chung_lu_5k, k3=1_000_000, kc=1_000_000, seed=7,
            desc=("Chung-Lu n=5,000, mean degree 20, exponent 2.5, max weight 500, graph seed 1; "
                  "k=10^6 3-path + 10^6 centred samples, Philox seed 7")),
        "social3m": dict(
            make=gg.social_chung_lu_3m, k3=1 << 27, kc=1 << 26, seed=3,
            desc=("social-network-shaped Chung-Lu n=3,000,000, exponent 2.1, max weight 33,000, "
                  "mean weight 78 (~117M edges), graph seed 3; k=2^27 3-path + 2^26 centred "
                  "samples, Philox seed 3")),
    }


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_tag() -> str:
    h = hashlib.sha1()
    for name in ("ps_sample.cuh", "ps_device.cuh", "ps_sample.cu", "ps_order.cu"):
        with open(os.path.join(ROOT, "paper_1411_4942_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(workload: str):
    """DRAM bytes of one 3-path sampler call (its draw sort and sampling
    kernels) from the committed ncu summary, when it was taken on the current
    kernel source."""
    path = os.path.join(ROOT, "profiles", f"ncu_k_sample_3path_{workload}.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    tag = re.search(r"kernel_source_tag:\s*(\w+)", text)
    val = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not tag or not val or tag.group(1) != kernel_source_tag():
        return None
    return float(val.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- distributed

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ CPU baseline

def oracle_rate(g, wl, slice_k: int, repeats: int = 1):
    """The oracle (plain C, all host cores for the sampling loops) on a bounded
    sample of the workload: the full prepare once, then `slice_k` sample ids
    of each sampler, scaled linearly to the workload's k3 and kc."""
    import oracle as O
    threads = max(1, O.max_threads())
    t0 = time.perf_counter()
    og = O.prepare(g.off, g.col)
    t_prep = time.perf_counter() - t0
    t3 = tc = 0.0
    for r in range(repeats):
        t0 = time.perf_counter()
        O.sample_3paths(og, slice_k, wl["seed"], r * slice_k, threads=threads)
        t3 += time.perf_counter() - t0
        t0 = time.perf_counter()
        O.sample_centered(og, slice_k, wl["seed"], r * slice_k, threads=threads)
        tc += time.perf_counter() - t0
    t3 /= repeats
    tc /= repeats
    total = t_prep + t3 * wl["k3"] / slice_k + tc * wl["kc"] / slice_k
    return {
        "value": (wl["k3"] + wl["kc"]) / total, "unit": UNIT, "cores": threads, "kind": "oracle",
        "sample": (f"oracle prepare (validate, relabel, edge table, prefixes) on the full graph "
                   f"once ({t_prep:.2f} s) + {slice_k} ids of each sampler on {threads} threads "
                   f"({t3:.3f} s, {tc:.3f} s), scaled linearly to k3={wl['k3']}, kc={wl['kc']}"),
        "seconds_full_workload": total,
    }


# --------------------------------------------------------------- GPU arm

def run_cuda(args):
    import torch
    from paper_1411_4942_gb300 import pathsample as ps

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, "nccl")
    wl = workloads()[args.workload]
    g = wl["make"]()
    k3, kc, seed = wl["k3"], wl["kc"], wl["seed"]
    first3 = rank * k3  # weak scaling: every rank its own id range
    firstc = rank * kc
    ps.load_library()

    stream = torch.cuda.Stream(device)
    sp = stream.cuda_stream
    with torch.cuda.stream(stream):
        d_off = torch.as_tensor(g.off).to(device)
        d_col = torch.as_tensor(g.col).to(device)
        nb = ps.ps_graph_workspace_bytes(g.n, g.nnz)
        ws = torch.empty(nb, dtype=torch.uint8, device=device)
        hist = torch.zeros(16, dtype=torch.int64, device=device)
        # scratch of the draw-ordered samplers: one chunk of max(k3, kc) samples
        osb = ps.ps_ordered_scratch_bytes(min(max(k3, kc, 1), ORDER_CHUNK))
        oscr = torch.empty(osb, dtype=torch.uint8, device=device)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)]
              for _ in range(args.steps + args.warmup)]
        last = {}

        def step(i):
            e = ev[i]
            e[0].record(stream)
            rc, h = ps.ps_load_csr(g.n, g.nnz, d_off.data_ptr(), d_col.data_ptr(), ws.data_ptr(), nb,
                                   None, sp)
            ps._check(rc, "ps_load_csr")
            rc, st = ps.ps_tau_prefix(h, sp)
            ps._check(rc, "ps_tau_prefix", (ps.PS_OK, ps.PS_NO_PATHS))
            e[1].record(stream)
            hist.zero_()
            ps._check(ps.ps_sample_3paths_ordered(h, k3, seed, first3, hist.data_ptr(),
                                                  oscr.data_ptr(), osb, sp),
                      "ps_sample_3paths_ordered", (ps.PS_OK, ps.PS_NO_PATHS))
            e[2].record(stream)
            ps._check(ps.ps_sample_centered_ordered(h, kc, seed, firstc, hist.data_ptr() + 64,
                                                    oscr.data_ptr(), osb, sp),
                      "ps_sample_centered_ordered", (ps.PS_OK, ps.PS_NO_PATHS))
            e[3].record(stream)
            hh = hist.cpu().numpy().astype(np.uint64)
            rc, est, lo, hi = ps.ps_estimate(st, hh[:6], k3, hh[8:12], kc, 0.01)
            e[4].record(stream)
            ps.ps_graph_free(h)
            last.update(stats=st, hist6=hh[:6].copy(), hist4=hh[8:12].copy(), est=est, lo=lo, hi=hi)

        for i in range(args.warmup):
            flush.zero_()
            step(i)
        torch.cuda.synchronize(device)
        barrier(world)
        torch.cuda.synchronize(device)
        clocks = ClockSampler(local)
        clocks.start()
        launches0 = ps.ps_kernel_launches()
        t_wall = time.perf_counter()
        for i in range(args.warmup, args.warmup + args.steps):
            flush.zero_()
            step(i)
        torch.cuda.synchronize(device)
        t_wall = time.perf_counter() - t_wall
        launches = ps.ps_kernel_launches() - launches0
        barrier(world)
        torch.cuda.synchronize(device)
        clk = clocks.stop()

    timed = ev[args.warmup:]
    step_ms = [e[0].elapsed_time(e[4]) for e in timed]
    prep_ms = [e[0].elapsed_time(e[1]) for e in timed]
    s3_ms = [e[1].elapsed_time(e[2]) for e in timed]
    sc_ms = [e[2].elapsed_time(e[3]) for e in timed]
    est_ms = [e[3].elapsed_time(e[4]) for e in timed]
    total_ms = reduce_max(sum(step_ms), world, device)
    value = world * args.steps * (k3 + kc) / (total_ms / 1e3)
    avg3 = statistics.mean(s3_ms)
    avgc = statistics.mean(sc_ms)
    peak, peak_kind = measured_peak_hbm()
    achieved = BYTES_3PATH * k3 / (avg3 / 1e3) / 1e9
    h4 = last["hist4"]
    f_c = 1.0 - float(h4[0]) / kc if kc else 0.0
    bytes_c = (7 + 2 * f_c) * SECTOR
    achieved_c = bytes_c * kc / (avgc / 1e3) / 1e9
    traffic = ncu_traffic(args.workload)

    # end to end through the host-buffer call (inputs copied from pinned memory every step)
    e2e = None
    if not args.no_e2e:
        h_off = torch.as_tensor(g.off).pin_memory()
        h_col = torch.as_tensor(g.col).pin_memory()
        nb2 = ps.ps_end_to_end_workspace_bytes(g.n, g.nnz) + osb  # + draw-order scratch
        del ws
        ws2 = torch.empty(nb2, dtype=torch.uint8, device=device)
        times = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            rc, est, lo, hi, h6, h4e, st2 = ps.ps_count_motifs_host(
                h_off, h_col, k3, kc, seed, 0.01, ws2.data_ptr(), nb2, None, sp)
            t1 = time.perf_counter()
            ps._check(rc, "ps_count_motifs_host", (ps.PS_OK, ps.PS_NO_PATHS))
            if i >= args.warmup:
                times.append(t1 - t0)
        e2e_s = reduce_max(sum(times), world, device)
        h2d = (g.n + 1) * 8 + g.nnz * 4
        d2h = 16 * 8 + 4 * 64 * 8  # histograms + the four status-block reads
        e2e = {"value": world * args.steps * (k3 + kc) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * e2e_s / args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(g, wl, args.cpu_slice)
        cpu.pop("seconds_full_workload", None)

    if rank == 0:
        st = last["stats"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}", "n": g.n, "m": g.m,
                       "W": int(st.W), "Lambda": int(st.Lambda), "d_max": int(st.d_max),
                       "k3": k3, "kc": kc, "samples_per_step": k3 + kc,
                       "l2": "256 MB buffer written between steps (outside the step events); "
                             "the graph's device arrays are ~1.2 GB, larger than L2",
                       "parallelism": f"replicas x{world}, disjoint sample-id ranges"},
            "breakdown_ms": {"load_and_prefix": statistics.mean(prep_ms),
                             "sample_3path": avg3, "sample_centred": avgc,
                             "readback_and_estimate": statistics.mean(est_ms)},
            "kernel_rates": {"3path_samples_per_s": k3 / (avg3 / 1e3),
                             "centred_samples_per_s": kc / (avgc / 1e3)},
            "roofline": {"bound": "hbm",
                         "kernel": "3-path sampler call: draw sort + k_sample_ordered<3-path>",
                         "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "peak_source": peak_kind,
                         "bytes_per_sample": BYTES_3PATH},
            "roofline_centred": {"bound": "hbm", "achieved": achieved_c, "peak": peak,
                                 "unit": "GB/s", "frac": achieved_c / peak,
                                 "bytes_per_sample": bytes_c, "centred_fraction": f_c},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / args.steps, "clocks": clk,
            "wall_s_timed_region": t_wall,
            "hist6": [int(x) for x in last["hist6"]], "hist4": [int(x) for x in last["hist4"]],
            "estimate": [float(x) for x in last["est"]],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------- batched and served arms

def _gen_many(specs, make, threads=16):
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(make, specs))


def batched_pool_specs(seed: int = 4):
    """512 R-MAT graphs: scale ~U{10..18}, edge factor ~U{8..32}, own seeds."""
    rs = np.random.default_rng(seed)
    return [(int(rs.integers(10, 19)), float(rs.integers(8, 33)), 1000 + i) for i in range(512)]


def _time_events(fn, reps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def run_batched(args):
    """512 graphs of uneven size, per-graph k, one persistent launch per step
    (captured in a CUDA graph), against 1024 plain per-graph launches."""
    import torch
    import graphgen as gg
    from paper_1411_4942_gb300 import batch as B
    from paper_1411_4942_gb300 import pathsample as ps

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, "nccl")
    t0 = time.perf_counter()
    specs = batched_pool_specs()
    hosts = _gen_many(specs, lambda s: gg.rmat(s[0], s[1], seed=s[2]))
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    graphs = [ps.Graph(h.off, h.col, device=device) for h in hosts]
    gset = B.GraphSet(graphs)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t0
    rs = np.random.default_rng(44)
    reqs = B.random_requests(rs, len(graphs), log2_k=(16, 22))
    for r in reqs:
        r.first_id = rank << 40  # disjoint id ranges per rank
    samples = sum(r.k for r in reqs)
    tuner = B.Autotuner()
    cfg = tuner.tune_launch(gset, reqs)
    runner = B.BatchRunner(gset, reqs, cfg)
    runner.capture()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)
    # correctness against the plain calls
    runner.launch()
    plain_hist = B.run_plain(gset, reqs)
    torch.cuda.synchronize()
    exact = bool(np.array_equal(runner.histograms(),
                                plain_hist.cpu().numpy().reshape(-1, 6).astype(np.uint64)))
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = ps.ps_kernel_launches()
    t_graph = _time_events(runner.replay, args.steps, args.warmup, flush, stream)
    t_eager = _time_events(runner.launch, args.steps, args.warmup, flush, stream)
    l_eager = ps.ps_kernel_launches() - l0
    t_plain = _time_events(lambda: B.run_plain(gset, reqs), args.steps, args.warmup, flush, stream)
    clk = clocks.stop()
    # plain calls captured in a CUDA graph (launch overhead removed)
    hist_c = torch.zeros(6 * len(reqs), dtype=torch.int64, device=device)
    g_plain = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device)
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        for r in reqs:
            fn = ps.ps_sample_3paths if r.sampler == 0 else ps.ps_sample_centered
            fn(gset.graphs[r.graph].handle, r.k, r.seed, r.first_id, hist_c.data_ptr() + 48 * r.slot)
    torch.cuda.synchronize()
    with torch.cuda.graph(g_plain):
        hist_c.zero_()
        for r in reqs:
            fn = ps.ps_sample_3paths if r.sampler == 0 else ps.ps_sample_centered
            fn(gset.graphs[r.graph].handle, r.k, r.seed, r.first_id, hist_c.data_ptr() + 48 * r.slot)
    t_plain_graph = _time_events(g_plain.replay, args.steps, args.warmup, flush, stream)
    ms = reduce_max(statistics.mean(t_graph), world, device)
    value = world * samples / (ms / 1e3)
    if rank == 0:
        edges = sum(g.m for g in hosts)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": ("batched512: 512 R-MAT graphs, scale ~U{10..18}, edge factor "
                                    "~U{8..32}, (0.57,0.19,0.19,0.05), seeds 1000..1511; per graph "
                                    "k = 2^U{16..22} 3-path + the same k centred samples, own "
                                    "Philox seeds; one persistent queue launch per step, CUDA graph"),
                       "graphs": len(graphs), "edges": edges, "samples_per_step": samples,
                       "device_bytes": gset.workspace_bytes,
                       "l2": "256 MB buffer written between steps (outside the step events)",
                       "parallelism": f"replicas x{world}, disjoint sample-id ranges"},
            "batched_graph_ms": statistics.mean(t_graph),
            "batched_eager_ms": statistics.mean(t_eager),
            "plain_eager_ms": statistics.mean(t_plain),
            "plain_graph_ms": statistics.mean(t_plain_graph),
            "batched_vs_plain_eager": statistics.mean(t_plain) / statistics.mean(t_graph),
            "batched_vs_plain_graph": statistics.mean(t_plain_graph) / statistics.mean(t_graph),
            "histograms_equal_plain": exact,
            "autotune": {"choice": vars(cfg), "trials": tuner.log},
            "generation_s": t_gen, "load_all_graphs_s": t_load,
            "gpu_launches": args.steps,  # one queue kernel per replayed step
            "gpu_launches_eager_timing": int(l_eager),
            "clocks": clk, "e2e": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)


def served_pool_specs(seed: int = 5):
    """64 Chung-Lu graphs: n log-uniform in [1e4, 1e6], exponent ~U[2.1, 2.8],
    mean weight 20, max weight sqrt(20 n)."""
    rs = np.random.default_rng(seed)
    return [(int(10 ** rs.uniform(4, 6)), float(rs.uniform(2.1, 2.8)), 2000 + i) for i in range(64)]


def run_served(args):
    """20,000 Poisson requests at 2,000 req/s over 64 resident graphs within a
    40 GB budget, continuously batched; against sequential plain calls."""
    import torch
    import graphgen as gg
    from paper_1411_4942_gb300 import batch as B
    from paper_1411_4942_gb300 import serve as S

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, "nccl")
    specs = served_pool_specs()
    t0 = time.perf_counter()
    hosts = _gen_many(specs, lambda s: gg.chung_lu(s[0], 20.0, s[1], (20.0 * s[0]) ** 0.5, s[2],
                                                  exact_pairs=False))
    t_gen = time.perf_counter() - t0
    sources = {f"cl{i}": (h.off, h.col) for i, h in enumerate(hosts)}
    budget = 40 << 30
    pool = S.GraphPool(sources, budget, device=device)
    for key in sources:  # warm pool: load what fits
        if pool.acquire(key) is not None:
            pool.release(key)
    rs = np.random.default_rng(55 + rank)
    n_req = args.requests
    reqs = S.poisson_requests(rs, list(sources), n_req, args.rate, log2_k=(14, 22))
    server = S.Server(pool, max_active=4096, cfg=B.LaunchConfig(256, 1 << 16))
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    results, report = server.run(reqs, realtime=True)
    clk = clocks.stop()
    # the same requests all queued at once: the server's saturated throughput
    sat_server = S.Server(pool, max_active=4096, cfg=B.LaunchConfig(256, 1 << 16))
    sat_results, sat_report = sat_server.run(reqs, realtime=False)
    seq, seq_report = S.run_sequential(pool, reqs)
    by_id = {rid: (h6, h4) for rid, h6, h4, _ in seq}
    exact = all(r.hist6.tolist() == by_id[r.rid][0].tolist() and
                r.hist4.tolist() == by_id[r.rid][1].tolist() for r in results + sat_results)
    value = reduce_max(-report["samples_per_s"], world, device) * -world
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1,
            "warmup": 0, "ms_per_step": 1e3 * report["makespan_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": ("served64: 64 Chung-Lu graphs, n log-uniform in [1e4, 1e6], "
                                    "exponent ~U[2.1, 2.8], mean weight 20, max weight sqrt(20 n); "
                                    f"{n_req} Poisson requests at {args.rate:g} req/s, k = "
                                    "2^U{14..22} per sampler, own seeds; 40 GB device budget"),
                       "graphs": len(hosts), "edges": sum(h.m for h in hosts),
                       "parallelism": f"replicas x{world}, own request streams"},
            "served": report, "served_saturated": sat_report, "sequential_plain": seq_report,
            "offered_samples_per_s": report["samples"] / max(r.arrival for r in reqs),
            "saturated_vs_sequential": sat_report["samples_per_s"] / seq_report["samples_per_s"],
            "results_equal_alone": exact, "generation_s": t_gen, "clocks": clk,
            "gpu_launches": report["iterations"], "e2e": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle on the host cores, as it stands, on the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    if args.workload not in workloads():
        print(json.dumps({"impl": "reference", "unavailable": (
            f"the oracle arm covers single-graph workloads; {args.workload} is measured "
            "against plain per-graph GPU calls instead")}), flush=True)
        return
    wl = workloads()[args.workload]
    g = wl["make"]()
    threads = max(1, O.max_threads())
    t0 = time.perf_counter()
    og = O.prepare(g.off, g.col)
    t_prep = time.perf_counter() - t0
    slice_k = args.cpu_slice
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.sample_3paths(og, slice_k, wl["seed"], i * slice_k, threads=threads)
        O.sample_centered(og, slice_k, wl["seed"], i * slice_k, threads=threads)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_pair = statistics.mean(times)  # slice_k ids of each sampler
    full_s = t_prep + per_pair * (wl["k3"] + wl["kc"]) / (2 * slice_k)
    value = (wl["k3"] + wl["kc"]) / full_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * full_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": f"{args.workload}: {wl['desc']}", "n": g.n,
                                        "m": g.m, "k3": wl["k3"], "kc": wl["kc"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": (f"oracle prepare on the full graph once ({t_prep:.2f} s); "
                                    f"each step samples {slice_k} ids of each sampler on "
                                    f"{threads} threads; scaled linearly to k3 + kc")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", default="rmat20",
                    choices=["rmat20", "chung_lu_5k", "social3m", "batched512", "served64"])
    ap.add_argument("--cpu-slice", type=int, default=1 << 20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=20000, help="served64: number of requests")
    ap.add_argument("--rate", type=float, default=2000.0, help="served64: arrivals per second")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched512":
        run_batched(args)
    elif args.workload == "served64":
        run_served(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
