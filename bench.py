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
flushed between steps.  The default workload is the 3M-vertex, 117M-edge
social-network-shaped graph (k = 2^27 + 2^26 samples per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]
                    [--workload social3m|rmat20|chung_lu_5k|batched512|served64]

Under torchrun each rank samples its own contiguous range of sample ids on its
own replica of the graph (weak scaling); the only exchange is the per-step sum
of the 10 histogram words (shard.combine_histograms), after which rank 0's
estimates cover every rank's samples.

--impl reference times the oracle (plain C on the host cores) on the same
workload: its prepare once, then every step a new bounded range of ids.
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
# largest chunk of the draw-ordered samplers (their scratch is 5 B per sample
# of a chunk); by default one chunk holds all of a call's samples up to this
MAX_ORDER_CHUNK = 1 << 27
# the load step's streaming bytes per edge in the O(m) preprocessing model:
# 8 B per stored arc (its input column read, its relabelled column written;
# two arcs per edge) plus the two uint64 prefixes, 32 B
BYTES_LOAD_PER_EDGE = 48


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


L2_RESIDENT_BYTES = 64 << 20  # a workspace this small stays in the 129 MB L2


def measured_l2_read(device, stream) -> float:
    """L2 read bandwidth in GB/s, measured in this run: the library's probe
    reading a 32 MB buffer (which stays in L2) 200 times with L2-only loads,
    best of 5 launches timed with events on the launching stream."""
    import torch
    from paper_1411_4942_gb300 import pathsample as ps
    nbytes, passes = 32 << 20, 200
    with torch.cuda.stream(stream):
        buf = torch.ones(nbytes // 4, dtype=torch.int32, device=device)
        sink = torch.zeros(1, dtype=torch.int64, device=device)
        ps._check(ps.ps_l2_read_probe(buf.data_ptr(), nbytes, 1, sink.data_ptr(), stream.cuda_stream),
                  "ps_l2_read_probe")
        best = float("inf")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(5):
            e0.record(stream)
            ps._check(ps.ps_l2_read_probe(buf.data_ptr(), nbytes, passes, sink.data_ptr(), stream.cuda_stream),
                      "ps_l2_read_probe")
            e1.record(stream)
            torch.cuda.synchronize(device)
            best = min(best, e0.elapsed_time(e1))
    return nbytes * passes / (best / 1e3) / 1e9


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

# Bounded slices of the workload that the oracle samples (ids from 0 of each
# sampler, the same ids on every repeat), as (label, threads, repeats, k3, kc);
# threads 0 = every host core.  About 10-20 s of CPU work in all.
ORACLE_SLICES = [("all_cores", 0, 5, 1 << 22, 1 << 21), ("one_core", 1, 3, 1 << 19, 1 << 18)]
# per step of the reference arm: this many ids of each sampler (2:1 as k3:kc
# of the 3M-vertex workload), every step a new id range
REFERENCE_SLICE = (1 << 22, 1 << 21)


def _oracle_worker(conn, off, col, seed, slices):
    """The oracle in its own process: on request its prepare (validation,
    relabelling, edge table and prefixes), then the bounded sampling slices,
    timed.  It waits until the GPU arm's timed legs are over: running beside
    them, its 16 threads took the host cores and host memory bandwidth that
    the end-to-end leg's upload and launches need (36.3 against 33.0 ms per
    step on the 3M-vertex graph)."""
    if conn.recv() != "prepare":
        return
    sys.path.insert(0, ROOT)
    import oracle as O
    t0 = time.perf_counter()
    og = O.prepare(off, col)
    prep_s = time.perf_counter() - t0
    conn.send({"prepare_s": prep_s, "W": og.W, "Lambda": og.Lambda, "N1": og.N1})
    if conn.recv() != "go":
        return
    all_cores = max(1, O.max_threads())
    out = {"prepare_s": prep_s, "host_cores": all_cores, "slices": {}}
    for label, threads, reps, s3, sc in slices:
        th = threads or all_cores
        t3, tc = [], []
        for _ in range(reps):
            t0 = time.perf_counter()
            h6 = O.sample_3paths(og, s3, seed, 0, threads=th)
            t3.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            h4 = O.sample_centered(og, sc, seed, 0, threads=th)
            tc.append(time.perf_counter() - t0)
        out["slices"][label] = {
            "threads": th, "repeats": reps, "k3": s3, "kc": sc,
            "s_3path_median": statistics.median(t3), "s_centred_median": statistics.median(tc),
            "hist6": [int(x) for x in h6], "hist4": [int(x) for x in h4]}
    conn.send(out)


class OracleLeg:
    """The CPU baseline of the benchmark line: the oracle as it stands, on the
    host cores, on bounded slices of the same workload.  Started (spawned)
    before the GPU arm touches CUDA; it works only after the timed legs."""

    def __init__(self, g, seed, slices, k3, kc):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.slices = [(lb, th, reps, min(s3, k3), min(sc, kc)) for lb, th, reps, s3, sc in slices]
        self.proc = ctx.Process(target=_oracle_worker, args=(child, g.off, g.col, seed, self.slices),
                                daemon=True)
        self.proc.start()

    def _recv(self, limit_s=1800.0):
        # never wait on a worker that has died (a spawn or import failure)
        t0 = time.perf_counter()
        while not self.conn.poll(1.0):
            if not self.proc.is_alive():
                raise RuntimeError("the oracle leg's process ended before replying")
            if time.perf_counter() - t0 > limit_s:
                raise TimeoutError("the oracle leg did not reply in time")
        return self.conn.recv()

    def run(self):
        self.conn.send("prepare")
        ready = self._recv()
        self.conn.send("go")
        res = self._recv()
        res.update({k: ready[k] for k in ("W", "Lambda", "N1")})
        self.proc.join(timeout=60)
        return res

    def stop(self):
        try:
            self.conn.send("stop")
        except (OSError, BrokenPipeError):
            pass
        self.proc.join(timeout=10)
        if self.proc.is_alive():
            self.proc.terminate()


def cpu_baseline_line(res):
    """cpu_baseline of the JSON line from the oracle leg's timings: value =
    the oracle's sampling rate on all host cores over the workload's mix of
    the two samplers (its prepare is timed separately, once)."""
    a = res["slices"]["all_cores"]
    o = res["slices"]["one_core"]
    rate = lambda s: (s["k3"] + s["kc"]) / (s["s_3path_median"] + s["s_centred_median"])  # noqa: E731
    return {
        "value": rate(a), "unit": UNIT, "cores": a["threads"], "kind": "oracle",
        "sample": (f"oracle sampling loops, ids [0, {a['k3']}) of Alg. 1 and [0, {a['kc']}) of "
                   f"Alg. 3 on {a['threads']} threads, median of {a['repeats']} "
                   f"({a['s_3path_median']:.3f} s + {a['s_centred_median']:.3f} s); its prepare "
                   f"(validate, relabel, edge table, prefixes) of the whole graph once, "
                   f"{res['prepare_s']:.1f} s, not in value; nothing extrapolated"),
        "prepare_s": res["prepare_s"],
        "one_core": {"samples_per_s": rate(o), "k3": o["k3"], "kc": o["kc"], "repeats": o["repeats"],
                     "s_3path_median": o["s_3path_median"], "s_centred_median": o["s_centred_median"]},
        "all_cores": {"samples_per_s": rate(a), "3path_samples_per_s": a["k3"] / a["s_3path_median"],
                      "centred_samples_per_s": a["kc"] / a["s_centred_median"]},
    }


def workload_config(name, wl, n, m, W, Lambda, d_max, world):
    """The `config` object of both arms' JSON lines (the same dict)."""
    return {"workload": f"{name}: {wl['desc']}", "n": int(n), "m": int(m), "W": int(W),
            "Lambda": int(Lambda), "d_max": int(d_max), "k3": wl["k3"], "kc": wl["kc"],
            "samples_per_step": wl["k3"] + wl["kc"],
            "l2": ("a 256 MB buffer is written between steps, outside the step events, and the "
                   "graph's device arrays are larger than L2"),
            "parallelism": f"replicas x{world}, contiguous sample-id ranges, one histogram sum"}


# --------------------------------------------------------------- GPU arm

def run_cuda(args):
    rank, world, local = dist_env()
    wl = workloads()[args.workload]
    g = wl["make"]()
    # the oracle leg starts before this process initialises CUDA
    leg = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        leg = OracleLeg(g, wl["seed"], ORACLE_SLICES, wl["k3"], wl["kc"])
    try:
        _run_cuda(args, g, wl, leg)
    finally:
        if leg is not None:
            leg.stop()


def _run_cuda(args, g, wl, leg):
    import torch
    from paper_1411_4942_gb300 import pathsample as ps
    from paper_1411_4942_gb300 import shard

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, "nccl")
    k3, kc, seed = wl["k3"], wl["kc"], wl["seed"]
    # weak scaling: the job is world x (k3 + kc) samples, every rank one
    # contiguous range of ids of each sampler, histograms summed per step
    first3, n3 = shard.shard_range(world * k3, rank, world)
    firstc, nc = shard.shard_range(world * kc, rank, world)
    assert n3 == k3 and nc == kc
    ps.load_library()
    chunk = args.order_chunk or min(max(k3, kc, 1), MAX_ORDER_CHUNK)
    tuning = ps.make_tuning(adjacency=args.adjacency, hub_count=args.hub_count, draw_order=args.draw_order,
                            hub_span_log2=args.hub_span)

    stream = torch.cuda.Stream(device)
    sp = stream.cuda_stream
    with torch.cuda.stream(stream):
        d_off = torch.as_tensor(g.off).to(device)
        d_col = torch.as_tensor(g.col).to(device)
        nb = ps.ps_graph_workspace_bytes(g.n, g.nnz, tuning)
        ws = torch.empty(nb, dtype=torch.uint8, device=device)
        hist = torch.zeros(16, dtype=torch.int64, device=device)
        # scratch of the draw-ordered samplers: one chunk
        osb = ps.ps_ordered_scratch_bytes(chunk)
        oscr = torch.empty(osb, dtype=torch.uint8, device=device)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)]
              for _ in range(args.steps + args.warmup)]
        last = {}

        def step(i):
            e = ev[i]
            e[0].record(stream)
            rc, h = ps.ps_load_csr(g.n, g.nnz, d_off.data_ptr(), d_col.data_ptr(), ws.data_ptr(), nb,
                                   tuning, sp)
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
            shard.combine_histograms(hist)
            hh = hist.cpu().numpy().astype(np.uint64)
            rc, est, lo, hi = ps.ps_estimate(st, hh[shard.HIST6], world * k3, hh[shard.HIST4],
                                             world * kc, 0.01)
            e[4].record(stream)
            ps.ps_graph_free(h)
            last.update(stats=st, hist6=hh[shard.HIST6].copy(), hist4=hh[shard.HIST4].copy(),
                        est=est, lo=lo, hi=hi)

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
    f_c = 1.0 - float(h4[0]) / (world * kc) if kc else 0.0
    bytes_c = (7 + 2 * f_c) * SECTOR
    achieved_c = bytes_c * kc / (avgc / 1e3) / 1e9
    st = last["stats"]
    # the load step against streaming: 48 B per edge (the degree, offset and
    # column reads of the input, the records and both prefixes written)
    load_bytes = BYTES_LOAD_PER_EDGE * st.m
    achieved_load = load_bytes / (statistics.mean(prep_ms) / 1e3) / 1e9
    traffic = ncu_traffic(args.workload)
    # a graph whose whole workspace fits in L2: the samplers against L2 too
    roof_l2 = None
    if nb <= L2_RESIDENT_BYTES:
        l2 = measured_l2_read(device, stream)
        roof_l2 = {"bound": "l2", "achieved": achieved, "achieved_centred": achieved_c, "peak": l2,
                   "unit": "GB/s", "frac": achieved / l2, "frac_centred": achieved_c / l2,
                   "workspace_bytes": nb,
                   "peak_source": "measured in this run: ps_l2_read_probe, 200 L2-only read passes over a "
                                  "32 MB buffer, best of 5"}

    # end to end through the host-buffer call (inputs copied from pinned memory every step)
    e2e = None
    if not args.no_e2e:
        h_off = torch.as_tensor(g.off).pin_memory()
        h_col = torch.as_tensor(g.col).pin_memory()
        nb2 = ps.ps_end_to_end_workspace_bytes(g.n, g.nnz, tuning) + osb  # + draw-order scratch
        del ws
        ws2 = torch.empty(nb2, dtype=torch.uint8, device=device)
        times = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            rc, est, lo, hi, h6, h4e, st2 = ps.ps_count_motifs_host(
                h_off, h_col, k3, kc, seed, 0.01, ws2.data_ptr(), nb2, tuning, sp)
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
        del ws2

    cpu = None
    if leg is not None:
        res = leg.run()
        cpu = cpu_baseline_line(res)
        cpu["oracle_equals_gpu"] = _check_oracle_slices(g, wl, res, device)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args.workload, wl, g.n, st.m, st.W, st.Lambda, st.d_max,
                                      world),
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
            "roofline_load": {"bound": "hbm", "achieved": achieved_load, "peak": peak,
                              "unit": "GB/s", "frac": achieved_load / peak,
                              "bytes_per_edge": BYTES_LOAD_PER_EDGE,
                              "kernel": "ps_load_csr + ps_tau_prefix (all kernels, sorts included)"},
            "roofline_l2": roof_l2,
            "order_chunk": chunk,
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


def _check_oracle_slices(g, wl, res, device):
    """The oracle's slice histograms against the library's for the same ids
    (the draw-ordered samplers the step times), and W / Lambda / N_1."""
    import torch
    from paper_1411_4942_gb300 import pathsample as ps
    G = ps.Graph(g.off, g.col, device=device)
    ok = (int(G.stats.W), int(G.stats.Lambda), G.stats.N1) == (res["W"], res["Lambda"], res["N1"])
    for sl in res["slices"].values():
        h6 = G.sample_3paths_ordered(sl["k3"], wl["seed"]).cpu().numpy()[:6]
        h4 = G.sample_centered_ordered(sl["kc"], wl["seed"]).cpu().numpy()[:4]
        ok = ok and [int(x) for x in h6] == sl["hist6"] and [int(x) for x in h4] == sl["hist4"]
    torch.cuda.synchronize(device)
    G.close()
    return bool(ok)


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
    # hub-bitmap rows per graph-size bucket, tuned on each bucket's largest graph
    tuner = B.Autotuner()
    t0 = time.perf_counter()
    hub_choice = tuner.tune_hubs(hosts)
    t_tune_hubs = time.perf_counter() - t0
    t0 = time.perf_counter()
    graphs = [ps.Graph(h.off, h.col, device=device, tuning=tuner.graph_tuning(h.m)) for h in hosts]
    gset = B.GraphSet(graphs)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t0
    rs = np.random.default_rng(44)
    reqs = B.random_requests(rs, len(graphs), log2_k=(16, 22))
    for r in reqs:
        r.first_id = rank << 40  # disjoint id ranges per rank
    samples = sum(r.k for r in reqs)
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
            "autotune": {"choice": {**vars(cfg),
                                    "hub_rows_by_size_bucket": {
                                        f"edges<2^{[17, 20, 99][b]}" if b < 2 else "edges>=2^20":
                                            {"rows": rows, "min_degree": deg}
                                        for b, (rows, deg) in sorted(hub_choice.items())}},
                         "trials": tuner.log, "tune_hubs_s": t_tune_hubs},
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
    """The oracle on the host cores, as it stands, on the same workload: its
    prepare of the whole graph once, then every step a new bounded id range of
    both samplers on all host cores, each step timed as it ran."""
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
    s3, sc = min(REFERENCE_SLICE[0], wl["k3"]), min(REFERENCE_SLICE[1], wl["kc"])
    times, hists = [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        h6 = O.sample_3paths(og, s3, wl["seed"], i * s3, threads=threads)
        h4 = O.sample_centered(og, sc, wl["seed"], i * sc, threads=threads)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
        if i == 0:
            hists = ([int(x) for x in h6], [int(x) for x in h4])
    total_s = sum(times)
    value = args.steps * (s3 + sc) / total_s
    d_max = int(np.diff(g.off).max()) if g.n else 0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": workload_config(args.workload, wl, g.n, og.m, og.W, og.Lambda, d_max, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": (f"every step: oracle sampling loops over a new range of "
                                    f"{s3} ids of Alg. 1 and {sc} of Alg. 3 on {threads} threads, "
                                    f"timed as run (no extrapolation); the oracle's prepare of the "
                                    f"whole graph ran once before the steps ({t_prep:.1f} s) and "
                                    f"is not in value"),
                         "prepare_s": t_prep},
        "samples_per_step": s3 + sc,
        "step0_hist6": hists[0], "step0_hist4": hists[1],
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_oracle_protocol(args):
    """The oracle's own timings on the host cores, for the record: its prepare
    and each sampler timed separately, on one core and on all cores, median of
    `--oracle-reps` runs.  Sampling on one core takes a bounded slice of each
    sampler's ids (stated); nothing is extrapolated.  Prints one JSON line."""
    import oracle as O
    wl = workloads()[args.workload]
    g = wl["make"]()
    cores = max(1, O.max_threads())
    reps = args.oracle_reps
    prep = []
    for _ in range(reps):
        t0 = time.perf_counter()
        og = O.prepare(g.off, g.col)
        prep.append(time.perf_counter() - t0)
    out = {"workload": args.workload, "host_cores": cores, "repeats": reps,
           "prepare_s_median": statistics.median(prep), "prepare_s": prep, "sampling": {}}
    for label, th, k3, kc in (("one_core", 1, min(wl["k3"], 1 << 20), min(wl["kc"], 1 << 20)),
                              ("all_cores", cores, wl["k3"], wl["kc"])):
        t3, tc = [], []
        for _ in range(reps):
            t0 = time.perf_counter()
            h6 = O.sample_3paths(og, k3, wl["seed"], 0, threads=th)
            t3.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            h4 = O.sample_centered(og, kc, wl["seed"], 0, threads=th)
            tc.append(time.perf_counter() - t0)
        out["sampling"][label] = {
            "threads": th, "k3": k3, "kc": kc, "s_3path_median": statistics.median(t3),
            "s_centred_median": statistics.median(tc),
            "3path_samples_per_s": k3 / statistics.median(t3),
            "centred_samples_per_s": kc / statistics.median(tc),
            "hist6": [int(x) for x in h6], "hist4": [int(x) for x in h4]}
    print(json.dumps({"oracle_protocol": out}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", default="social3m",
                    choices=["rmat20", "chung_lu_5k", "social3m", "batched512", "served64"])
    ap.add_argument("--order-chunk", type=int, default=0,
                    help="samples per chunk of the draw-ordered samplers (0: all of a call's "
                         f"samples, up to {MAX_ORDER_CHUNK})")
    ap.add_argument("--adjacency", type=int, default=0,
                    help="adjacency test: 0 default (hash set), 1 hash set, 2 search + hub rows, "
                         "3 per-vertex tables")
    ap.add_argument("--hub-count", type=int, default=0, help="hub bitmap rows (0 default, -1 none)")
    ap.add_argument("--hub-span", type=int, default=0, help="hub rows cover the top 2^k labels (0 default, -1 all)")
    ap.add_argument("--draw-order", type=int, default=0,
                    help="draw-ordered samplers: 0 by size (default), 1 one pass (256 ranges of r), "
                         "2 two passes (65536 ranges), -1 id order")
    ap.add_argument("--oracle-protocol", action="store_true",
                    help="time the oracle alone (prepare and samplers separately, one core and all "
                         "cores) on --workload and print its JSON line")
    ap.add_argument("--oracle-reps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=20000, help="served64: number of requests")
    ap.add_argument("--rate", type=float, default=2000.0, help="served64: arrivals per second")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.oracle_protocol:
        run_oracle_protocol(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched512":
        run_batched(args)
    elif args.workload == "served64":
        run_served(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
