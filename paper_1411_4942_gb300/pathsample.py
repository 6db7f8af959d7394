"""ctypes binding of libpathsample.so (include/pathsample.h).

The functions named ``ps_*`` mirror the C interface one to one and only
marshal arguments; every step of the sampling path runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace and histograms) and
streams.  There is no fallback: if the library cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

PS_OK, PS_NO_PATHS = 0, 1
PS_ERR_ARG, PS_ERR_NOT_SIMPLE, PS_ERR_ASYMMETRIC = -1, -2, -3
PS_ERR_WORKSPACE, PS_ERR_OVERFLOW, PS_ERR_TIMEOUT = -4, -5, -6
PS_ERR_CUDA, PS_ERR_STATE, PS_ERR_NOMEM = -7, -8, -9

PS_ARRAY_OFFSETS, PS_ARRAY_COLUMNS, PS_ARRAY_RANK = 0, 1, 2
PS_ARRAY_EDGES, PS_ARRAY_PTAU, PS_ARRAY_PLAMBDA = 3, 4, 5

EXPORTED = [
    "ps_graph_workspace_bytes", "ps_load_csr", "ps_tau_prefix", "ps_sample_3paths",
    "ps_sample_centered", "ps_estimate", "ps_graph_free", "ps_strerror", "ps_graph_copy",
    "ps_end_to_end_workspace_bytes", "ps_count_motifs_host", "ps_batch_table_bytes",
    "ps_batch_sample", "ps_batch_prepare", "ps_batch_sample_prepared", "ps_kernel_launches",
    "ps_exact_scratch_bytes", "ps_count_exact", "ps_estimate_ex", "ps_count_adaptive",
    "ps_ingest_workspace_bytes", "ps_csr_from_edges", "ps_ordered_scratch_bytes",
    "ps_sample_3paths_ordered", "ps_sample_centered_ordered",
]

PS_EST_C1_FROM_CENTRED = 1
PS_EST_3PATH_ONLY = 2


class PathSampleError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ps_strerror(code)} (status {code})")


class PsTuning(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("guide_log2_ratio", ctypes.c_int32), ("hub_count", ctypes.c_int32),
                ("samples_per_thread", ctypes.c_int32), ("adjacency", ctypes.c_int32),
                ("draw_order", ctypes.c_int32), ("hub_min_degree", ctypes.c_int32),
                ("hub_span_log2", ctypes.c_int32)]


class PsStats(ctypes.Structure):
    _fields_ = [("W", ctypes.c_uint64), ("Lambda", ctypes.c_uint64), ("N1_lo", ctypes.c_uint64),
                ("N1_hi", ctypes.c_uint64), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("d_max", ctypes.c_int64), ("hubs", ctypes.c_int64), ("tau_shift", ctypes.c_int32),
                ("lambda_shift", ctypes.c_int32)]

    @property
    def N1(self) -> int:
        return int(self.N1_lo) | (int(self.N1_hi) << 64)

    def as_dict(self) -> dict:
        return {"W": int(self.W), "Lambda": int(self.Lambda), "N1": self.N1, "n": int(self.n),
                "m": int(self.m), "d_max": int(self.d_max), "hubs": int(self.hubs),
                "tau_shift": int(self.tau_shift), "lambda_shift": int(self.lambda_shift)}


class PsWork(ctypes.Structure):
    _fields_ = [("first_id", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("count", ctypes.c_uint32),
                ("graph", ctypes.c_uint32), ("slot", ctypes.c_uint32), ("sampler", ctypes.c_uint32)]


WORK_DTYPE = np.dtype([("first_id", np.uint64), ("seed", np.uint64), ("count", np.uint32),
                       ("graph", np.uint32), ("slot", np.uint32), ("sampler", np.uint32)])
assert WORK_DTYPE.itemsize == ctypes.sizeof(PsWork) == 32

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpathsample.so (building it with nvcc when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1411_4942_gb300._build.build()")
        lib = ctypes.CDLL(path)
        V, I32, I64, U64, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                ctypes.c_size_t)
        P = ctypes.POINTER
        sig = {
            "ps_graph_workspace_bytes": ([I64, I64, V], SZ),
            "ps_load_csr": ([I64, I64, V, V, V, SZ, V, V, P(V)], I32),
            "ps_tau_prefix": ([V, V, P(PsStats)], I32),
            "ps_sample_3paths": ([V, U64, U64, U64, V, V], I32),
            "ps_sample_centered": ([V, U64, U64, U64, V, V], I32),
            "ps_ordered_scratch_bytes": ([U64], SZ),
            "ps_sample_3paths_ordered": ([V, U64, U64, U64, V, V, SZ, V], I32),
            "ps_sample_centered_ordered": ([V, U64, U64, U64, V, V, SZ, V], I32),
            "ps_estimate": ([P(PsStats), V, U64, V, U64, ctypes.c_double, V, V, V], I32),
            "ps_graph_free": ([V], None),
            "ps_strerror": ([I32], ctypes.c_char_p),
            "ps_graph_copy": ([V, I32, V, SZ, V], I32),
            "ps_end_to_end_workspace_bytes": ([I64, I64, V], SZ),
            "ps_count_motifs_host": ([I64, I64, V, V, U64, U64, U64, ctypes.c_double, V, SZ, V, V,
                                      V, V, P(PsStats), V, V, V], I32),
            "ps_batch_table_bytes": ([I32], SZ),
            "ps_batch_sample": ([V, I32, V, I64, V, V, V, V, V], I32),
            "ps_batch_prepare": ([V, I32, V, V], I32),
            "ps_batch_sample_prepared": ([V, I32, V, I64, V, V, V, V], I32),
            "ps_kernel_launches": ([], U64),
            "ps_prefix_pairs_static": ([V, V, V, V, I64, V], I32),
            "ps_l2_read_probe": ([V, U64, I32, V, V], I32),
            "ps_selftest_bounded_wait": ([V, ctypes.c_uint32, V], I32),
            "ps_exact_scratch_bytes": ([V, I32], SZ),
            "ps_ingest_workspace_bytes": ([I64, I64], SZ),
            "ps_csr_from_edges": ([I64, I64, V, V, V, SZ, V, V, P(I64), V], I32),
            "ps_estimate_ex": ([P(PsStats), V, U64, V, U64, ctypes.c_double, ctypes.c_uint32, V, V,
                                V], I32),
            "ps_count_adaptive": ([V, U64, ctypes.c_double, ctypes.c_double, U64, U64, ctypes.c_uint32,
                                   ctypes.c_uint32, V, V, V, P(U64), V, V, V, V, V], I32),
            "ps_count_exact": ([V, V, SZ, V, V, V], I32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(code: int, where: str, allow=(PS_OK,)) -> int:
    if code not in allow:
        raise PathSampleError(code, where)
    return code


def _tuning_ptr(t):
    return ctypes.byref(t) if t is not None else None


def _stream_ptr(stream) -> int | None:
    """cudaStream_t of a torch stream (None: torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


# ----------------------------------------------------------- C-level calls

def ps_strerror(code: int) -> str:
    return load_library().ps_strerror(code).decode()


def ps_graph_workspace_bytes(n: int, nnz: int, tuning: PsTuning | None = None) -> int:
    return int(load_library().ps_graph_workspace_bytes(n, nnz, _tuning_ptr(tuning)))


def ps_end_to_end_workspace_bytes(n: int, nnz: int, tuning: PsTuning | None = None) -> int:
    return int(load_library().ps_end_to_end_workspace_bytes(n, nnz, _tuning_ptr(tuning)))


def ps_load_csr(n, nnz, d_off, d_col, d_workspace, ws_bytes, tuning=None, stream=None):
    """Returns (status, handle); handle is None unless status == PS_OK."""
    h = ctypes.c_void_p()
    rc = load_library().ps_load_csr(n, nnz, d_off, d_col, d_workspace, ws_bytes,
                                    _tuning_ptr(tuning), _stream_ptr(stream), ctypes.byref(h))
    return int(rc), (h.value if rc == PS_OK else None)


def ps_tau_prefix(handle, stream=None):
    st = PsStats()
    rc = load_library().ps_tau_prefix(handle, _stream_ptr(stream), ctypes.byref(st))
    return int(rc), st


def ps_sample_3paths(handle, k, seed, first_id, d_hist6, stream=None) -> int:
    return int(load_library().ps_sample_3paths(handle, k, seed, first_id, d_hist6,
                                               _stream_ptr(stream)))


def ps_sample_centered(handle, k, seed, first_id, d_hist4, stream=None) -> int:
    return int(load_library().ps_sample_centered(handle, k, seed, first_id, d_hist4,
                                                 _stream_ptr(stream)))


def ps_ordered_scratch_bytes(k_chunk) -> int:
    return int(load_library().ps_ordered_scratch_bytes(k_chunk))


def ps_sample_3paths_ordered(handle, k, seed, first_id, d_hist6, d_scratch, scratch_bytes,
                             stream=None) -> int:
    return int(load_library().ps_sample_3paths_ordered(handle, k, seed, first_id, d_hist6, d_scratch,
                                                       scratch_bytes, _stream_ptr(stream)))


def ps_sample_centered_ordered(handle, k, seed, first_id, d_hist4, d_scratch, scratch_bytes,
                               stream=None) -> int:
    return int(load_library().ps_sample_centered_ordered(handle, k, seed, first_id, d_hist4,
                                                         d_scratch, scratch_bytes,
                                                         _stream_ptr(stream)))


def ps_estimate(stats: PsStats, hist6, k3: int, hist4, kc: int, delta: float = 0.01):
    h6 = np.ascontiguousarray(hist6, dtype=np.uint64)
    h4 = np.ascontiguousarray(hist4, dtype=np.uint64)
    est, lo, hi = np.zeros(6), np.zeros(6), np.zeros(6)
    rc = load_library().ps_estimate(ctypes.byref(stats), h6.ctypes.data, k3, h4.ctypes.data, kc,
                                    delta, est.ctypes.data, lo.ctypes.data, hi.ctypes.data)
    return int(rc), est, lo, hi


def ps_estimate_ex(stats: PsStats, hist6, k3: int, hist4, kc: int, delta: float = 0.01,
                   flags: int = 0):
    h6 = np.ascontiguousarray(hist6, dtype=np.uint64)
    h4 = np.ascontiguousarray(hist4, dtype=np.uint64)
    est, lo, hi = np.zeros(6), np.zeros(6), np.zeros(6)
    rc = load_library().ps_estimate_ex(ctypes.byref(stats), h6.ctypes.data, k3, h4.ctypes.data, kc,
                                       delta, flags, est.ctypes.data, lo.ctypes.data,
                                       hi.ctypes.data)
    return int(rc), est, lo, hi


def ps_count_adaptive(handle, seed: int, target: float, delta: float, k0: int, k_max: int,
                      d_hist6: int, d_hist4: int, motif_mask: int = 0x3F, flags: int = 0,
                      stream=None):
    """Returns (status, k_used, hist6, hist4, est, lo, hi)."""
    k_used = ctypes.c_uint64(0)
    h6 = np.zeros(6, dtype=np.uint64)
    h4 = np.zeros(4, dtype=np.uint64)
    est, lo, hi = np.zeros(6), np.zeros(6), np.zeros(6)
    rc = load_library().ps_count_adaptive(handle, seed, target, delta, k0, k_max, motif_mask, flags,
                                          d_hist6, d_hist4, _stream_ptr(stream), ctypes.byref(k_used),
                                          h6.ctypes.data, h4.ctypes.data, est.ctypes.data,
                                          lo.ctypes.data, hi.ctypes.data)
    return int(rc), int(k_used.value), h6, h4, est, lo, hi


def ps_graph_free(handle) -> None:
    if handle:
        load_library().ps_graph_free(handle)


def ps_graph_copy(handle, which: int, dst_ptr: int, nbytes: int, stream=None) -> int:
    return int(load_library().ps_graph_copy(handle, which, dst_ptr, nbytes, _stream_ptr(stream)))


def ps_count_motifs_host(off: np.ndarray, col: np.ndarray, k3: int, kc: int, seed: int,
                         delta: float, d_workspace: int, ws_bytes: int, tuning=None, stream=None):
    """The whole path from host CSR arrays; returns (status, est, lo, hi, hist6, hist4, stats)."""
    n = off.shape[0] - 1
    est, lo, hi = np.zeros(6), np.zeros(6), np.zeros(6)
    h6 = np.zeros(6, dtype=np.uint64)
    h4 = np.zeros(4, dtype=np.uint64)
    st = PsStats()
    rc = load_library().ps_count_motifs_host(
        n, col.shape[0], off.ctypes.data if isinstance(off, np.ndarray) else off.data_ptr(),
        col.ctypes.data if isinstance(col, np.ndarray) else col.data_ptr(), k3, kc, seed, delta,
        d_workspace, ws_bytes, _tuning_ptr(tuning), _stream_ptr(stream), h6.ctypes.data,
        h4.ctypes.data, ctypes.byref(st), est.ctypes.data, lo.ctypes.data, hi.ctypes.data)
    return int(rc), est, lo, hi, h6, h4, st


def ps_kernel_launches() -> int:
    return int(load_library().ps_kernel_launches())


def ps_selftest_bounded_wait(d_scratch: int, spin_limit: int, stream=None) -> int:
    """The scans' bounded device wait on a flag nothing sets: PS_ERR_TIMEOUT."""
    return int(load_library().ps_selftest_bounded_wait(d_scratch, spin_limit, _stream_ptr(stream)))


PS_ERR_TOO_LARGE = -10
PS_PREFIX_STATIC_MAX_ITEMS = 1 << 27


def ps_prefix_pairs_static(d_a, d_b, d_pa, d_pb, count: int, stream=None) -> int:
    """Exact uint64 prefix sums of two device arrays with no device allocation
    (scratch is a fixed array inside the library); for callers that cannot
    allocate device memory."""
    return int(load_library().ps_prefix_pairs_static(d_a, d_b, d_pa, d_pb, count,
                                                     _stream_ptr(stream)))


def ps_l2_read_probe(d_buf, nbytes: int, passes: int, d_sink, stream=None) -> int:
    """Measurement aid: reads a device buffer `passes` times with L2-only
    loads (time it with events; for a buffer that fits in L2 this is the L2
    read bandwidth)."""
    return int(load_library().ps_l2_read_probe(d_buf, nbytes, passes, d_sink, _stream_ptr(stream)))


def ps_exact_scratch_bytes(handle, max_blocks: int = 0) -> int:
    return int(load_library().ps_exact_scratch_bytes(handle, max_blocks))


def ps_count_exact(handle, d_scratch: int, nbytes: int, stream=None):
    """Exact counts; returns (status, N uint64[6], C int64[6])."""
    N = np.zeros(6, dtype=np.uint64)
    C = np.zeros(6, dtype=np.int64)
    rc = load_library().ps_count_exact(handle, d_scratch, nbytes, _stream_ptr(stream),
                                       N.ctypes.data, C.ctypes.data)
    return int(rc), N, C


def ps_ingest_workspace_bytes(n: int, n_edges: int) -> int:
    return int(load_library().ps_ingest_workspace_bytes(n, n_edges))


def ps_csr_from_edges(n: int, n_edges: int, d_src: int, d_dst: int, d_workspace: int, ws_bytes: int,
                      d_off: int, d_col: int, stream=None):
    """Returns (status, nnz)."""
    nnz = ctypes.c_int64(0)
    rc = load_library().ps_csr_from_edges(n, n_edges, d_src, d_dst, d_workspace, ws_bytes, d_off,
                                          d_col, ctypes.byref(nnz), _stream_ptr(stream))
    return int(rc), int(nnz.value)


def csr_from_edges(n: int, src, dst, stream=None):
    """Device CSR (off int64 [n + 1], col int32 [nnz]) of the simple undirected
    graph listed by the int32 device (or host) arrays src / dst."""
    import torch
    dev = src.device if isinstance(src, torch.Tensor) and src.is_cuda else torch.device("cuda")
    s = torch.as_tensor(src, dtype=torch.int32).to(dev).contiguous()
    d = torch.as_tensor(dst, dtype=torch.int32).to(dev).contiguous()
    e = int(s.shape[0])
    nbytes = ps_ingest_workspace_bytes(n, e)
    if nbytes == 0:
        raise PathSampleError(PS_ERR_ARG, "ps_ingest_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(2 * e, 1), dtype=torch.int32, device=dev)
    rc, nnz = ps_csr_from_edges(n, e, s.data_ptr() if e else None, d.data_ptr() if e else None,
                                ws.data_ptr(), nbytes, off.data_ptr(), col.data_ptr(), stream)
    _check(rc, "ps_csr_from_edges")
    return off, col[:nnz]


def ps_batch_table_bytes(n_graphs: int) -> int:
    return int(load_library().ps_batch_table_bytes(n_graphs))


def ps_batch_prepare(handles, d_table: int, stream=None) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    return int(load_library().ps_batch_prepare(arr, len(handles), d_table, _stream_ptr(stream)))


def ps_batch_sample_prepared(d_table, n_graphs, d_items, n_items, d_hist, d_counter,
                             tuning=None, stream=None) -> int:
    return int(load_library().ps_batch_sample_prepared(d_table, n_graphs, d_items, n_items, d_hist,
                                                       d_counter, _tuning_ptr(tuning),
                                                       _stream_ptr(stream)))


def ps_batch_sample(handles, d_items, n_items, d_hist, d_table, d_counter, tuning=None,
                    stream=None) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    return int(load_library().ps_batch_sample(arr, len(handles), d_items, n_items, d_hist, d_table,
                                              d_counter, _tuning_ptr(tuning), _stream_ptr(stream)))


ADJ_HASH, ADJ_SEARCH, ADJ_VTAB = 1, 2, 3


def make_tuning(block_size=0, blocks_per_sm=0, guide_log2_ratio=0, hub_count=0,
                adjacency=0, draw_order=0, samples_per_thread=0, hub_min_degree=0,
                hub_span_log2=0) -> PsTuning:
    t = PsTuning()
    t.block_size, t.blocks_per_sm = block_size, blocks_per_sm
    t.guide_log2_ratio, t.hub_count = guide_log2_ratio, hub_count
    t.adjacency, t.draw_order = adjacency, draw_order
    t.samples_per_thread, t.hub_min_degree = samples_per_thread, hub_min_degree
    t.hub_span_log2 = hub_span_log2
    return t


# ------------------------------------------------------- torch convenience

class Graph:
    """A graph loaded on the GPU: owns its workspace tensor and the handle.

    ``off`` / ``col`` may be numpy arrays or torch tensors (host or device);
    host arrays are copied to the device first.
    """

    def __init__(self, off, col, tuning: PsTuning | None = None, stream=None, device=None):
        import torch
        dev = torch.device(device) if device is not None else torch.device("cuda",
                                                                           torch.cuda.current_device())
        self.device = dev
        self.tuning = tuning
        t_off = torch.as_tensor(off, dtype=torch.int64).to(dev)
        t_col = torch.as_tensor(col, dtype=torch.int32).to(dev)
        self.n = int(t_off.shape[0] - 1)
        self.nnz = int(t_col.shape[0])
        nbytes = ps_graph_workspace_bytes(self.n, self.nnz, tuning)
        if nbytes == 0:
            raise PathSampleError(PS_ERR_ARG, "ps_graph_workspace_bytes")
        # 256-byte aligned: torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.handle = None
        with torch.cuda.device(dev):
            rc, h = ps_load_csr(self.n, self.nnz, t_off.data_ptr(),
                                t_col.data_ptr() if self.nnz else None,
                                self.workspace.data_ptr(), nbytes, tuning, stream)
            _check(rc, "ps_load_csr")
            self.handle = h
            rc, st = ps_tau_prefix(self.handle, stream)
            _check(rc, "ps_tau_prefix", (PS_OK, PS_NO_PATHS))
        self.stats = st
        self.prefix_status = rc

    def close(self):
        if self.handle:
            ps_graph_free(self.handle)
            self.handle = None
        self.workspace = None
        self._order_scratch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_hist(self):
        import torch
        return torch.zeros(8, dtype=torch.int64, device=self.device)

    def sample_3paths(self, k: int, seed: int, first_id: int = 0, hist=None, stream=None):
        hist = self.new_hist() if hist is None else hist
        rc = ps_sample_3paths(self.handle, k, seed, first_id, hist.data_ptr(), stream)
        _check(rc, "ps_sample_3paths", (PS_OK, PS_NO_PATHS))
        return hist

    def sample_centered(self, k: int, seed: int, first_id: int = 0, hist=None, stream=None):
        hist = self.new_hist() if hist is None else hist
        rc = ps_sample_centered(self.handle, k, seed, first_id, hist.data_ptr(), stream)
        _check(rc, "ps_sample_centered", (PS_OK, PS_NO_PATHS))
        return hist

    ORDER_CHUNK = 1 << 24

    def order_scratch(self, k: int):
        """Scratch of the ordered samplers for chunks of min(k, 2^24) samples,
        kept for the next calls (one scratch per Graph: calls on different
        streams need their own, passed to the ps_* functions directly)."""
        import torch
        need = ps_ordered_scratch_bytes(max(1, min(int(k), self.ORDER_CHUNK)))
        cur = getattr(self, "_order_scratch", None)
        if cur is None or cur.numel() < need:
            cur = torch.empty(need, dtype=torch.uint8, device=self.device)
            self._order_scratch = cur
        return cur

    def sample_3paths_ordered(self, k: int, seed: int, first_id: int = 0, hist=None, stream=None):
        hist = self.new_hist() if hist is None else hist
        sc = self.order_scratch(k)
        rc = ps_sample_3paths_ordered(self.handle, k, seed, first_id, hist.data_ptr(), sc.data_ptr(),
                                      sc.numel(), stream)
        _check(rc, "ps_sample_3paths_ordered", (PS_OK, PS_NO_PATHS))
        return hist

    def sample_centered_ordered(self, k: int, seed: int, first_id: int = 0, hist=None, stream=None):
        hist = self.new_hist() if hist is None else hist
        sc = self.order_scratch(k)
        rc = ps_sample_centered_ordered(self.handle, k, seed, first_id, hist.data_ptr(),
                                        sc.data_ptr(), sc.numel(), stream)
        _check(rc, "ps_sample_centered_ordered", (PS_OK, PS_NO_PATHS))
        return hist

    def copy(self, which: int) -> np.ndarray:
        n, m = self.n, int(self.stats.m)
        spec = {PS_ARRAY_OFFSETS: (np.int64, (n + 1,)), PS_ARRAY_COLUMNS: (np.int32, (self.nnz,)),
                PS_ARRAY_RANK: (np.int32, (n,)), PS_ARRAY_EDGES: (np.int32, (m, 8)),
                PS_ARRAY_PTAU: (np.uint64, (m,)), PS_ARRAY_PLAMBDA: (np.uint64, (m,))}[which]
        out = np.zeros(spec[1], dtype=spec[0])
        rc = ps_graph_copy(self.handle, which, out.ctypes.data, out.nbytes)
        _check(rc, "ps_graph_copy")
        return out

    def count_exact(self, max_blocks: int = 0, stream=None):
        """Exact counts of the graph: (N1..N6 non-induced, C1..C6 induced, t_e
        per edge as an int32 device tensor in edge order)."""
        import torch
        nbytes = ps_exact_scratch_bytes(self.handle, max_blocks)
        if nbytes == 0:
            raise PathSampleError(PS_ERR_STATE, "ps_exact_scratch_bytes")
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        rc, N, C = ps_count_exact(self.handle, scratch.data_ptr(), nbytes, stream)
        _check(rc, "ps_count_exact")
        m = int(self.stats.m)
        te = scratch[: 4 * m].view(torch.int32) if m else torch.zeros(0, dtype=torch.int32,
                                                                       device=self.device)
        return N, C, te

    def count_adaptive(self, seed: int, target: float, delta: float = 0.01, k0: int = 1 << 16,
                       k_max: int = 1 << 26, motif_mask: int = 0x3F, c1_from_centred: bool = False,
                       stream=None):
        """Samples until the bars are narrow; (k_used, hist6, hist4, est, lo, hi)."""
        h6, h4 = self.new_hist(), self.new_hist()
        rc, k, a, b, est, lo, hi = ps_count_adaptive(
            self.handle, seed, target, delta, k0, k_max, h6.data_ptr(), h4.data_ptr(), motif_mask,
            PS_EST_C1_FROM_CENTRED if c1_from_centred else 0, stream)
        _check(rc, "ps_count_adaptive", (PS_OK, PS_NO_PATHS))
        return k, a, b, est, lo, hi

    def estimate(self, hist6, k3, hist4, kc, delta=0.01):
        h6 = np.asarray(hist6.cpu().numpy() if hasattr(hist6, "cpu") else hist6)[:6]
        h4 = np.asarray(hist4.cpu().numpy() if hasattr(hist4, "cpu") else hist4)[:4]
        rc, est, lo, hi = ps_estimate(self.stats, h6.astype(np.uint64), k3, h4.astype(np.uint64),
                                      kc, delta)
        _check(rc, "ps_estimate", (PS_OK, PS_NO_PATHS))
        return est, lo, hi
