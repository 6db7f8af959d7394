"""CPU oracle for the path-sampling method -- TEST INFRASTRUCTURE.

A plain, slow statement in C (``oracle.c``) of what the method computes:
validation and degree-ordered relabelling of the graph, the tau / lambda edge
weights and their exact prefixes, both samplers replayed draw for draw, the
estimates and their error bars, and exact induced counts (brute force and the
non-induced counts of Eq. (1)).  Only the tests, the smoke check and the CPU
baseline of the benchmark may use it; the CUDA library never does, and the
two share no code.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

OK, NO_PATHS = 0, 1
ERR_ARG, ERR_NOT_SIMPLE, ERR_ASYMMETRIC, ERR_OVERFLOW, ERR_NOMEM = -1, -2, -3, -5, -9

# Eq. (1): A[i][j] = copies of motif i in motif j (1 = 3-star ... 6 = 4-clique)
EQ1_MATRIX = np.array([
    [1, 0, 1, 0, 2, 4],
    [0, 1, 2, 4, 6, 12],
    [0, 0, 1, 0, 4, 12],
    [0, 0, 0, 1, 1, 3],
    [0, 0, 0, 0, 1, 6],
    [0, 0, 0, 0, 0, 1],
], dtype=np.int64)
A2 = EQ1_MATRIX[1]            # 3-paths per motif (row 2)
B_CENTRED = np.array([0, 0, 0, 1, 1, 3])  # Lemma 4.2


def _src_tag() -> str:
    with open(_SRC, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:16]


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (skipped when up to date)."""
    tag_path = _LIB_PATH + ".tag"
    tag = _src_tag()
    if not force and os.path.exists(_LIB_PATH) and os.path.exists(tag_path):
        with open(tag_path) as f:
            if f.read().strip() == tag:
                return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    with open(tag_path, "w") as f:
        f.write(tag)
    return _LIB_PATH


class _Graph(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("m", ctypes.c_int64),
        ("off", ctypes.c_void_p), ("col", ctypes.c_void_p),
        ("eu", ctypes.c_void_p), ("ev", ctypes.c_void_p),
        ("eiu", ctypes.c_void_p), ("ejv", ctypes.c_void_p),
        ("ptau", ctypes.c_void_p), ("plam", ctypes.c_void_p),
        ("W", ctypes.c_uint64), ("Lambda", ctypes.c_uint64),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            V, I64, U64, U32, I32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_int)
            G = ctypes.POINTER(_Graph)
            sig = {
                "or_validate": ([I64, I64, V, V], I32),
                "or_canonicalize": ([I64, I64, V, V, V, V, V], I32),
                "or_num_edges": ([I64, V, V], I64),
                "or_edge_table": ([I64, V, V, V, V, V, V, V, V, V, V, V], I32),
                "or_philox4x32_10": ([V, V, V], None),
                "or_lemire64_step": ([U64, U64, V], I32),
                "or_lemire32_step": ([U32, U32, V], I32),
                "or_draw_r": ([U64, U64, U32, U64], U64),
                "or_draw_small": ([U64, U64, U32, U32, U32], U32),
                "or_upper_bound": ([V, I64, U64], I64),
                "or_classify_3path": ([G, I64, U32, U32], I32),
                "or_classify_centered": ([G, I64, U32, U32], I32),
                "or_sample_3paths": ([G, U64, U64, U64, V], None),
                "or_sample_centered": ([G, U64, U64, U64, V], None),
                "or_sample_mt": ([G, I32, U64, U64, U64, V, I32], I32),
                "or_max_threads": ([], I32),
                "or_enumerate_3path": ([G, V], None),
                "or_enumerate_centered": ([G, V], None),
                "or_chernoff_bounds": ([U64, U64, ctypes.c_double, V, V], None),
                "or_estimate": ([U64, U64, U64, U64, V, U64, V, U64, ctypes.c_double, V, V, V],
                                I32),
                "or_estimate_ex": ([U64, U64, U64, U64, V, U64, V, U64, ctypes.c_double, I32, V, V,
                                    V], I32),
                "or_bruteforce_counts": ([I64, V, V, V], I32),
                "or_exact_counts": ([I64, V, V, V, V], I32),
                "or_triangles_per_edge": ([I64, V, V, I64, V, V, V], I32),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _csr(off, col):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return off, col


# ------------------------------------------------------------------- graph

def validate(off, col) -> int:
    """Section 2: 0 if (off, col) is an undirected simple graph, else an error code."""
    off, col = _csr(off, col)
    n = off.shape[0] - 1
    return int(_load().or_validate(n, col.shape[0], _p(off), _p(col)))


def csr_from_edges(n: int, src, dst):
    """Section 2's input from a raw edge list: the undirected simple graph on
    vertices [0, n) with an edge {u, v} for every listed pair with u != v
    (self-loops dropped, repeats and both directions merged), as (off, col)
    with both arcs of every edge and each row ascending."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.shape != dst.shape or (src.size and (min(src.min(), dst.min()) < 0 or
                                                max(src.max(), dst.max()) >= n)):
        raise ValueError("edge ids outside [0, n)")
    keep = src != dst
    a, b = np.minimum(src, dst)[keep], np.maximum(src, dst)[keep]
    pairs = np.unique(a * n + b)                 # each undirected edge once
    u, v = pairs // n, pairs % n
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    order = np.lexsort((cols, rows))             # by row, then column
    rows, cols = rows[order], cols[order]
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return off, cols.astype(np.int32)


def canonicalize(off, col):
    """Section 4 order: returns (rank, coff, ccol) of the relabelled graph."""
    off, col = _csr(off, col)
    n = off.shape[0] - 1
    rank = np.zeros(max(n, 0), dtype=np.int32)
    coff = np.zeros(n + 1, dtype=np.int64)
    ccol = np.zeros(col.shape[0], dtype=np.int32)
    rc = _load().or_canonicalize(n, col.shape[0], _p(off), _p(col), _p(rank), _p(coff), _p(ccol))
    if rc != 0:
        raise RuntimeError(f"or_canonicalize: {rc}")
    return rank, coff, ccol


@dataclass
class OracleGraph:
    """Canonical graph plus the edge table of Sections 3-4."""

    rank: np.ndarray
    off: np.ndarray
    col: np.ndarray
    eu: np.ndarray
    ev: np.ndarray
    eiu: np.ndarray
    ejv: np.ndarray
    tau: np.ndarray
    lam: np.ndarray
    ptau: np.ndarray
    plam: np.ndarray
    W: int
    Lambda: int
    N1: int
    status: int

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])

    def struct(self) -> _Graph:
        s = _Graph()
        s.n, s.m = self.n, self.m
        s.off, s.col = _p(self.off), _p(self.col)
        s.eu, s.ev, s.eiu, s.ejv = _p(self.eu), _p(self.ev), _p(self.eiu), _p(self.ejv)
        s.ptau, s.plam = _p(self.ptau), _p(self.plam)
        s.W, s.Lambda = self.W, self.Lambda
        return s


def prepare(off, col) -> OracleGraph:
    """Validate, relabel and build the tau / lambda tables (raises on invalid input)."""
    off, col = _csr(off, col)
    rc = validate(off, col)
    if rc != 0:
        raise ValueError(f"invalid graph: status {rc}")
    lib = _load()
    rank, coff, ccol = canonicalize(off, col)
    n = coff.shape[0] - 1
    m = int(lib.or_num_edges(n, _p(coff), _p(ccol)))
    z = lambda dt: np.zeros(m, dtype=dt)  # noqa: E731
    eu, ev, eiu, ejv = z(np.int32), z(np.int32), z(np.int32), z(np.int32)
    tau, lam, ptau, plam = z(np.uint64), z(np.uint64), z(np.uint64), z(np.uint64)
    totals = np.zeros(4, dtype=np.uint64)
    st = lib.or_edge_table(n, _p(coff), _p(ccol), _p(eu), _p(ev), _p(eiu), _p(ejv), _p(tau),
                           _p(lam), _p(ptau), _p(plam), _p(totals))
    if st not in (OK, ERR_OVERFLOW):
        raise RuntimeError(f"or_edge_table: {st}")
    n1 = int(totals[2]) | (int(totals[3]) << 64)
    return OracleGraph(rank, coff, ccol, eu, ev, eiu, ejv, tau, lam, ptau, plam,
                       int(totals[0]), int(totals[1]), n1, int(st))


# ------------------------------------------------------------ random draws

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def lemire64_step(x: int, s: int):
    r = ctypes.c_uint64()
    ok = _load().or_lemire64_step(x, s, ctypes.byref(r))
    return (int(r.value) if ok else None)


def lemire32_step(x: int, s: int):
    r = ctypes.c_uint32()
    ok = _load().or_lemire32_step(x, s, ctypes.byref(r))
    return (int(r.value) if ok else None)


def draw_r(seed: int, sample_id: int, stream: int, W: int) -> int:
    return int(_load().or_draw_r(seed, sample_id, stream, W))


def draw_small(seed: int, sample_id: int, stream: int, slot: int, s: int) -> int:
    return int(_load().or_draw_small(seed, sample_id, stream, slot, s))


def upper_bound(P: np.ndarray, r: int) -> int:
    P = np.ascontiguousarray(P, dtype=np.uint64)
    return int(_load().or_upper_bound(_p(P), P.shape[0], r))


# --------------------------------------------------------------- samplers

def classify_3path(g: OracleGraph, j: int, a: int, b: int) -> int:
    s = g.struct()
    return int(_load().or_classify_3path(ctypes.byref(s), j, a, b))


def classify_centered(g: OracleGraph, j: int, a: int, b: int) -> int:
    s = g.struct()
    return int(_load().or_classify_centered(ctypes.byref(s), j, a, b))


def sample_3paths(g: OracleGraph, k: int, seed: int, first_id: int = 0,
                  threads: int = 1) -> np.ndarray:
    """Alg. 2's sampling loop: class counts [triangle, 3-path, tailed, 4-cycle,
    chordal, clique] over sample ids first_id .. first_id + k - 1."""
    hist = np.zeros(6, dtype=np.uint64)
    s = g.struct()
    lib = _load()
    if threads <= 1:
        lib.or_sample_3paths(ctypes.byref(s), k, seed, first_id, _p(hist))
    elif g.W > 0:
        rc = lib.or_sample_mt(ctypes.byref(s), 0, k, seed, first_id, _p(hist), threads)
        if rc != 0:
            raise RuntimeError(rc)
    return hist


def sample_centered(g: OracleGraph, k: int, seed: int, first_id: int = 0,
                    threads: int = 1) -> np.ndarray:
    """Alg. 4's sampling loop: counts [not centred, 4-cycle, chordal, clique]."""
    hist = np.zeros(4, dtype=np.uint64)
    s = g.struct()
    lib = _load()
    if threads <= 1:
        lib.or_sample_centered(ctypes.byref(s), k, seed, first_id, _p(hist))
    elif g.Lambda > 0:
        buf = np.zeros(6, dtype=np.uint64)
        rc = lib.or_sample_mt(ctypes.byref(s), 1, k, seed, first_id, _p(buf), threads)
        if rc != 0:
            raise RuntimeError(rc)
        hist += buf[:4]
    return hist


def max_threads() -> int:
    return int(_load().or_max_threads())


def enumerate_3path(g: OracleGraph) -> np.ndarray:
    cnt = np.zeros(6, dtype=np.uint64)
    s = g.struct()
    _load().or_enumerate_3path(ctypes.byref(s), _p(cnt))
    return cnt


def enumerate_centered(g: OracleGraph) -> np.ndarray:
    cnt = np.zeros(4, dtype=np.uint64)
    s = g.struct()
    _load().or_enumerate_centered(ctypes.byref(s), _p(cnt))
    return cnt


# ------------------------------------------------------------- estimation

def chernoff_bounds(count: int, k: int, delta: float):
    pl, pu = ctypes.c_double(), ctypes.c_double()
    _load().or_chernoff_bounds(count, k, delta, ctypes.byref(pl), ctypes.byref(pu))
    return pl.value, pu.value


def estimate(W: int, Lambda: int, N1: int, hist6, k3: int, hist4, kc: int,
             delta: float = 0.01, c1_from_centred: bool = False, three_path_only: bool = False):
    """Estimates and error bars of all six induced counts (motif 1..6);
    c1_from_centred feeds C1 with the centred sampler's C5 and C6;
    three_path_only reports Alg. 2's own C4..C6 (3-path sampler)."""
    h6 = np.ascontiguousarray(hist6, dtype=np.uint64)
    h4 = np.ascontiguousarray(hist4, dtype=np.uint64)
    est, lo, hi = (np.zeros(6), np.zeros(6), np.zeros(6))
    st = _load().or_estimate_ex(W, Lambda, N1 & ((1 << 64) - 1), N1 >> 64, _p(h6), k3, _p(h4), kc,
                                delta, int(bool(c1_from_centred)) | (2 if three_path_only else 0),
                                _p(est), _p(lo), _p(hi))
    return int(st), est, lo, hi


def adaptive(g: OracleGraph, seed: int, target: float, delta: float, k0: int, k_max: int,
             motif_mask: int = 0x3F, c1_from_centred: bool = False, threads: int = 1):
    """Sampling until the Corollary 5.3 bars are narrow: both samplers over ids
    [0, k) for k = k0, 2 k0, ... capped at k_max; every look's bars at
    delta / (number of looks the schedule allows), so the union bound holds
    over the early stop; stops when every selected motif i has
    max(hi - est, est - lo) <= target * |est|, or at k_max.
    Returns (k, hist6, hist4, est, lo, hi, status)."""
    looks, k = 1, k0
    while k < k_max:
        k = k_max if k > k_max // 2 else 2 * k
        looks += 1
    h6 = np.zeros(6, dtype=np.uint64)
    h4 = np.zeros(4, dtype=np.uint64)
    done, k = 0, k0
    while True:
        if g.W > 0:
            h6 += sample_3paths(g, k - done, seed, done, threads)
        if g.Lambda > 0:
            h4 += sample_centered(g, k - done, seed, done, threads)
        done = k
        st, est, lo, hi = estimate(g.W, g.Lambda, g.N1, h6, k, h4, k, delta / looks,
                                   c1_from_centred)
        met = all(max(hi[i] - est[i], est[i] - lo[i]) <= target * abs(est[i])
                  for i in range(6) if (motif_mask >> i) & 1)
        if met or st == NO_PATHS or k == k_max:
            return done, h6, h4, est, lo, hi, st
        k = k_max if k > k_max // 2 else 2 * k


def bruteforce_counts(off, col) -> np.ndarray:
    """Induced counts C1..C6 by visiting every 4-vertex subset (tiny graphs)."""
    off, col = _csr(off, col)
    C = np.zeros(6, dtype=np.uint64)
    rc = _load().or_bruteforce_counts(off.shape[0] - 1, _p(off), _p(col), _p(C))
    if rc != 0:
        raise ValueError(f"or_bruteforce_counts: {rc}")
    return C.astype(np.int64)


def triangles_per_edge(off, col, eu, ev) -> np.ndarray:
    """|N(u) ∩ N(v)| for each given edge (u, v); rows must be sorted."""
    off, col = _csr(off, col)
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    t = np.zeros(eu.shape[0], dtype=np.uint32)
    rc = _load().or_triangles_per_edge(off.shape[0] - 1, _p(off), _p(col), eu.shape[0], _p(eu),
                                       _p(ev), _p(t))
    if rc != 0:
        raise ValueError(f"or_triangles_per_edge: {rc}")
    return t


def exact_counts(off, col):
    """(N1..N6 non-induced, C1..C6 induced) via Eq. (1); rows must be sorted."""
    off, col = _csr(off, col)
    N = np.zeros(6, dtype=np.uint64)
    C = np.zeros(6, dtype=np.int64)
    rc = _load().or_exact_counts(off.shape[0] - 1, _p(off), _p(col), _p(N), _p(C))
    if rc != 0:
        raise RuntimeError(f"or_exact_counts: {rc}")
    return N.astype(np.int64), C
