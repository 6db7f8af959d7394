"""Seeded synthetic input graphs (CSR: int64 offsets, int32 sorted columns).

This module produces inputs only.  It holds none of the arithmetic of the
path-sampling method, and both the CUDA library and the CPU oracle read its
output.  The heavy generators (Chung-Lu, R-MAT) are C in ``graphgen.c``,
compiled on first use with gcc; the tiny named graphs used by the closed-form
tests are built here with numpy.

Every graph is a pure function of its parameters (counter-based hashing), so a
test that generates the same graph twice sees the same bytes.
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
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("off", ctypes.POINTER(ctypes.c_int64)),
        ("col", ctypes.POINTER(ctypes.c_int32)),
    ]


def _src_tag() -> str:
    with open(_SRC, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:16]


def build(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so (skipped when up to date)."""
    tag_path = _LIB_PATH + ".tag"
    tag = _src_tag()
    if not force and os.path.exists(_LIB_PATH) and os.path.exists(tag_path):
        with open(tag_path) as f:
            if f.read().strip() == tag:
                return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    with open(tag_path, "w") as f:
        f.write(tag)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.gg_chung_lu.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_int, P(_CSR)]
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_int, P(_CSR)]
            lib.gg_from_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, P(_CSR)]
            lib.gg_chung_lu_weights.argtypes = [ctypes.c_int64, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double,
                                                ctypes.c_void_p, P(ctypes.c_double)]
            lib.gg_free.argtypes = [P(_CSR)]
            lib.gg_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected simple graph in CSR form (both arc directions stored)."""

    off: np.ndarray  # int64 [n+1]
    col: np.ndarray  # int32 [nnz], each row sorted ascending
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.off)


def _take(csr: _CSR, name: str) -> Graph:
    lib = _load()
    try:
        n, nnz = int(csr.n), int(csr.nnz)
        off = np.ctypeslib.as_array(csr.off, shape=(n + 1,)).copy()
        col = (np.ctypeslib.as_array(csr.col, shape=(nnz,)).copy() if nnz > 0
               else np.zeros(0, dtype=np.int32))
    finally:
        lib.gg_free(ctypes.byref(csr))
    return Graph(off=off.astype(np.int64, copy=False), col=col.astype(np.int32, copy=False),
                 name=name)


def chung_lu(n: int, avg_deg: float, gamma: float, w_max: float, seed: int,
             exact_pairs: bool | None = None, permute: bool = True) -> Graph:
    """Chung-Lu graph with power-law expected degrees (see graphgen.c)."""
    lib = _load()
    if exact_pairs is None:
        exact_pairs = n <= 20000
    csr = _CSR()
    rc = lib.gg_chung_lu(n, avg_deg, gamma, w_max, seed, int(exact_pairs), int(permute),
                         ctypes.byref(csr))
    if rc != 0:
        raise ValueError(f"gg_chung_lu failed with {rc}")
    return _take(csr, f"chung_lu(n={n},avg={avg_deg},gamma={gamma},wmax={w_max},seed={seed})")


def chung_lu_weights(n: int, avg_deg: float, gamma: float, w_max: float):
    lib = _load()
    w = np.zeros(n, dtype=np.float64)
    i0 = ctypes.c_double()
    rc = lib.gg_chung_lu_weights(n, avg_deg, gamma, w_max, w.ctypes.data, ctypes.byref(i0))
    if rc != 0:
        raise ValueError("bad Chung-Lu parameters")
    return w, i0.value


def rmat(scale: int, edge_factor: float, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True) -> Graph:
    """R-MAT graph: edge_factor * 2^scale draws, symmetrised and deduplicated."""
    lib = _load()
    csr = _CSR()
    rc = lib.gg_rmat(scale, edge_factor, a, b, c, seed, int(permute), ctypes.byref(csr))
    if rc != 0:
        raise ValueError(f"gg_rmat failed with {rc}")
    return _take(csr, f"rmat(scale={scale},ef={edge_factor},seed={seed})")


def from_pairs(n: int, pairs) -> Graph:
    """Simple undirected graph from an iterable of (u, v) pairs."""
    lib = _load()
    arr = np.asarray(list(pairs) if not isinstance(pairs, np.ndarray) else pairs,
                     dtype=np.int32).reshape(-1, 2)
    pu = np.ascontiguousarray(arr[:, 0])
    pv = np.ascontiguousarray(arr[:, 1])
    csr = _CSR()
    rc = lib.gg_from_pairs(n, pu.shape[0], pu.ctypes.data, pv.ctypes.data, ctypes.byref(csr))
    if rc != 0:
        raise ValueError(f"gg_from_pairs failed with {rc}")
    return _take(csr, f"pairs(n={n})")


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Same graph with vertex v renamed perm[v]."""
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    pairs = np.stack([perm[src], perm[g.col]], axis=1)
    pairs = pairs[pairs[:, 0] < pairs[:, 1]]
    return from_pairs(g.n, pairs)


# --------------------------------------------------------------- named graphs

def path(n: int) -> Graph:
    return from_pairs(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n: int) -> Graph:
    return from_pairs(n, [(i, (i + 1) % n) for i in range(n)])


def complete(n: int) -> Graph:
    return from_pairs(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def star(leaves: int) -> Graph:
    return from_pairs(leaves + 1, [(0, i) for i in range(1, leaves + 1)])


def complete_bipartite(a: int, b: int) -> Graph:
    return from_pairs(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def gnp(n: int, p: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, p) for small test graphs (numpy PCG64 stream)."""
    rs = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, 1)
    keep = rs.random(iu.shape[0]) < p
    return from_pairs(n, np.stack([iu[keep], ju[keep]], axis=1))


def empty(n: int) -> Graph:
    return Graph(off=np.zeros(n + 1, dtype=np.int64), col=np.zeros(0, dtype=np.int32),
                 name=f"empty({n})")


# ----------------------------------------------------- workloads of the method

def chung_lu_5k(seed: int = 1) -> Graph:
    """Chung-Lu, n=5,000, mean expected degree 20, exponent 2.5, max weight 500."""
    return chung_lu(5000, 20.0, 2.5, 500.0, seed)


def rmat20(seed: int = 11) -> Graph:
    """R-MAT scale 20, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05)."""
    return rmat(20, 16.0, 0.57, 0.19, 0.19, seed)


def social_chung_lu_3m(seed: int = 3) -> Graph:
    """Social-network-shaped Chung-Lu: n=3,000,000, exponent 2.1, max weight
    33,000, mean weight 78 (about 117M undirected edges)."""
    return chung_lu(3_000_000, 78.0, 2.1, 33000.0, seed, exact_pairs=False)


def num_threads() -> int:
    return int(_load().gg_num_threads())
