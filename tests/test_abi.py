"""The C interface: the library builds for sm_103a, loads, and exports every
function include/pathsample.h declares.  No GPU needed (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_1411_4942_gb300 import _build
from paper_1411_4942_gb300 import pathsample as ps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ps_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(ps.EXPORTED) <= declared


def test_l2_probe_rejects_bad_arguments_before_any_cuda_call():
    # dummy (never dereferenced) pointers: every case fails the argument checks
    probe = ps.load_library().ps_l2_read_probe
    assert probe(4096, 0, 1, 4096, None) == ps.PS_ERR_ARG       # no bytes
    assert probe(4096, 24, 1, 4096, None) == ps.PS_ERR_ARG      # not a multiple of 16
    assert probe(4104, 32, 1, 4096, None) == ps.PS_ERR_ARG      # buffer not 16-byte aligned
    assert probe(4096, 32, 0, 4096, None) == ps.PS_ERR_ARG      # no passes
    assert probe(None, 32, 1, 4096, None) == ps.PS_ERR_ARG
    assert probe(4096, 32, 1, None, None) == ps.PS_ERR_ARG


def test_built_for_sm_103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_and_workspace_sizes():
    assert ps.ps_strerror(0) == "ok"
    assert "symmetric" in ps.ps_strerror(ps.PS_ERR_ASYMMETRIC)
    a = ps.ps_graph_workspace_bytes(1000, 10000)
    b = ps.ps_graph_workspace_bytes(1000, 20000)
    assert 0 < a < b and a % 256 == 0
    assert ps.ps_graph_workspace_bytes(0, 0) > 0
    assert ps.ps_graph_workspace_bytes(-1, 0) == 0
    assert ps.ps_graph_workspace_bytes(1 << 31, 10) == 0  # labels must fit in int32
    # hubs and guide tables change the size, never the results
    t_off = ps.make_tuning(hub_count=-1, guide_log2_ratio=-1)
    assert ps.ps_graph_workspace_bytes(100000, 1000000, t_off) < ps.ps_graph_workspace_bytes(100000, 1000000)
    assert ps.ps_end_to_end_workspace_bytes(1000, 10000) > a
    # 1024 hub rows over the top 2^20 of 2^22 labels take 128 MB, full-width rows 512 MB
    n, nnz = 1 << 22, 1 << 24
    narrow = ps.ps_graph_workspace_bytes(n, nnz, ps.make_tuning(hub_count=1024, hub_span_log2=20))
    full = ps.ps_graph_workspace_bytes(n, nnz, ps.make_tuning(hub_count=1024, hub_span_log2=-1))
    assert full - narrow == 1024 * 4 * ((n >> 5) - (1 << 15))


def test_ordered_scratch_sizes():
    """Scratch of the draw-ordered samplers: a fixed header plus 11 bytes per
    sample of a chunk (its id in both passes' orders, its bucket byte, its
    high byte in both orders); chunks of 1 .. 2^31."""
    one = ps.ps_ordered_scratch_bytes(1)
    assert one > 0
    assert ps.ps_ordered_scratch_bytes(0) == 0
    assert ps.ps_ordered_scratch_bytes((1 << 31) + 1) == 0
    # 11 bytes per sample: two uint32 orders and three byte arrays
    assert ps.ps_ordered_scratch_bytes(1 << 31) == one - 11 + 11 * (1 << 31)
    for k in (2, 1000, 1 << 24):
        assert ps.ps_ordered_scratch_bytes(k) == one + 11 * (k - 1)
    # nine int32 tuning fields, the last one the hub-row span
    import ctypes
    assert ctypes.sizeof(ps.PsTuning) == 9 * 4
    assert ps.make_tuning(draw_order=-1).draw_order == -1
    assert ps.make_tuning(hub_span_log2=-1).hub_span_log2 == -1
