"""Edge-list ingest on the device (ps_csr_from_edges) against the oracle's
csr_from_edges: offsets and columns bit for bit, from lists with repeats,
both directions and self-loops, up to the R-MAT scale 20 graph."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1411_4942_gb300 import pathsample as ps  # noqa: E402


def _check(n, src, dst):
    off, col = ps.csr_from_edges(n, np.asarray(src, np.int32), np.asarray(dst, np.int32))
    ooff, ocol = O.csr_from_edges(n, src, dst)
    assert np.array_equal(off.cpu().numpy(), ooff)
    assert np.array_equal(col.cpu().numpy(), ocol)
    return off, col


@pytest.mark.parametrize("n,e,seed", [(1, 0, 0), (5, 0, 0), (2, 7, 1), (50, 300, 2),
                                      (1000, 5000, 3), (70000, 400000, 4), (3, 100000, 5)])
def test_ingest_matches_oracle(n, e, seed):
    rs = np.random.Generator(np.random.PCG64(seed))
    _check(n, rs.integers(0, n, e), rs.integers(0, n, e))


def test_ingest_complete_graph_from_messy_list():
    src = [0, 1, 2, 3, 0, 1, 3, 2, 2, 0, 1, 0, 3]
    dst = [1, 0, 3, 2, 2, 3, 0, 1, 2, 3, 1, 1, 3]
    off, col = _check(4, src, dst)
    k4 = gg.complete(4)
    assert np.array_equal(off.cpu().numpy(), k4.off) and np.array_equal(col.cpu().numpy(), k4.col)


def test_ingest_errors():
    s = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    d = torch.tensor([1, 5], dtype=torch.int32, device="cuda")
    nb = ps.ps_ingest_workspace_bytes(3, 2)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    off = torch.empty(4, dtype=torch.int64, device="cuda")
    col = torch.empty(4, dtype=torch.int32, device="cuda")
    rc, _ = ps.ps_csr_from_edges(3, 2, s.data_ptr(), d.data_ptr(), ws.data_ptr(), nb, off.data_ptr(),
                                 col.data_ptr())
    assert rc == ps.PS_ERR_ARG  # id 5 outside [0, 3)
    rc, _ = ps.ps_csr_from_edges(6, 2, s.data_ptr(), d.data_ptr(), ws.data_ptr(), 16, off.data_ptr(),
                                 col.data_ptr())
    assert rc == ps.PS_ERR_WORKSPACE
    rc, _ = ps.ps_csr_from_edges(6, 2, s.data_ptr(), d.data_ptr(), ws.data_ptr() + 8, nb,
                                 off.data_ptr(), col.data_ptr())
    assert rc == ps.PS_ERR_WORKSPACE
    assert ps.ps_ingest_workspace_bytes(-1, 2) == 0


def test_ingest_rmat20_raw_list_then_sampling():
    """The R-MAT scale 20 graph listed as a raw edge list -- every arc, 2^20
    repeats, 2^16 self-loops, shuffled -- comes back as the generator's CSR,
    and the path runs on it unchanged."""
    g = gg.rmat20()
    rs = np.random.Generator(np.random.PCG64(77))
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off))
    dst = g.col.astype(np.int64)
    rep = rs.integers(0, src.shape[0], 1 << 20)
    loops = rs.integers(0, g.n, 1 << 16)
    src = np.concatenate([src, dst[rep], loops])
    dst = np.concatenate([dst, src[rep], loops])
    perm = rs.permutation(src.shape[0])
    src, dst = src[perm].astype(np.int32), dst[perm].astype(np.int32)
    off, col = ps.csr_from_edges(g.n, src, dst)
    assert np.array_equal(off.cpu().numpy(), g.off) and np.array_equal(col.cpu().numpy(), g.col)
    ooff, ocol = O.csr_from_edges(g.n, src, dst)
    assert np.array_equal(ooff, g.off) and np.array_equal(ocol, g.col)
    G = ps.Graph(off, col)
    h = G.sample_3paths(1 << 20, 11)
    assert int(h.sum().item()) == 1 << 20
