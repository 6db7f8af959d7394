"""GPU exact counter (ps_count_exact) against the oracle: the non-induced counts
N_1..N_6 of Eq. (1), the induced counts C_1..C_6 and the triangles of every
edge must match bit for bit; at R-MAT scale 20, sampled edges and identities
that hold at any size (plus the stored oracle counts when present)."""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1411_4942_gb300 import pathsample as ps  # noqa: E402

GRAPHS = {
    "K7": lambda: gg.complete(7),
    "C4": lambda: gg.cycle(4),
    "C9": lambda: gg.cycle(9),
    "P6": lambda: gg.path(6),
    "K3,5": lambda: gg.complete_bipartite(3, 5),
    "star9": lambda: gg.star(9),
    "gnp60": lambda: gg.gnp(60, 0.3, 5),
    "gnp200": lambda: gg.gnp(200, 0.08, 6),
    "cl3000": lambda: gg.chung_lu(3000, 10.0, 2.2, 300.0, 8),
    "rmat12": lambda: gg.rmat(12, 8.0, seed=4),
}


def _oracle_counts(g):
    og = O.prepare(g.off, g.col)
    N, C = O.exact_counts(og.off, og.col)
    t = O.triangles_per_edge(og.off, og.col, og.eu, og.ev)
    return og, N, C, t


def _check(g, tuning=None, max_blocks=0):
    og, N, C, t = _oracle_counts(g)
    G = ps.Graph(g.off, g.col, tuning=tuning)
    gN, gC, te = G.count_exact(max_blocks=max_blocks)
    assert gN.astype(np.int64).tolist() == N.tolist()
    assert gC.tolist() == C.tolist()
    assert np.array_equal(te.cpu().numpy().astype(np.uint32), t)
    return G


@pytest.mark.parametrize("name", list(GRAPHS))
def test_exact_counts_match_oracle(name):
    _check(GRAPHS[name]())


@pytest.mark.parametrize("adjacency", [ps.ADJ_HASH, ps.ADJ_SEARCH, ps.ADJ_VTAB])
def test_exact_counts_every_adjacency_variant(adjacency):
    for g in (gg.chung_lu(3000, 10.0, 2.2, 300.0, 8), gg.rmat(12, 8.0, seed=4)):
        _check(g, tuning=ps.make_tuning(adjacency=adjacency))


def test_exact_counts_with_one_counter_block():
    _check(gg.rmat(12, 8.0, seed=4), max_blocks=1)


def test_exact_counts_chung_lu_5k():
    """The small configuration (Chung-Lu n = 5000, seed 1) in full."""
    _check(gg.chung_lu_5k())


def test_exact_counts_degenerate():
    for g in (gg.empty(5), gg.path(2), gg.star(2)):
        G = ps.Graph(g.off, g.col)
        N, C, _ = G.count_exact()
        assert N.tolist() == [0] * 6 and C.tolist() == [0] * 6


def test_exact_count_errors():
    g = gg.complete(6)
    G = ps.Graph(g.off, g.col)
    nbytes = ps.ps_exact_scratch_bytes(G.handle, 1)
    assert nbytes > 0
    buf = torch.empty(nbytes + 512, dtype=torch.uint8, device="cuda")
    rc, _, _ = ps.ps_count_exact(G.handle, buf.data_ptr(), nbytes - 1)
    assert rc == ps.PS_ERR_WORKSPACE
    rc, _, _ = ps.ps_count_exact(G.handle, buf.data_ptr() + 8, nbytes)
    assert rc == ps.PS_ERR_WORKSPACE
    rc, N, C = ps.ps_count_exact(G.handle, buf.data_ptr(), nbytes)
    assert rc == ps.PS_OK and C.tolist() == [0, 0, 0, 0, 0, 15]
    # a graph that has not been through the prefix step
    off = torch.as_tensor(g.off).cuda()
    col = torch.as_tensor(g.col).cuda()
    wsb = ps.ps_graph_workspace_bytes(g.n, g.nnz, None)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    rc, h = ps.ps_load_csr(g.n, g.nnz, off.data_ptr(), col.data_ptr(), ws.data_ptr(), wsb, None, None)
    assert rc == ps.PS_OK
    assert ps.ps_exact_scratch_bytes(h, 0) == 0
    rc, _, _ = ps.ps_count_exact(h, buf.data_ptr(), nbytes)
    assert rc == ps.PS_ERR_STATE
    ps.ps_graph_free(h)
    torch.cuda.synchronize()


def test_rmat20_exact_counts():
    """R-MAT scale 20 (seed 11): triangles of 4096 random edges against the
    oracle one by one, identities that hold at any size, the sampled
    estimates inside their error bars around the exact counts, and the
    stored oracle counts when the golden file is present."""
    g = gg.rmat20()
    G = ps.Graph(g.off, g.col)
    N, C, te = G.count_exact()
    te = te.cpu().numpy().astype(np.int64)
    rec = G.copy(ps.PS_ARRAY_EDGES)
    off, col = G.copy(ps.PS_ARRAY_OFFSETS), G.copy(ps.PS_ARRAY_COLUMNS)
    rs = np.random.Generator(np.random.PCG64(2024))
    pick = rs.choice(rec.shape[0], size=4096, replace=False)
    t = O.triangles_per_edge(off, col, rec[pick, 0], rec[pick, 1])
    assert np.array_equal(te[pick], t.astype(np.int64))
    st = G.stats
    T3 = int(te.sum())
    assert T3 % 3 == 0
    assert int(N[1]) == int(st.W) - T3  # N_2 = W - 3T
    assert int(N[0]) == st.N1
    assert int(N[4]) == int((te * (te - 1) // 2).sum())
    assert (C >= 0).all()
    assert np.array_equal(O.EQ1_MATRIX @ C, N.astype(np.int64))
    # estimates from 2^24 samples per sampler inside 99.99% bars around the truth
    k = 1 << 24
    h6 = G.sample_3paths(k, 11, 0)
    h4 = G.sample_centered(k, 11, 0)
    est, lo, hi = G.estimate(h6.cpu().numpy()[:6], k, h4.cpu().numpy()[:4], k, delta=1e-4)
    assert (lo <= C).all() and (C <= hi).all(), (est, lo, hi, C)
    golden = os.path.join(os.path.dirname(__file__), "golden", "exact_counts_rmat20.json")
    if os.path.exists(golden):
        with open(golden) as f:
            ref = json.load(f)
        assert N.astype(np.int64).tolist() == ref["N"]
        assert C.tolist() == ref["C"]
