"""The samplers with samples taken in edge-draw order (ps_sample_*_ordered).

Samples of Alg. 1 and Alg. 3 are independent and the histograms are sums, so
the ordered samplers must give exactly the histograms of the plain samplers
and of the CPU oracle for the same (k, seed, first_id), whatever the chunk
size; this checks that bit for bit, plus the error paths.  Small graphs and
chunks take the plain sampler by default, so most cases force the sort with
the tuning's draw_order = 1 (and check the default and -1 give the same).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1411_4942_gb300 import pathsample as ps  # noqa: E402


def _both(G, k, seed, first_id=0, scratch=None):
    """(plain, ordered) histograms of both samplers."""
    out = []
    for ordered in (False, True):
        h6, h4 = G.new_hist(), G.new_hist()
        if not ordered:
            G.sample_3paths(k, seed, first_id, h6)
            G.sample_centered(k, seed, first_id, h4)
        elif scratch is None:
            G.sample_3paths_ordered(k, seed, first_id, h6)
            G.sample_centered_ordered(k, seed, first_id, h4)
        else:
            for fn, h in ((ps.ps_sample_3paths_ordered, h6), (ps.ps_sample_centered_ordered, h4)):
                rc = fn(G.handle, k, seed, first_id, h.data_ptr(), scratch.data_ptr(), scratch.numel())
                assert rc == ps.PS_OK
        torch.cuda.synchronize()
        out.append((h6.cpu().numpy()[:6].tolist(), h4.cpu().numpy()[:4].tolist()))
    return out


@pytest.mark.parametrize("name,make", [
    ("K9", lambda: gg.complete(9)),
    ("gnp300", lambda: gg.gnp(300, 0.06, 3)),
    ("chung_lu_5k", gg.chung_lu_5k),
])
@pytest.mark.parametrize("order", [1, 2])
def test_ordered_equals_oracle(name, make, order):
    g = make()
    og = O.prepare(g.off, g.col)
    G = ps.Graph(g.off, g.col, tuning=ps.make_tuning(draw_order=order))
    k, seed, first = 30000, 17, 123
    h6, h4 = G.new_hist(), G.new_hist()
    G.sample_3paths_ordered(k, seed, first, h6)
    G.sample_centered_ordered(k, seed, first, h4)
    torch.cuda.synchronize()
    assert h6.cpu().numpy()[:6].tolist() == O.sample_3paths(og, k, seed, first).tolist()
    assert h4.cpu().numpy()[:4].tolist() == O.sample_centered(og, k, seed, first).tolist()


@pytest.mark.parametrize("k", [1, 31, 4097, (1 << 18) + 5])
@pytest.mark.parametrize("order", [2, 1, 0, -1])
def test_ordered_equals_plain(k, order):
    g = gg.chung_lu(20000, 15.0, 2.3, 800.0, 9)
    G = ps.Graph(g.off, g.col, tuning=ps.make_tuning(draw_order=order))
    plain, ordered = _both(G, k, 5, first_id=1 << 40)
    assert plain == ordered
    assert sum(ordered[0]) == k and sum(ordered[1]) == k


@pytest.mark.parametrize("adjacency", [1, 2, 3])
@pytest.mark.parametrize("block", [128, 512, 1024])
def test_ordered_every_variant(adjacency, block):
    g = gg.chung_lu(5000, 12.0, 2.2, 600.0, 4)
    G = ps.Graph(g.off, g.col, tuning=ps.make_tuning(adjacency=adjacency, block_size=block, draw_order=1))
    plain, ordered = _both(G, 50000, 21, first_id=3)
    assert plain == ordered


def test_ordered_in_chunks():
    """Scratch for 1000 samples: k = 12345 runs 13 sorted chunks, ragged last;
    scratch for one sample sorts chunks of one; by default a chunk of 2^18 + 7
    is sorted and the ragged last one (12324) is below the cut-off."""
    g = gg.gnp(2000, 0.01, 4)
    for order in (1, 2):  # one pass, two passes
        G = ps.Graph(g.off, g.col, tuning=ps.make_tuning(draw_order=order))
        nb = ps.ps_ordered_scratch_bytes(1000)
        sc = torch.empty(nb, dtype=torch.uint8, device="cuda")
        plain, ordered = _both(G, 12345, 77, first_id=9, scratch=sc)
        assert plain == ordered
        one = torch.empty(ps.ps_ordered_scratch_bytes(1), dtype=torch.uint8, device="cuda")
        plain, ordered = _both(G, 300, 78, scratch=one)
        assert plain == ordered
    r = gg.rmat(17, 16.0, 0.57, 0.19, 0.19, 3)  # about 2^20 edges: the default sorts
    R = ps.Graph(r.off, r.col)
    assert R.stats.m >= 1 << 20, R.stats.m
    nb = ps.ps_ordered_scratch_bytes((1 << 18) + 7)
    sc = torch.empty(nb, dtype=torch.uint8, device="cuda")
    plain, ordered = _both(R, 3 * ((1 << 18) + 7) + 12324, 77, first_id=9, scratch=sc)
    assert plain == ordered


@pytest.mark.parametrize("order", [0, 2])
def test_ordered_rmat20_matches_plain(order):
    """The R-MAT-20 graph and size: 2^24 samples per sampler, one chunk, in
    the default order and the two-pass order."""
    g = gg.rmat20()
    G = ps.Graph(g.off, g.col, tuning=ps.make_tuning(draw_order=order))
    plain, ordered = _both(G, 1 << 24, 11)
    assert plain == ordered


def test_ordered_errors_and_degenerate():
    assert ps.ps_ordered_scratch_bytes(0) == 0
    assert ps.ps_ordered_scratch_bytes((1 << 31) + 1) == 0
    assert ps.ps_ordered_scratch_bytes(2) > ps.ps_ordered_scratch_bytes(1) > 0
    g = gg.gnp(100, 0.1, 2)
    G = ps.Graph(g.off, g.col)
    nb = ps.ps_ordered_scratch_bytes(64)
    sc = torch.empty(nb + 16, dtype=torch.uint8, device="cuda")
    h = G.new_hist()
    f = ps.ps_sample_3paths_ordered
    assert f(G.handle, 10, 1, 0, h.data_ptr(), None, nb) == ps.PS_ERR_WORKSPACE
    assert f(G.handle, 10, 1, 0, h.data_ptr(), sc.data_ptr() + 4, nb) == ps.PS_ERR_WORKSPACE
    assert f(G.handle, 10, 1, 0, h.data_ptr(), sc.data_ptr(), ps.ps_ordered_scratch_bytes(1) - 1) == \
        ps.PS_ERR_WORKSPACE
    assert f(G.handle, 10, 1, 0, None, sc.data_ptr(), nb) == ps.PS_ERR_ARG
    assert f(G.handle, 0, 1, 0, h.data_ptr(), sc.data_ptr(), nb) == ps.PS_OK
    torch.cuda.synchronize()
    assert int(h.sum()) == 0
    # a star has no 3-path (W = 0) and no centred 3-path: nothing is added
    s = gg.star(6)
    S = ps.Graph(s.off, s.col)
    h6, h4 = S.new_hist(), S.new_hist()
    assert f(S.handle, 10, 1, 0, h6.data_ptr(), sc.data_ptr(), nb) == ps.PS_NO_PATHS
    assert ps.ps_sample_centered_ordered(S.handle, 10, 1, 0, h4.data_ptr(), sc.data_ptr(), nb) == \
        ps.PS_NO_PATHS
    torch.cuda.synchronize()
    assert int(h6.sum()) == 0 and int(h4.sum()) == 0
    # before ps_tau_prefix
    off = torch.as_tensor(g.off).cuda()
    col = torch.as_tensor(g.col).cuda()
    wsb = ps.ps_graph_workspace_bytes(g.n, g.nnz, None)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    rc, hd = ps.ps_load_csr(g.n, g.nnz, off.data_ptr(), col.data_ptr(), ws.data_ptr(), wsb, None, None)
    assert rc == ps.PS_OK
    assert f(hd, 10, 1, 0, h.data_ptr(), sc.data_ptr(), nb) == ps.PS_ERR_STATE
    ps.ps_graph_free(hd)
    torch.cuda.synchronize()
