"""GPU parity of the estimator options and of sampling until the error bars
are narrow (ps_estimate_ex, ps_count_adaptive) against the oracle: the same
stopping k, bit-identical histograms, estimates to 1e-12 relative."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1411_4942_gb300 import pathsample as ps  # noqa: E402

EST_RTOL = 1e-12


@pytest.mark.parametrize("c1_from_centred", [False, True])
def test_estimate_options_match_oracle(c1_from_centred):
    g = gg.chung_lu(3000, 10.0, 2.2, 300.0, 8)
    og = O.prepare(g.off, g.col)
    G = ps.Graph(g.off, g.col)
    for k in (1000, 1 << 16):
        h6 = G.sample_3paths(k, 9).cpu().numpy()[:6].astype(np.uint64)
        h4 = G.sample_centered(k, 9).cpu().numpy()[:4].astype(np.uint64)
        flags = ps.PS_EST_C1_FROM_CENTRED if c1_from_centred else 0
        rc, est, lo, hi = ps.ps_estimate_ex(G.stats, h6, k, h4, k, 0.01, flags)
        ost, oest, olo, ohi = O.estimate(og.W, og.Lambda, og.N1, h6, k, h4, k, 0.01, c1_from_centred)
        assert rc == ost
        for a, b in ((est, oest), (lo, olo), (hi, ohi)):
            np.testing.assert_allclose(a, b, rtol=EST_RTOL)
    assert ps.ps_estimate_ex(G.stats, h6, k, h4, k, 0.01, 4)[0] == ps.PS_ERR_ARG


@pytest.mark.parametrize("case", [
    ("chung_lu_5k", 0.02, 0x3F, False),
    ("chung_lu_5k", 0.01, 0b11, True),
    ("cl3000", 1e-9, 0x3F, False),   # unreachable: runs to k_max
    ("cl3000", 10.0, 0x3F, False),   # met at the first look
    ("K7", 0.05, 0b100000, False),   # cliques only
    ("C9", 0.05, 0x3F, False),       # zero counts never meet a relative target
])
def test_adaptive_matches_oracle(case):
    name, target, mask, cen = case
    g = {"chung_lu_5k": gg.chung_lu_5k, "cl3000": lambda: gg.chung_lu(3000, 10.0, 2.2, 300.0, 8),
         "K7": lambda: gg.complete(7), "C9": lambda: gg.cycle(9)}[name]()
    og = O.prepare(g.off, g.col)
    G = ps.Graph(g.off, g.col)
    k0, k_max = 1 << 12, 1 << 20
    k, h6, h4, est, lo, hi = G.count_adaptive(17, target, 0.01, k0, k_max, mask, cen)
    ok, oh6, oh4, oest, olo, ohi, _ = O.adaptive(og, 17, target, 0.01, k0, k_max, mask, cen,
                                                 threads=max(1, O.max_threads()))
    assert k == ok
    assert h6.tolist() == oh6.tolist() and h4.tolist() == oh4.tolist()
    for a, b in ((est, oest), (lo, olo), (hi, ohi)):
        np.testing.assert_allclose(a, b, rtol=EST_RTOL)


def test_adaptive_arguments():
    g = gg.complete(6)
    G = ps.Graph(g.off, g.col)
    h6, h4 = G.new_hist(), G.new_hist()
    call = lambda **kw: ps.ps_count_adaptive(G.handle, kw.get("seed", 1), kw.get("target", 0.1), 0.01,  # noqa: E731
                                             kw.get("k0", 64), kw.get("k_max", 1024), h6.data_ptr(),
                                             h4.data_ptr(), kw.get("mask", 0x3F), kw.get("flags", 0))[0]
    assert call() in (ps.PS_OK, ps.PS_NO_PATHS)
    assert call(k0=0) == ps.PS_ERR_ARG
    assert call(k0=2048) == ps.PS_ERR_ARG
    assert call(mask=0x40) == ps.PS_ERR_ARG
    assert call(flags=4) == ps.PS_ERR_ARG
    assert call(target=0.0) == ps.PS_ERR_ARG
