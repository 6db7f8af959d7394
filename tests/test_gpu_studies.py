"""Accuracy studies through the batched path (paper_1411_4942_gb300.studies):
one run's histograms and estimates against the oracle, and the behaviour the
paper reports in Section 6 -- errors shrink with k, the error bars hold the
exact counts, the centred sampler beats the 3-path sampler on 4-cycles."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1411_4942_gb300 import batch as B  # noqa: E402
from paper_1411_4942_gb300 import pathsample as ps  # noqa: E402
from paper_1411_4942_gb300 import studies  # noqa: E402


def test_study_chung_lu_5k():
    g = gg.chung_lu_5k()
    G = ps.Graph(g.off, g.col)
    seeds, ks = list(range(1, 9)), [1 << e for e in range(12, 18)]
    res = studies.run({"cl5k": G}, seeds, ks, delta=0.01)["cl5k"]
    og = O.prepare(g.off, g.col)
    _, C = O.exact_counts(og.off, og.col)
    assert res["exact"] == C.tolist()
    rows = res["by_k"]
    # errors shrink with k (first vs last sample size, every motif)
    assert all(b < a for a, b in zip(rows[0]["rel_err"], rows[-1]["rel_err"]))
    # the bars hold the exact counts in most runs (each fails with probability <= 1%)
    assert min(min(r["coverage"]) for r in rows) >= 0.75
    assert np.mean([r["coverage"] for r in rows]) >= 0.97
    # the centred sampler is the more accurate one for 4-cycles (motif 4)
    cen = np.mean([r["rel_err"][3] for r in rows])
    basic = np.mean([r["rel_err_3path_only"][3] for r in rows])
    assert cen < basic
    # one run of the batch against the oracle's replay
    reqs = [B.Request(0, 0, ks[0], 3, slot=0), B.Request(0, 1, ks[0], 3, slot=1)]
    runner = B.BatchRunner(B.GraphSet([G]), reqs, B.LaunchConfig())
    runner.launch()
    h = runner.histograms()
    assert h[0].tolist() == O.sample_3paths(og, ks[0], 3).tolist()
    assert h[1][:4].tolist() == O.sample_centered(og, ks[0], 3).tolist()
    rc, est, lo, hi = ps.ps_estimate_ex(G.stats, h[0], ks[0], h[1][:4], ks[0], 0.01, ps.PS_EST_3PATH_ONLY)
    _, oest, olo, ohi = O.estimate(og.W, og.Lambda, og.N1, h[0], ks[0], h[1][:4], ks[0], 0.01,
                                   three_path_only=True)
    np.testing.assert_allclose(est, oest, rtol=1e-12)
    np.testing.assert_allclose(lo, olo, rtol=1e-12)
    assert "| 2^12 |" in studies.table({"cl5k": res})
