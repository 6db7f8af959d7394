"""Batched launch and serving loop on the GPU: every request's class counts
must equal those of the oracle for the same (graph, k, seed, ids) and of the
same request run alone with the plain calls (integer counts, so bit for bit;
estimates to 1e-12 relative)."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1411_4942_gb300 import batch as B  # noqa: E402
from paper_1411_4942_gb300 import pathsample as ps  # noqa: E402
from paper_1411_4942_gb300 import serve as S  # noqa: E402


@pytest.fixture(scope="module")
def graph_set():
    rs = np.random.default_rng(5)
    graphs = []
    for i in range(10):
        scale = int(rs.integers(8, 13))
        g = gg.rmat(scale, float(rs.integers(8, 33)), seed=300 + i)
        # alternate adjacency variants: a batch may mix them
        t = ps.make_tuning(adjacency=(ps.ADJ_HASH, ps.ADJ_SEARCH, ps.ADJ_VTAB)[i % 3])
        graphs.append(ps.Graph(g.off, g.col, tuning=t))
    return B.GraphSet(graphs)


def _plain(gset, reqs):
    h = B.run_plain(gset, reqs)
    torch.cuda.synchronize()
    return h.cpu().numpy().reshape(-1, 6).astype(np.uint64)


def test_batched_equals_plain(graph_set):
    rs = np.random.default_rng(7)
    reqs = B.random_requests(rs, len(graph_set), log2_k=(10, 17))
    want = _plain(graph_set, reqs)
    for cfg in (B.LaunchConfig(256, 1 << 16, 0), B.LaunchConfig(128, 777, 3),
                B.LaunchConfig(512, 1 << 12, 1), B.LaunchConfig(256, 1 << 13, 0, 2),
                B.LaunchConfig(128, 999, 0, 2)):
        run = B.BatchRunner(graph_set, [B.Request(**vars(r)) for r in reqs], cfg)
        run.launch()
        torch.cuda.synchronize()
        assert np.array_equal(run.histograms(), want)


def test_cuda_graph_replay(graph_set):
    rs = np.random.default_rng(8)
    reqs = B.random_requests(rs, len(graph_set), log2_k=(12, 15))
    want = _plain(graph_set, reqs)
    run = B.BatchRunner(graph_set, reqs, B.LaunchConfig(256, 1 << 13))
    run.capture()
    for _ in range(2):
        run.replay()
        torch.cuda.synchronize()
        assert np.array_equal(run.histograms(), want)


def test_autotuner_choice_keeps_results(graph_set):
    import dataclasses
    rs = np.random.default_rng(9)
    reqs = B.random_requests(rs, len(graph_set), log2_k=(12, 15))
    tuner = B.Autotuner(block_sizes=(128, 256), chunks=(1 << 12, 1 << 15), blocks_per_sm=(0,))
    cfg = tuner.tune_launch(graph_set, reqs, budget_samples=1 << 18)
    assert dataclasses.replace(cfg, ordered_min_k=B.NEVER) in tuner.candidates
    assert {c.samples_per_thread for c in tuner.candidates} == {1, 2}
    assert len(tuner.log) == len(tuner.candidates) + len(B.Autotuner.ORDERED_MIN_K)
    run = B.BatchRunner(graph_set, reqs, cfg)
    run.launch()
    torch.cuda.synchronize()
    assert np.array_equal(run.histograms(), _plain(graph_set, reqs))
    g = gg.rmat(11, 16.0, seed=3)
    t = tuner.tune_graph_variant(g.off, g.col, k=1 << 16)
    assert int(t.adjacency) in (ps.ADJ_HASH, ps.ADJ_SEARCH, ps.ADJ_VTAB)
    # hub rows per size bucket; the chosen load-time tuning keeps every count
    hosts = [gg.rmat(10, 8.0, seed=41), gg.rmat(14, 16.0, seed=42)]
    choice = tuner.tune_hubs(hosts, k=1 << 15)
    assert set(choice) == {B.Autotuner.size_bucket(h.m) for h in hosts}
    assert all(c in B.Autotuner.HUB_CHOICES for c in choice.values())
    for h in hosts:
        G = ps.Graph(h.off, h.col, tuning=tuner.graph_tuning(h.m))
        og = O.prepare(h.off, h.col)
        got = G.sample_3paths(1 << 14, 5).cpu().numpy()[:6].astype(np.uint64)
        assert got.tolist() == O.sample_3paths(og, 1 << 14, 5).tolist()


def _sources(n_graphs):
    rs = np.random.default_rng(11)
    out = {}
    for i in range(n_graphs):
        n = int(10 ** rs.uniform(3, 4))
        gamma = float(rs.uniform(2.1, 2.8))
        g = gg.chung_lu(n, 12.0, gamma, (12.0 * n) ** 0.5, 50 + i)
        out[f"g{i}"] = (g.off, g.col)
    return out


@pytest.mark.parametrize("realtime", [True, False])
def test_served_results_equal_requests_alone(realtime):
    sources = _sources(6)
    sizes = [ps.ps_graph_workspace_bytes(len(o) - 1, len(c)) for o, c in sources.values()]
    budget = int(sum(sizes) * 0.6)  # forces evictions between requests
    pool = S.GraphPool(sources, budget)
    server = S.Server(pool, quantum=1 << 13, max_active=64, cfg=B.LaunchConfig(256, 1 << 12))
    rs = np.random.default_rng(12)
    reqs = S.poisson_requests(rs, list(sources), 120, 4000.0, log2_k=(8, 15))
    results, report = server.run(reqs, realtime=realtime)
    assert report["requests"] == len(reqs) == len(results)
    assert report["graph_evictions"] > 0 and pool.used_bytes <= budget
    assert report["latency_p99_ms"] >= report["latency_p50_ms"] > 0
    alone, _ = S.run_sequential(S.GraphPool(sources, 10 * budget), reqs)
    by_id = {rid: (h6, h4, est) for rid, h6, h4, est in alone}
    for r in results:
        h6, h4, est = by_id[r.rid]
        assert r.hist6.tolist() == h6.tolist() and r.hist4.tolist() == h4.tolist()
        np.testing.assert_allclose(r.est, est, rtol=1e-12)


def _oracle_hist(og, sampler, k, seed, first_id=0):
    threads = max(1, min(16, O.max_threads()))
    if sampler == B.SAMPLER_3PATH:
        return O.sample_3paths(og, k, seed, first_id, threads=threads) if og.W else np.zeros(6, np.uint64)
    h = O.sample_centered(og, k, seed, first_id, threads=threads) if og.Lambda else np.zeros(4, np.uint64)
    return np.concatenate([h, np.zeros(2, np.uint64)])


def test_batched_slots_equal_oracle():
    """One batch over nine graphs of uneven size -- eight R-MAT graphs of
    scales 8..12 (the three adjacency variants mixed) and one R-MAT scale-17
    graph of over 2^20 edges -- with per-request k and seeds, ids starting past
    2^32 for some requests: every slot equals the oracle's histogram."""
    rs = np.random.default_rng(31)
    hosts = [gg.rmat(int(rs.integers(8, 13)), float(rs.integers(8, 33)), seed=700 + i) for i in range(8)]
    hosts.append(gg.rmat(17, 16.0, seed=777))
    assert hosts[-1].m >= 1 << 20
    graphs = [ps.Graph(h.off, h.col, tuning=ps.make_tuning(adjacency=(ps.ADJ_HASH, ps.ADJ_SEARCH,
                                                                       ps.ADJ_VTAB)[i % 3]))
              for i, h in enumerate(hosts)]
    gset = B.GraphSet(graphs)
    reqs = B.random_requests(rs, len(graphs), log2_k=(10, 16))
    for i, r in enumerate(reqs):
        if i % 3 == 1:
            r.first_id = (1 << 32) - 1000 + i
    ogs = [O.prepare(h.off, h.col) for h in hosts]
    # one sample per thread; two per thread with the large graph's requests
    # taken by the draw-ordered samplers
    for cfg in (B.LaunchConfig(256, 1 << 12, 0), B.LaunchConfig(256, 1 << 12, 0, 2, ordered_min_k=1 << 10)):
        run = B.BatchRunner(gset, reqs, cfg)
        assert bool(run.ordered) == (cfg.ordered_min_k < B.NEVER)
        run.launch()
        torch.cuda.synchronize()
        got = run.histograms()
        for r in reqs:
            want = _oracle_hist(ogs[r.graph], r.sampler, r.k, r.seed, r.first_id)
            assert got[r.slot].tolist() == want.tolist(), (cfg, r, got[r.slot], want)


@pytest.mark.parametrize("realtime", [True, False])
def test_served_results_equal_oracle(realtime):
    """Every served request (mixed graphs, evictions forced by the budget,
    Poisson arrivals replayed or all at once) against the oracle: both
    histograms bit for bit and the estimates to 1e-12."""
    sources = _sources(6)
    sizes = [ps.ps_graph_workspace_bytes(len(o) - 1, len(c)) for o, c in sources.values()]
    budget = int(sum(sizes) * 0.6)
    pool = S.GraphPool(sources, budget)
    server = S.Server(pool, quantum=1 << 13, max_active=64, cfg=B.LaunchConfig(256, 1 << 12))
    rs = np.random.default_rng(13)
    reqs = S.poisson_requests(rs, list(sources), 60, 4000.0, log2_k=(8, 15))
    results, report = server.run(reqs, realtime=realtime)
    assert report["graph_evictions"] > 0 and len(results) == len(reqs)
    ogs = {key: O.prepare(off, col) for key, (off, col) in sources.items()}
    by_id = {r.rid: r for r in reqs}
    for res in results:
        req = by_id[res.rid]
        og = ogs[req.graph]
        h6 = _oracle_hist(og, B.SAMPLER_3PATH, req.k, req.seed)
        h4 = _oracle_hist(og, B.SAMPLER_CENTRED, req.k, req.seed)[:4]
        assert res.hist6.tolist() == h6.tolist() and res.hist4.tolist() == h4.tolist()
        _, est, lo, hi = O.estimate(og.W, og.Lambda, og.N1, h6, req.k, h4, req.k, 0.01)
        np.testing.assert_allclose(res.est, est, rtol=1e-12)
        np.testing.assert_allclose(res.lo, lo, rtol=1e-12)
        np.testing.assert_allclose(res.hi, hi, rtol=1e-12)
