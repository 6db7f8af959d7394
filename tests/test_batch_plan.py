"""Host logic of the batched launch: work-item planning (CPU only)."""
import numpy as np

from paper_1411_4942_gb300 import batch as B
from paper_1411_4942_gb300 import pathsample as ps


def test_items_cover_every_request_exactly_once():
    rs = np.random.default_rng(1)
    reqs = B.random_requests(rs, 7, log2_k=(3, 12))
    for chunk in (1, 5, 64, 4096):
        items, slots = B.plan_items([B.Request(**vars(r)) for r in reqs], chunk)
        assert slots == len(reqs)
        assert items.dtype == ps.WORK_DTYPE and np.all(items["count"] <= chunk)
        # ids of each (slot) form exactly [first_id, first_id + k)
        for r in reqs:
            sel = items[items["slot"] == r.slot]
            assert np.all(sel["graph"] == r.graph) and np.all(sel["sampler"] == r.sampler)
            assert np.all(sel["seed"] == r.seed)
            ids = np.concatenate([np.arange(f, f + c) for f, c in zip(sel["first_id"], sel["count"])])
            assert np.array_equal(np.sort(ids), np.arange(r.first_id, r.first_id + r.k))
        # grouped by graph (each graph's items contiguous), most work first
        g = items["graph"].astype(np.int64)
        starts = np.flatnonzero(np.r_[True, g[1:] != g[:-1]])
        assert len(starts) == len(set(g.tolist()))
        work = [int(items["count"][g == gg_].sum()) for gg_ in g[starts]]
        assert work == sorted(work, reverse=True)


def test_slots_assigned_when_missing():
    reqs = [B.Request(0, 0, 10, 1), B.Request(1, 1, 10, 2), B.Request(0, 1, 3, 3, slot=5)]
    items, slots = B.plan_items(reqs, 4)
    assert slots == 6 and reqs[0].slot == 0 and reqs[1].slot == 1


def test_poisson_requests():
    from paper_1411_4942_gb300 import serve as S
    rs = np.random.default_rng(2)
    reqs = S.poisson_requests(rs, ["a", "b"], 20000, 2000.0)
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert abs(arr[-1] / 20000 - 1 / 2000.0) < 0.05 / 2000.0 * 10
    ks = np.array([r.k for r in reqs])
    assert set(np.log2(ks).astype(int)) == set(range(14, 23))
