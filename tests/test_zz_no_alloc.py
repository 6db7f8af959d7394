"""The allocation-free prefix call, for callers that cannot allocate device
memory (a plugin whose host owns all device memory, or a serving process
that reserved its HBM up front).  Its results must equal the prefixes the
ordinary path (ps_load_csr + ps_tau_prefix, which uses a caller workspace)
computes for the same graph, bit for bit, on consecutive calls that reuse the
library's fixed scratch array.

This file is collected last so that a failure here cannot hide others.
"""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1411_4942_gb300 import pathsample as ps  # noqa: E402


def _weights_and_reference(g):
    G = ps.Graph(g.off, g.col)
    rec = G.copy(ps.PS_ARRAY_EDGES).astype(np.uint64)
    du, dv, iu, jv = rec[:, 2], rec[:, 3], rec[:, 4], rec[:, 5]
    tau = (du - 1) * (dv - 1)
    lam = (du - 1 - iu) * (dv - 1 - jv)
    return tau, lam, G.copy(ps.PS_ARRAY_PTAU), G.copy(ps.PS_ARRAY_PLAMBDA)


def _run_static(a, b):
    d_a = torch.from_numpy(a.view(np.int64)).cuda()
    d_b = torch.from_numpy(b.view(np.int64)).cuda()
    d_pa = torch.empty_like(d_a)
    d_pb = torch.empty_like(d_b)
    torch.cuda.synchronize()
    rc = ps.ps_prefix_pairs_static(d_a.data_ptr(), d_b.data_ptr(), d_pa.data_ptr(),
                                   d_pb.data_ptr(), a.shape[0])
    return rc, d_pa.cpu().numpy().view(np.uint64), d_pb.cpu().numpy().view(np.uint64)


def test_static_prefix_matches_workspace_path_on_consecutive_calls():
    # a larger graph first, then a smaller one: the second call must not see
    # anything the first left in the shared scratch array
    for g in (gg.rmat(16, 12.0, seed=21), gg.chung_lu(3000, 10.0, 2.3, 200.0, 5)):
        tau, lam, ptau, plam = _weights_and_reference(g)
        rc, pa, pb = _run_static(tau, lam)
        assert rc == ps.PS_OK
        assert np.array_equal(pa, ptau) and np.array_equal(pb, plam)


def test_static_prefix_limits():
    a = np.ones(4, dtype=np.uint64)
    d = torch.from_numpy(a.view(np.int64)).cuda()
    out = torch.empty_like(d)
    p = d.data_ptr()
    assert ps.ps_prefix_pairs_static(p, p, out.data_ptr(), out.data_ptr(),
                                     ps.PS_PREFIX_STATIC_MAX_ITEMS + 1) == ps.PS_ERR_TOO_LARGE
    assert ps.ps_prefix_pairs_static(p, p, out.data_ptr(), out.data_ptr(), -1) == ps.PS_ERR_ARG
    # sums past 2^64 are reported, not wrapped silently
    big = np.array([1 << 63, 1 << 63, 5], dtype=np.uint64)
    rc, _, _ = _run_static(big, np.ones(3, dtype=np.uint64))
    assert rc == ps.PS_ERR_OVERFLOW
    rc, pa, pb = _run_static(np.arange(10, dtype=np.uint64), np.ones(10, dtype=np.uint64))
    assert rc == ps.PS_OK and pa.tolist() == np.cumsum(np.arange(10)).tolist()
