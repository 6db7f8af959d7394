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
import oracle as O

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


def test_static_prefix_equals_oracle_prefixes():
    # the oracle's own tau / lambda weights in, its own prefixes expected out
    # (two graphs, two calls in a row)
    for g in (gg.chung_lu(4000, 12.0, 2.2, 250.0, 17), gg.rmat(14, 10.0, seed=23)):
        og = O.prepare(g.off, g.col)
        rc, pa, pb = _run_static(og.tau, og.lam)
        assert rc == ps.PS_OK
        assert np.array_equal(pa, og.ptau) and np.array_equal(pb, og.plam)


def test_static_prefix_allocates_nothing():
    """The call's defining property: once the first call on the device has
    done its set-up, calls of any size leave the device's free memory exactly
    as it was (no cudaMalloc, no allocating library routine, no growth of a
    pool).  Every buffer is allocated before the first reading."""
    sizes = (1, 4095, 1 << 16, 3 << 18)
    bufs = []
    for n in sizes:
        a = torch.arange(n, dtype=torch.int64, device="cuda")
        b = torch.ones(n, dtype=torch.int64, device="cuda")
        bufs.append((a, b, torch.empty_like(a), torch.empty_like(b)))
    torch.cuda.synchronize()
    a, b, pa, pb = bufs[0]
    assert ps.ps_prefix_pairs_static(a.data_ptr(), b.data_ptr(), pa.data_ptr(), pb.data_ptr(), 1) == ps.PS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for (a, b, pa, pb), n in zip(bufs, sizes):
            assert ps.ps_prefix_pairs_static(a.data_ptr(), b.data_ptr(), pa.data_ptr(),
                                             pb.data_ptr(), n) == ps.PS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    a, b, pa, pb = bufs[-1]
    n = sizes[-1]
    assert pa.cpu().numpy().tolist() == np.cumsum(np.arange(n)).tolist()
    assert pb.cpu().numpy().tolist() == list(range(1, n + 1))
