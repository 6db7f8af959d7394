"""The library's host estimator (ps_estimate, no GPU involved) against the
oracle's, bit for bit, over histograms from every regime of Corollary 5.3's
bisection: counts of 0, 1, k - 1 and k, tiny and large fractions, small and
huge k.  The library stops each bisection once its midpoint rounds to an end
of the interval; the oracle always halves 200 times; the bars must still be
the same doubles."""
import numpy as np
import pytest

import oracle as O

ps = pytest.importorskip("paper_1411_4942_gb300.pathsample")


def _lib():
    try:
        ps.load_library(build_if_missing=False)
    except Exception as e:  # library not built in this checkout
        pytest.skip(f"library not built: {e}")


def _cases():
    rs = np.random.Generator(np.random.PCG64(99))
    for k in (1, 2, 7, 1000, 1 << 20, 1 << 24, (1 << 40) + 3):
        for _ in range(25):
            h6 = np.zeros(6, dtype=np.uint64)
            h4 = np.zeros(4, dtype=np.uint64)
            for h in (h6, h4):
                left = k
                for i in rs.permutation(len(h)):
                    pick = int(rs.choice([0, 1, left, max(left - 1, 0),
                                          int(rs.integers(0, left + 1)),
                                          int(left * 10.0 ** -rs.uniform(0, 12))]))
                    pick = min(pick, left)
                    h[i] = pick
                    left -= pick
                h[int(rs.integers(0, len(h)))] += left
            yield k, h6, h4


def test_host_estimate_matches_oracle_bit_for_bit():
    _lib()
    W, Lam, N1 = 40830043145588, 969788827508, (1 << 70) + 12345
    st = ps.PsStats()
    st.W, st.Lambda = W, Lam
    st.N1_lo, st.N1_hi = N1 & ((1 << 64) - 1), N1 >> 64
    n = 0
    for delta in (0.01, 1e-9):
        for k, h6, h4 in _cases():
            rc, est, lo, hi = ps.ps_estimate(st, h6, k, h4, k, delta)
            orc, oest, olo, ohi = O.estimate(W, Lam, N1, h6, k, h4, k, delta)
            assert rc == orc
            assert est.tobytes() == oest.tobytes(), (k, h6, h4)
            assert lo.tobytes() == olo.tobytes(), (k, h6, h4, lo, olo)
            assert hi.tobytes() == ohi.tobytes(), (k, h6, h4, hi, ohi)
            n += 1
    assert n == 2 * 7 * 25
