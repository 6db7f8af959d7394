"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these compare the oracle with itself: each checks it against a
printed value (Eq. (1), Lemma 4.2, the Philox known answers), a closed form,
an exact identity (Claims 3.1 / 4.3 with Theorem 3.2), brute force on tiny
graphs, or a distributional property.  All run on the CPU.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

MOTIF_EDGES = {
    1: [(0, 1), (0, 2), (0, 3)],                          # 3-star
    2: [(0, 1), (1, 2), (2, 3)],                          # 3-path
    3: [(0, 1), (1, 2), (2, 0), (2, 3)],                  # tailed triangle
    4: [(0, 1), (1, 2), (2, 3), (3, 0)],                  # 4-cycle
    5: [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)],          # chordal 4-cycle
    6: [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)],  # 4-clique
}


def _read_rows(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _triangles(g):
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for v in range(g.n):
        A[v, g.col[g.off[v]:g.off[v + 1]]] = 1
    return int(np.trace(A @ A @ A)) // 6


# ------------------------------------------------------------------ Philox

def test_philox_known_answers(golden_dir):
    rows = _read_rows(os.path.join(golden_dir, "philox4x32_10_kat.txt"))
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_draw_r_uses_words_0_1_of_block_0():
    seed, W = 0x123456789ABCDEF, 10 ** 15 + 7
    for sid in range(50):
        w = O.philox4x32_10([sid & 0xFFFFFFFF, sid >> 32, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        x = (int(w[1]) << 32) | int(w[0])
        r = O.lemire64_step(x, W)
        if r is not None:
            assert O.draw_r(seed, sid, 0, W) == r


def test_draw_walks_attempts_on_rejection():
    # W = 2^63 + 1 rejects about half of all 64-bit words; the draw must then
    # take the same word pair of block t = 1, 2, ...
    seed, W = 99, (1 << 63) + 1
    seen_reject = 0
    for sid in range(200):
        for t in range(64):
            w = O.philox4x32_10([sid, 0, t, 1], [seed, 0])
            r = O.lemire64_step((int(w[1]) << 32) | int(w[0]), W)
            if r is not None:
                break
            seen_reject += 1
        assert O.draw_r(seed, sid, 1, W) == r
    assert seen_reject > 50
    s = (1 << 31) + 1
    for sid in range(200):
        for t in range(64):
            w = O.philox4x32_10([sid, 0, t, 0], [seed, 0])
            r = O.lemire32_step(int(w[3]), s)
            if r is not None:
                break
        assert O.draw_small(seed, sid, 0, 3, s) == r


# ------------------------------------------------------------------ Lemire

def test_lemire_small_cases():
    # s = 3: 2^32 mod 3 = 1, so exactly x = 0 is rejected
    assert O.lemire32_step(0, 3) is None
    assert O.lemire32_step(1, 3) == 0
    assert O.lemire32_step(0xFFFFFFFF, 3) == 2
    assert O.lemire32_step(0x55555556, 3) == 1
    # s = 1 always yields 0 and never rejects
    for x in (0, 1, 12345, 0xFFFFFFFF):
        assert O.lemire32_step(x, 1) == 0
    # s = 2^k: 2^32 mod s = 0, no rejection, result = top k bits
    assert O.lemire32_step(0xDEADBEEF, 1 << 8) == 0xDE
    assert O.lemire64_step(0xDEADBEEF00000000, 1 << 16) == 0xDEAD
    assert O.lemire64_step(0, 3) is None


@pytest.mark.parametrize("bits", [32, 64])
def test_lemire_removes_multiply_shift_bias(bits):
    # s = 3 * 2^(bits-2): plain multiply-shift maps 2 inputs to every y = 0
    # mod 3 and 1 input to the others (P[y%3==0] = 1/2); exact rejection
    # makes it 1/3 and accepts 3/4 of the words.
    rs = np.random.Generator(np.random.PCG64(5))
    s = 3 << (bits - 2)
    n = 60000
    xs = rs.integers(0, 1 << bits, size=n, dtype=np.uint64 if bits == 64 else np.uint64)
    acc, zero = 0, 0
    for x in xs:
        r = O.lemire64_step(int(x), s) if bits == 64 else O.lemire32_step(int(x) & 0xFFFFFFFF, s)
        if r is None:
            continue
        assert 0 <= r < s
        acc += 1
        zero += (r % 3 == 0)
    assert abs(acc / n - 0.75) < 0.01
    assert abs(zero / acc - 1 / 3) < 0.012


def test_small_draws_uniform_chi_square():
    s, k = 7, 70000
    counts = np.zeros(s)
    for sid in range(k):
        counts[O.draw_small(42, sid, 0, 2, s)] += 1
    chi2 = float(((counts - k / s) ** 2 / (k / s)).sum())
    assert chi2 < 30.0  # 6 dof: P(chi2 > 30) < 1e-4


# ------------------------------------------------- inverse-CDF edge choice

@pytest.mark.parametrize("maker", [lambda: gg.complete(5), lambda: gg.gnp(9, 0.5, 3),
                                   lambda: gg.complete_bipartite(2, 4)])
def test_upper_bound_gives_each_edge_tau_of_W(maker):
    g = maker()
    og = O.prepare(g.off, g.col)
    hits = np.zeros(og.m, dtype=np.int64)
    for r in range(og.W):
        hits[O.upper_bound(og.ptau, r)] += 1
    assert np.array_equal(hits, og.tau.astype(np.int64))  # P(e) = tau_e / W exactly


# ------------------------------------------------------ relabelling order

def _canonical_checks(g):
    rank, coff, ccol = O.canonicalize(g.off, g.col)
    n = g.n
    assert sorted(rank.tolist()) == list(range(n))
    d = g.degrees()
    inv = np.empty(n, dtype=np.int64)
    inv[rank] = np.arange(n)
    # labels ordered by (degree, input id)
    keys = [(int(d[inv[r]]), int(inv[r])) for r in range(n)]
    assert keys == sorted(keys)
    # same edge set under the relabelling, rows ascending
    orig = {(int(rank[v]), int(rank[w])) for v in range(n) for w in g.col[g.off[v]:g.off[v + 1]]}
    canon = set()
    for r in range(n):
        row = ccol[coff[r]:coff[r + 1]]
        assert np.all(np.diff(row) > 0)
        canon |= {(r, int(x)) for x in row}
    assert orig == canon


def test_canonical_relabel_order():
    for seed in range(5):
        _canonical_checks(gg.gnp(30, 0.2, seed))
    _canonical_checks(gg.star(6))
    _canonical_checks(gg.chung_lu(300, 8.0, 2.3, 60.0, 4))


def test_lambda_from_order_definition():
    # Section 4: L_{u,v} = neighbours of u after v in the order, evaluated on
    # the input labels without relabelling
    for seed in range(4):
        g = gg.gnp(25, 0.3, seed)
        d = g.degrees()
        key = lambda x: (int(d[x]), int(x))  # noqa: E731
        lam = 0
        for u in range(g.n):
            for v in g.col[g.off[u]:g.off[u + 1]]:
                if u < v:
                    Luv = sum(1 for w in g.col[g.off[u]:g.off[u + 1]] if key(w) > key(v))
                    Lvu = sum(1 for w in g.col[g.off[v]:g.off[v + 1]] if key(w) > key(u))
                    lam += Luv * Lvu
        W = sum((int(d[u]) - 1) * (int(d[v]) - 1) for u in range(g.n)
                for v in g.col[g.off[u]:g.off[u + 1]] if u < v)
        og = O.prepare(g.off, g.col)
        assert og.Lambda == lam and og.W == W
        assert og.N1 == sum(math.comb(int(x), 3) for x in d)


# ------------------------------------------------------------- validation

def test_validation_codes():
    g = gg.cycle(5)
    assert O.validate(g.off, g.col) == O.OK
    col = g.col.copy()
    col[0] = 0  # vertex 0 lists itself
    assert O.validate(g.off, col) == O.ERR_NOT_SIMPLE
    col = g.col.copy()
    col[1] = col[0]  # repeated neighbour
    assert O.validate(g.off, col) == O.ERR_NOT_SIMPLE
    col = g.col.copy()
    col[0] = 2  # 0 -> 2 without 2 -> 0 (and 1 -> 0 without 0 -> 1)
    assert O.validate(g.off, col) == O.ERR_ASYMMETRIC
    col = g.col.copy()
    col[0] = 9
    assert O.validate(g.off, col) == O.ERR_ARG
    off = g.off.copy()
    off[-1] += 1
    assert O.validate(off, g.col) == O.ERR_ARG
    # unsorted rows are accepted
    col = g.col.copy()
    col[0], col[1] = col[1], col[0]
    assert O.validate(g.off, col) == O.OK


# ------------------------------------------------------ Eq. (1), Lemma 4.2

def test_eq1_matrix_from_motif_graphs(golden_dir):
    M = np.array(_read_rows(os.path.join(golden_dir, "eq1_matrix.txt")), dtype=np.int64)
    assert np.array_equal(M, O.EQ1_MATRIX)
    for j, edges in MOTIF_EDGES.items():
        g = gg.from_pairs(4, edges)
        N, C = O.exact_counts(g.off, g.col)
        assert np.array_equal(N, M[:, j - 1]), j
        e = np.zeros(6, dtype=np.int64)
        e[j - 1] = 1
        assert np.array_equal(C, e)
        assert np.array_equal(O.bruteforce_counts(g.off, g.col), e)


def test_sampler_outcomes_per_motif(golden_dir):
    B = {int(r[0]): int(r[1]) for r in _read_rows(os.path.join(golden_dir,
                                                               "centred_paths_per_motif.txt"))}
    for j, edges in MOTIF_EDGES.items():
        for perm in itertools.permutations(range(4)):
            g = gg.from_pairs(4, [(perm[a], perm[b]) for a, b in edges])
            og = O.prepare(g.off, g.col)
            c6 = O.enumerate_3path(og).astype(np.int64)
            exp = np.zeros(6, dtype=np.int64)
            if j >= 2:
                exp[j - 1] = O.EQ1_MATRIX[1, j - 1]
            exp[0] = 3 * _triangles(g)
            assert np.array_equal(c6, exp), (j, perm)
            c4 = O.enumerate_centered(og).astype(np.int64)
            cent = c4[1:].tolist()
            want = [B.get(4, 0) if j == 4 else 0, B.get(5, 0) if j == 5 else 0,
                    B.get(6, 0) if j == 6 else 0]
            assert cent == want, (j, perm)
            assert int(c4.sum()) == og.Lambda


# -------------------------------------------- exact outcome distribution

def _check_exact_distribution(g):
    og = O.prepare(g.off, g.col)
    C = O.bruteforce_counts(g.off, g.col)
    c6 = O.enumerate_3path(og).astype(np.int64)
    assert int(c6.sum()) == og.W
    # Claim 3.1 + Theorem 3.2: W P[class i] = A_{2,i} C_i; triangles 3T
    assert c6[0] == 3 * _triangles(g)
    assert np.array_equal(c6[1:], O.EQ1_MATRIX[1, 1:] * C[1:])
    # Claim 4.3 + Lemma 4.2: Lambda P[class i] = B_i C_i
    c4 = O.enumerate_centered(og).astype(np.int64)
    assert int(c4.sum()) == og.Lambda
    assert np.array_equal(c4[1:], O.B_CENTRED[3:] * C[3:])
    return og, C


def test_exact_distribution_all_graphs_on_5_vertices():
    pairs = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        _check_exact_distribution(gg.from_pairs(5, edges))


def test_exact_distribution_random_graphs():
    rs = np.random.Generator(np.random.PCG64(17))
    for t in range(40):
        n = int(rs.integers(6, 13))
        g = gg.gnp(n, float(rs.uniform(0.25, 0.8)), 1000 + t)
        g = gg.relabel(g, rs.permutation(n))
        _check_exact_distribution(g)


def test_exact_counts_match_bruteforce():
    rs = np.random.Generator(np.random.PCG64(3))
    for t in range(25):
        n = int(rs.integers(8, 41))
        g = gg.gnp(n, float(rs.uniform(0.1, 0.7)), 500 + t)
        N, C = O.exact_counts(g.off, g.col)
        assert np.array_equal(C, O.bruteforce_counts(g.off, g.col))
        assert np.array_equal(O.EQ1_MATRIX @ C, N)


def _edge_triangles(g):
    og = O.prepare(g.off, g.col)
    return og, O.triangles_per_edge(og.off, og.col, og.eu, og.ev).astype(np.int64)


def test_triangles_per_edge_closed_forms():
    for n in (3, 4, 7):
        _, t = _edge_triangles(gg.complete(n))
        assert (t == n - 2).all()
    for n in (4, 5, 9):
        _, t = _edge_triangles(gg.cycle(n))
        assert (t == 0).all()
    k = 6  # wheel: hub 0 joined to the rim cycle 1..k
    pairs = [(0, i) for i in range(1, k + 1)] + [(i, i % k + 1) for i in range(1, k + 1)]
    og, t = _edge_triangles(gg.from_pairs(k + 1, pairs))
    hub = og.rank[0]
    spoke = (og.eu == hub) | (og.ev == hub)
    assert (t[spoke] == 2).all() and (t[~spoke] == 1).all()


def test_triangles_per_edge_bruteforce():
    rs = np.random.Generator(np.random.PCG64(11))
    for trial in range(12):
        n = int(rs.integers(6, 40))
        g = gg.gnp(n, float(rs.uniform(0.1, 0.7)), 900 + trial)
        og, t = _edge_triangles(g)
        A = np.zeros((n, n), dtype=np.int64)
        for v in range(n):
            A[v, og.col[og.off[v]:og.off[v + 1]]] = 1
        common = np.array([sum(A[u, w] * A[v, w] for w in range(n)) for u, v in zip(og.eu, og.ev)])
        assert np.array_equal(t, common)
        assert int(t.sum()) == 3 * _triangles(g)
        N, _ = O.exact_counts(og.off, og.col)
        assert int(N[4]) == int((t * (t - 1) // 2).sum())  # chordal 4-cycles: triangle pairs


# -------------------------------------------------------- closed forms

def _run(g, k=4000, seed=7):
    og = O.prepare(g.off, g.col)
    h6 = O.sample_3paths(og, k, seed)
    h4 = O.sample_centered(og, k, seed)
    st, est, lo, hi = O.estimate(og.W, og.Lambda, og.N1, h6, k, h4, k)
    return og, h6, h4, st, est


def test_path_graph():
    for n in (4, 5, 9):
        og, h6, h4, st, est = _run(gg.path(n))
        assert og.W == n - 3
        assert h6.tolist() == [0, 4000, 0, 0, 0, 0]
        assert est[1] == n - 3 and est[0] == 0  # C2 exact; paths have no 3-star
        assert np.all(est[2:] == 0)


def test_cycle_graphs():
    og, h6, h4, st, est = _run(gg.cycle(4))
    assert og.W == 4 and og.Lambda == 1
    assert h6.tolist() == [0, 0, 0, 4000, 0, 0] and h4.tolist() == [0, 4000, 0, 0]
    assert est.tolist() == [0, 0, 0, 1, 0, 0]
    for n in (5, 8):
        og, h6, h4, st, est = _run(gg.cycle(n))
        assert og.W == n and h6.tolist() == [0, 4000, 0, 0, 0, 0]
        assert int(h4[1:].sum()) == 0
        assert est.tolist() == [0, n, 0, 0, 0, 0]


def test_complete_bipartite():
    for a, b in ((2, 2), (2, 5), (3, 4), (4, 6)):
        og, h6, h4, st, est = _run(gg.complete_bipartite(a, b))
        c4 = math.comb(a, 2) * math.comb(b, 2)
        assert h6.tolist() == [0, 0, 0, 4000, 0, 0]
        assert h4.tolist() == [0, 4000, 0, 0] and og.Lambda == c4
        assert est[3] == c4
        assert est[0] == a * math.comb(b, 3) + b * math.comb(a, 3)
        assert est[1] == 0 and est[2] == 0 and est[4] == 0 and est[5] == 0


def test_star_and_triangle():
    og, h6, h4, st, est = _run(gg.star(7))
    assert og.W == 0 and og.Lambda == 0 and st == O.NO_PATHS
    assert h6.sum() == 0 and est.tolist() == [math.comb(7, 3), 0, 0, 0, 0, 0]
    og, h6, h4, st, est = _run(gg.complete(3))
    assert og.W == 3 and h6.tolist() == [4000, 0, 0, 0, 0, 0]
    assert np.all(est == 0)


def test_complete_graph_closed_forms():
    n = 9
    og = O.prepare(*[gg.complete(n).off, gg.complete(n).col])
    assert og.W == math.comb(n, 2) * (n - 2) ** 2
    assert og.Lambda == sum((n - 1 - v) * (n - 2 - u) for u in range(n) for v in range(u + 1, n))
    c6 = O.enumerate_3path(og)
    assert c6[0] * (n - 2) == og.W and c6[5] == 12 * math.comb(n, 4)
    c4 = O.enumerate_centered(og)
    assert c4[3] == 3 * math.comb(n, 4) and c4[1] == 0 and c4[2] == 0
    k = 90000
    h6 = O.sample_3paths(og, k, 3)
    assert h6[1:5].sum() == 0  # only cliques among 4-vertex classes
    p0 = 1 / (n - 2)
    assert abs(int(h6[0]) - k * p0) < 5 * math.sqrt(k * p0 * (1 - p0))


# ---------------------------------------------------- statistical pins

def test_sampler_frequencies_match_exact_probabilities():
    # Theorem 3.2: E[count_i] = k A_{2,i} C_i / W (and the centred analogue);
    # every class stays within 5 standard deviations
    for seed, g in ((1, gg.gnp(14, 0.45, 8)), (2, gg.chung_lu(200, 10.0, 2.4, 40.0, 5))):
        og = O.prepare(g.off, g.col)
        k = 200000
        p6 = O.enumerate_3path(og).astype(np.float64) / og.W
        p4 = O.enumerate_centered(og).astype(np.float64) / og.Lambda
        h6 = O.sample_3paths(og, k, seed).astype(np.float64)
        h4 = O.sample_centered(og, k, seed).astype(np.float64)
        for h, p in ((h6, p6), (h4, p4)):
            sd = np.sqrt(k * p * (1 - p))
            assert np.all(np.abs(h - k * p) <= 5 * sd + 1e-9), (h, k * p)


def test_estimates_inside_chernoff_bars():
    # Corollary 5.3 with delta = 0.01 (the 99% bars of Section 6)
    for t in range(8):
        g = gg.gnp(30, 0.35, 40 + t)
        og = O.prepare(g.off, g.col)
        C = O.bruteforce_counts(g.off, g.col)
        k = 100000
        h6 = O.sample_3paths(og, k, 100 + t)
        h4 = O.sample_centered(og, k, 200 + t)
        st, est, lo, hi = O.estimate(og.W, og.Lambda, og.N1, h6, k, h4, k, 0.01)
        assert np.all(lo <= C + 1e-6) and np.all(C <= hi + 1e-6), (C, lo, hi)
        assert np.all(lo <= est + 1e-6) and np.all(est <= hi + 1e-6)


def test_ideal_histograms_give_exact_counts():
    # With the exact outcome counts as histograms (k = W, kc = Lambda), the
    # estimators of Alg. 2 / Alg. 4 return the exact induced counts.
    for t in range(10):
        g = gg.gnp(16, 0.5, 70 + t)
        og = O.prepare(g.off, g.col)
        C = O.bruteforce_counts(g.off, g.col)
        c6 = O.enumerate_3path(og)
        c4 = O.enumerate_centered(og)
        st, est, lo, hi = O.estimate(og.W, og.Lambda, og.N1, c6, og.W, c4, og.Lambda)
        assert np.allclose(est, C, rtol=1e-12, atol=1e-9)
        # the centred-fed 3-star identity is exact on exact inputs too
        st, est, lo, hi = O.estimate(og.W, og.Lambda, og.N1, c6, og.W, c4, og.Lambda,
                                     c1_from_centred=True)
        assert np.allclose(est, C, rtol=1e-12, atol=1e-9)


def test_c1_variant_changes_only_c1():
    g = gg.gnp(40, 0.3, 12)
    og = O.prepare(g.off, g.col)
    h6, h4 = O.sample_3paths(og, 20000, 3), O.sample_centered(og, 20000, 3)
    _, a, alo, ahi = O.estimate(og.W, og.Lambda, og.N1, h6, 20000, h4, 20000)
    _, b, blo, bhi = O.estimate(og.W, og.Lambda, og.N1, h6, 20000, h4, 20000, c1_from_centred=True)
    assert np.array_equal(a[1:], b[1:]) and np.array_equal(alo[1:], blo[1:])
    assert a[0] != b[0]


# ------------------------------------------------------- adaptive sample size

def test_adaptive_schedule_and_stop_rule():
    g = gg.chung_lu(400, 8.0, 2.4, 60.0, 9)
    og = O.prepare(g.off, g.col)
    k0, k_max, delta, target = 1 << 10, 1 << 17, 0.01, 0.05
    k, h6, h4, est, lo, hi, st = O.adaptive(og, 5, target, delta, k0, k_max, motif_mask=0b11)
    # the histograms equal one run of k ids
    assert np.array_equal(h6, O.sample_3paths(og, k, 5)) and np.array_equal(h4, O.sample_centered(og, k, 5))
    # it stopped at the first look of the schedule where C1 and C2 met the target
    looks = [k0 << i for i in range(8)]  # 2^10 .. 2^17
    assert k in looks
    for kk in looks[:looks.index(k) + 1]:
        _, e, l, h = O.estimate(og.W, og.Lambda, og.N1, O.sample_3paths(og, kk, 5), kk,
                                O.sample_centered(og, kk, 5), kk, delta / len(looks))
        met = all(max(h[i] - e[i], e[i] - l[i]) <= target * abs(e[i]) for i in (0, 1))
        assert met == (kk == k)
    # unreachable target: runs to k_max; trivial target: stops at k0
    assert O.adaptive(og, 5, 1e-9, delta, k0, k_max)[0] == k_max
    assert O.adaptive(og, 5, 1e9, delta, k0, k_max)[0] == k0
    # k_max not a power-of-two multiple of k0 is the last look
    assert O.adaptive(og, 5, 1e-9, delta, 1000, 5000)[0] == 5000


def test_adaptive_bars_cover_exact_counts():
    g = gg.gnp(30, 0.35, 41)
    og = O.prepare(g.off, g.col)
    C = O.bruteforce_counts(g.off, g.col)
    for seed in range(6):
        k, _, _, est, lo, hi, _ = O.adaptive(og, seed, 0.02, 0.01, 1 << 10, 1 << 16)
        assert ((lo <= C) & (C <= hi)).all(), (seed, k, est, C)


# ---------------------------------------------------------- error bars

def test_chernoff_roots():
    for count, k in ((37, 1000), (1, 50), (990, 1000), (12345, 100000)):
        a = count / k
        pl, pu = O.chernoff_bounds(count, k, 0.01)
        assert 0 < pl < a < pu < 1
        for p in (pl, pu):
            D = a * math.log(a / p) + (1 - a) * math.log((1 - a) / (1 - p))
            assert math.isclose(math.exp(-k * D), 0.01, rel_tol=1e-9)
    pl, pu = O.chernoff_bounds(0, 500, 0.01)
    assert pl == 0 and math.isclose((1 - pu) ** 500, 0.01, rel_tol=1e-12)
    pl, pu = O.chernoff_bounds(500, 500, 0.01)
    assert pu == 1 and math.isclose(pl ** 500, 0.01, rel_tol=1e-12)


def test_chernoff_width_matches_normal_limit():
    # D(a, p) ~ (a - p)^2 / (2 a (1 - a)) near p = a, so for large k the
    # half-width tends to sqrt(2 a (1 - a) ln(1/delta) / k)
    a, k, delta = 0.2, 10 ** 9, 0.01
    pl, pu = O.chernoff_bounds(int(a * k), k, delta)
    w = math.sqrt(2 * a * (1 - a) * math.log(1 / delta) / k)
    assert abs((pu - a) / w - 1) < 1e-3 and abs((a - pl) / w - 1) < 1e-3


def test_threaded_oracle_equals_single_thread():
    g = gg.chung_lu(400, 12.0, 2.3, 60.0, 9)
    og = O.prepare(g.off, g.col)
    for first in (0, 12345):
        a = O.sample_3paths(og, 30001, 5, first)
        b = O.sample_3paths(og, 30001, 5, first, threads=4)
        assert np.array_equal(a, b)
        a = O.sample_centered(og, 30001, 5, first)
        b = O.sample_centered(og, 30001, 5, first, threads=3)
        assert np.array_equal(a, b)
    # split ranges compose
    whole = O.sample_3paths(og, 20000, 8)
    parts = O.sample_3paths(og, 7000, 8) + O.sample_3paths(og, 13000, 8, 7000)
    assert np.array_equal(whole, parts)


def test_stored_oracle_values(golden_dir):
    # regression fixture written by tests/golden/make_golden.py (oracle only)
    import json
    with open(os.path.join(golden_dir, "oracle_values.json")) as f:
        stored = json.load(f)
    for name, rec in stored.items():
        g = {"complete9": lambda: gg.complete(9), "gnp40": lambda: gg.gnp(40, 0.3, 12),
             "chung_lu_2000": lambda: gg.chung_lu(2000, 12.0, 2.4, 150.0, 21)}[name]()
        og = O.prepare(g.off, g.col)
        assert (og.m, og.W, og.Lambda, og.N1) == (rec["m"], rec["W"], rec["Lambda"], rec["N1"])
        assert O.sample_3paths(og, rec["k"], rec["seed"]).tolist() == rec["hist6"]
        assert O.sample_centered(og, rec["k"], rec["seed"]).tolist() == rec["hist4"]
        assert O.exact_counts(g.off, g.col)[1].tolist() == rec["exact_C"]


# --------------------------------------------------------- edge-list ingest

def test_csr_from_edges_closed_form():
    # K4 listed with repeats, both directions and self-loops
    src = [0, 1, 2, 3, 0, 1, 3, 2, 2, 0, 1, 0, 3]
    dst = [1, 0, 3, 2, 2, 3, 0, 1, 2, 3, 1, 1, 3]
    off, col = O.csr_from_edges(4, src, dst)
    k4 = gg.complete(4)
    assert np.array_equal(off, k4.off) and np.array_equal(col, k4.col)
    off, col = O.csr_from_edges(3, [], [])
    assert off.tolist() == [0, 0, 0, 0] and col.size == 0
    with pytest.raises(ValueError):
        O.csr_from_edges(3, [0], [3])


def test_csr_from_edges_matches_generator_and_validates():
    rs = np.random.Generator(np.random.PCG64(5))
    for trial in range(10):
        n = int(rs.integers(1, 300))
        e = int(rs.integers(0, 4 * n))
        src = rs.integers(0, n, e)
        dst = rs.integers(0, n, e)
        off, col = O.csr_from_edges(n, src, dst)
        assert O.validate(off, col) == 0
        keep = src != dst
        ref = gg.from_pairs(n, np.stack([src[keep], dst[keep]], 1))
        assert np.array_equal(off, ref.off) and np.array_equal(col, ref.col)
        # every listed pair is an edge and every edge was listed
        listed = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist()) if a != b}
        got = {(u, int(v)) for u in range(n) for v in col[off[u]:off[u + 1]] if u < v}
        assert listed == got


def test_three_path_only_estimates():
    # Alg. 2 estimates every motif with a 3-path: on exact outcome histograms
    # its C4..C6 are exact too, and the flag leaves C1..C3 alone
    for t in range(5):
        g = gg.gnp(16, 0.5, 170 + t)
        og = O.prepare(g.off, g.col)
        C = O.bruteforce_counts(g.off, g.col)
        c6, c4 = O.enumerate_3path(og), O.enumerate_centered(og)
        _, a, _, _ = O.estimate(og.W, og.Lambda, og.N1, c6, og.W, c4, og.Lambda, three_path_only=True)
        assert np.allclose(a, C, rtol=1e-12, atol=1e-9)
    h6, h4 = O.sample_3paths(og, 5000, 1), O.sample_centered(og, 5000, 1)
    _, a, _, _ = O.estimate(og.W, og.Lambda, og.N1, h6, 5000, h4, 5000)
    _, b, _, _ = O.estimate(og.W, og.Lambda, og.N1, h6, 5000, h4, 5000, three_path_only=True)
    assert np.array_equal(a[:3], b[:3])


def test_stored_rmat20_exact_counts_are_consistent():
    """The stored exact counts of the R-MAT-20 benchmark graph (written by
    tests/golden/make_exact_rmat20.py from the oracle alone) satisfy Eq. (1)
    between the non-induced N and the induced C, N_1 = sum_v C(d_v, 3) from the
    degrees, and N_2 <= W (N_2 = W - 3T, Section 3) with W from the degrees of
    every edge's endpoints."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "exact_counts_rmat20.json")
    if not os.path.exists(path):
        pytest.skip("tests/golden/exact_counts_rmat20.json not written yet")
    with open(path) as f:
        ref = json.load(f)
    N = np.array(ref["N"], dtype=object)
    C = np.array(ref["C"], dtype=object)
    A = O.EQ1_MATRIX.astype(object)
    assert (A.dot(C) == N).all()
    g = gg.rmat20()
    deg = np.diff(g.off).astype(object)
    assert N[0] == sum(d * (d - 1) * (d - 2) // 6 for d in deg)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    up = src < g.col
    d = np.diff(g.off).astype(np.int64)
    W = int(((d[src[up]] - 1) * (d[g.col[up]] - 1)).sum())
    assert 0 <= W - N[1] and (W - N[1]) % 3 == 0
