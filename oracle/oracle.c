/*
 * oracle.c -- TEST INFRASTRUCTURE.  A plain, slow, single-threaded CPU
 * statement of the path-sampling method of Jha, Seshadhri & Pinar, "Path
 * Sampling: A Fast and Provable Method for Estimating 4-Vertex Subgraph
 * Counts".  It exists to check the CUDA library: only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may call it.  It shares no
 * code, header or table with the library.
 *
 * Every random draw of the method is replayed exactly, so the library's class
 * histograms must equal the ones computed here bit for bit.  The replay rules
 * are the readings below of steps the paper leaves open.
 *
 * Readings of the paper used here:
 *  R1 Motif numbering follows the matrix of Eq. (1): 1 = 3-star, 2 = 3-path,
 *     3 = tailed triangle, 4 = 4-cycle, 5 = chordal 4-cycle, 6 = 4-clique.
 *  R2 The order of Section 4 (u before v iff d_u < d_v, ties by smaller input
 *     id) is made the integer order by relabelling vertex v to its rank; each
 *     adjacency list is then sorted ascending.
 *  R3 Edges are enumerated as (u, v) with u < v in the relabelled graph, u
 *     ascending then v ascending; edge j carries iu = position of v in N(u)
 *     and jv = position of u in N(v).
 *  R4 The edge draw of Alg. 1 / Alg. 3 ("pick e with probability p_e") is an
 *     exact integer inverse-CDF: r uniform in [0, W), e = the first edge whose
 *     inclusive prefix of weights exceeds r.
 *  R5 Random words come from Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
 *     SC'11) with key (seed lo, seed hi) and counter (id lo, id hi, t, s):
 *     id is the sample index, t the attempt, s = 0 for Alg. 1, 1 for Alg. 3.
 *     The edge draw reads words 0-1 of block t, the first neighbour word 2,
 *     the second neighbour word 3; each walks t = 0, 1, ... on rejection.
 *  R6 Bounded integers use Lemire's multiply-and-reject method (ACM TOMACS
 *     2019), exact for every range.
 *  R7 "Uniform neighbour of u other than v" (Alg. 1): a uniform in
 *     [0, d_u - 1), x = N(u)[a], and if x == v take the last entry of N(u).
 *  R8 "Uniform neighbour u' of u with v before u'" (Alg. 3): a uniform in
 *     [0, L_{u,v}), u' = N(u)[iu + 1 + a] (the entries after v).
 *  R9 Alg. 1 outputs with u' == v' (a triangle) count toward k and toward no
 *     motif; Alg. 3 outputs that are not centred (Definition 4.1) likewise.
 *  R10 The 3-star estimate uses the Alg. 2 (basic sampler) estimates of the
 *     tailed triangle, chordal 4-cycle and 4-clique; the final report takes
 *     C1..C3 from Alg. 2 and C4..C6 from Alg. 4 (end of Section 4).
 *  R11 Error bars (Corollary 5.3): the roots p_l < alpha < p_u of
 *     exp(-k D(alpha, p)) = delta found by bisection; alpha = 0 or 1 use the
 *     closed forms; the 3-star bar adds the bars of C3, 2 C5 and 4 C6.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* status codes (numeric values are part of the library's C interface) */
#define OR_OK 0
#define OR_NO_PATHS 1
#define OR_ERR_ARG (-1)
#define OR_ERR_NOT_SIMPLE (-2)
#define OR_ERR_ASYMMETRIC (-3)
#define OR_ERR_OVERFLOW (-5)
#define OR_ERR_NOMEM (-9)

/* ------------------------------------------------------------------ graph */

/* Section 2: the input is an undirected simple graph.  Checks, in order of
 * priority: offsets well formed and columns in range (OR_ERR_ARG); no
 * self-loop and no repeated neighbour (OR_ERR_NOT_SIMPLE); every arc has its
 * reverse (OR_ERR_ASYMMETRIC).  Rows need not be sorted. */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int or_validate(int64_t n, int64_t nnz, const int64_t *off, const int32_t *col) {
    if (n < 0 || nnz < 0 || n > INT32_MAX) return OR_ERR_ARG;
    if (off[0] != 0 || off[n] != nnz) return OR_ERR_ARG;
    for (int64_t v = 0; v < n; v++)
        if (off[v + 1] < off[v]) return OR_ERR_ARG;
    for (int64_t i = 0; i < nnz; i++)
        if (col[i] < 0 || col[i] >= n) return OR_ERR_ARG;
    /* sorted copy of every row: repeated neighbours become adjacent, and the
     * reverse-arc lookups below can bisect */
    int32_t *scol = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!scol) return OR_ERR_NOMEM;
    memcpy(scol, col, (size_t)nnz * sizeof(int32_t));
    int bad_simple = 0;
    for (int64_t v = 0; v < n; v++) {
        int32_t *row = scol + off[v];
        int64_t d = off[v + 1] - off[v];
        qsort(row, (size_t)d, sizeof(int32_t), cmp_i32);
        for (int64_t i = 0; i < d; i++) {
            if (row[i] == v) bad_simple = 1;
            if (i > 0 && row[i] == row[i - 1]) bad_simple = 1;
        }
    }
    int status = OR_OK;
    if (bad_simple) status = OR_ERR_NOT_SIMPLE;
    for (int64_t v = 0; v < n && status == OR_OK; v++)
        for (int64_t i = off[v]; i < off[v + 1]; i++) {
            int32_t w = col[i], key = (int32_t)v;
            if (!bsearch(&key, scol + off[w], (size_t)(off[w + 1] - off[w]), sizeof(int32_t), cmp_i32)) {
                status = OR_ERR_ASYMMETRIC;
                break;
            }
        }
    free(scol);
    return status;
}

/* Section 4: u precedes v iff d_u < d_v, or d_u == d_v and id_u < id_v.
 * rank[v] = number of vertices preceding v; the canonical graph names v by
 * rank[v] and lists each row ascending (reading R2). */
static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

int or_canonicalize(int64_t n, int64_t nnz, const int64_t *off, const int32_t *col,
                    int32_t *rank, int64_t *coff, int32_t *ccol) {
    uint64_t *key = (uint64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    if (!key) return OR_ERR_NOMEM;
    for (int64_t v = 0; v < n; v++)
        key[v] = ((uint64_t)(off[v + 1] - off[v]) << 32) | (uint64_t)v;
    qsort(key, (size_t)n, sizeof(uint64_t), cmp_u64);
    for (int64_t r = 0; r < n; r++) rank[(int64_t)(key[r] & 0xffffffffu)] = (int32_t)r;
    coff[0] = 0;
    for (int64_t r = 0; r < n; r++) {
        int64_t v = (int64_t)(key[r] & 0xffffffffu);
        int64_t d = off[v + 1] - off[v];
        coff[r + 1] = coff[r] + d;
        for (int64_t i = 0; i < d; i++) ccol[coff[r] + i] = rank[col[off[v] + i]];
        qsort(ccol + coff[r], (size_t)d, sizeof(int32_t), cmp_i32);
    }
    (void)nnz;
    free(key);
    return OR_OK;
}

/* position of y in the sorted row x, or -1 */
static int64_t find_pos(const int64_t *off, const int32_t *col, int32_t x, int32_t y) {
    const int32_t *row = col + off[x];
    const int32_t *p = (const int32_t *)bsearch(&y, row, (size_t)(off[x + 1] - off[x]),
                                                sizeof(int32_t), cmp_i32);
    return p ? (int64_t)(p - row) : -1;
}

/* adjacency test on the canonical graph */
static int adj(const int64_t *off, const int32_t *col, int32_t x, int32_t y) {
    return x != y && find_pos(off, col, x, y) >= 0;
}

/* number of edges (u < v) of the canonical graph */
int64_t or_num_edges(int64_t n, const int64_t *coff, const int32_t *ccol) {
    int64_t m = 0;
    for (int64_t u = 0; u < n; u++)
        for (int64_t i = coff[u]; i < coff[u + 1]; i++)
            if (ccol[i] > u) m++;
    return m;
}

/* Section 3 (tau_e = (d_u - 1)(d_v - 1), W = sum tau_e), Section 4
 * (L_{u,v} = neighbours of u after v, lambda_e = L_{u,v} L_{v,u}, Lambda =
 * sum lambda_e) and Alg. 2 (N_1 = sum_v C(d_v, 3)).  Edges in the order of
 * reading R3; P_tau and P_lambda are inclusive prefix sums.  Returns
 * OR_ERR_OVERFLOW when W or Lambda does not fit in 64 bits. */
int or_edge_table(int64_t n, const int64_t *coff, const int32_t *ccol, int32_t *eu, int32_t *ev,
                  int32_t *eiu, int32_t *ejv, uint64_t *tau, uint64_t *lam, uint64_t *ptau,
                  uint64_t *plam, uint64_t *totals /* W, Lambda, N1 lo, N1 hi */) {
    int64_t j = 0;
    u128 sw = 0, sl = 0, n1 = 0;
    for (int64_t u = 0; u < n; u++) {
        int64_t du = coff[u + 1] - coff[u];
        n1 += (u128)du * (u128)(du > 0 ? du - 1 : 0) * (u128)(du > 1 ? du - 2 : 0) / 6;
        for (int64_t p = 0; p < du; p++) {
            int32_t v = ccol[coff[u] + p];
            if (v <= u) continue;
            int64_t dv = coff[v + 1] - coff[v];
            int64_t q = find_pos(coff, ccol, v, (int32_t)u);
            if (q < 0) return OR_ERR_ASYMMETRIC;
            uint64_t t = (uint64_t)(du - 1) * (uint64_t)(dv - 1);
            uint64_t luv = (uint64_t)(du - 1 - p), lvu = (uint64_t)(dv - 1 - q);
            uint64_t l = luv * lvu;
            sw += t;
            sl += l;
            eu[j] = (int32_t)u;
            ev[j] = v;
            eiu[j] = (int32_t)p;
            ejv[j] = (int32_t)q;
            tau[j] = t;
            lam[j] = l;
            ptau[j] = (uint64_t)sw;
            plam[j] = (uint64_t)sl;
            j++;
        }
    }
    totals[0] = (uint64_t)sw;
    totals[1] = (uint64_t)sl;
    totals[2] = (uint64_t)n1;
    totals[3] = (uint64_t)(n1 >> 64);
    if ((sw >> 64) != 0 || (sl >> 64) != 0) return OR_ERR_OVERFLOW;
    return OR_OK;
}

/* ------------------------------------------------------------ random draws */

/* Philox4x32-10, as defined by Salmon et al. (SC'11): ten rounds of the
 * two-multiplier S-box on a 128-bit counter, the 64-bit key advanced by the
 * Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void block_words(uint64_t seed, uint64_t id, uint32_t t, uint32_t stream, uint32_t w[4]) {
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), t, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, w);
}

/* Lemire's method, 64-bit: x * s as 128 bits; accept unless the low half is
 * below 2^64 mod s. */
int or_lemire64_step(uint64_t x, uint64_t s, uint64_t *result) {
    u128 p = (u128)x * (u128)s;
    uint64_t lo = (uint64_t)p;
    if (lo < s) {
        uint64_t thr = (0 - s) % s;
        if (lo < thr) return 0;
    }
    *result = (uint64_t)(p >> 64);
    return 1;
}

int or_lemire32_step(uint32_t x, uint32_t s, uint32_t *result) {
    uint64_t p = (uint64_t)x * (uint64_t)s;
    uint32_t lo = (uint32_t)p;
    if (lo < s) {
        uint32_t thr = (0u - s) % s;
        if (lo < thr) return 0;
    }
    *result = (uint32_t)(p >> 32);
    return 1;
}

/* r uniform in [0, W) for sample id (reading R5/R6, words 0-1) */
uint64_t or_draw_r(uint64_t seed, uint64_t id, uint32_t stream, uint64_t W) {
    uint32_t w[4];
    uint64_t r;
    for (uint32_t t = 0;; t++) {
        block_words(seed, id, t, stream, w);
        uint64_t x = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
        if (or_lemire64_step(x, W, &r)) return r;
    }
}

/* uniform in [0, s) from word `slot` (2 or 3) */
uint32_t or_draw_small(uint64_t seed, uint64_t id, uint32_t stream, uint32_t slot, uint32_t s) {
    uint32_t w[4];
    uint32_t r;
    for (uint32_t t = 0;; t++) {
        block_words(seed, id, t, stream, w);
        if (or_lemire32_step(w[slot], s, &r)) return r;
    }
}

/* The edge draw of Alg. 1 / Alg. 3: the first j with P[j] > r (reading R4) */
int64_t or_upper_bound(const uint64_t *P, int64_t m, uint64_t r) {
    int64_t lo = 0, hi = m; /* answer in [lo, hi] */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (P[mid] > r) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------ the samplers */

typedef struct {
    int64_t n, m;
    const int64_t *off;
    const int32_t *col;
    const int32_t *eu, *ev, *eiu, *ejv;
    const uint64_t *ptau, *plam;
    uint64_t W, Lambda;
} or_graph;

/* Classification of one Alg. 1 output, given the edge j and the raw
 * neighbour draws a in [0, d_u - 1), b in [0, d_v - 1).  Bins:
 * 0 = triangle (u' == v', no motif), 1 = 3-path, 2 = tailed triangle,
 * 3 = 4-cycle, 4 = chordal 4-cycle, 5 = 4-clique. */
int or_classify_3path(const or_graph *g, int64_t j, uint32_t a, uint32_t b) {
    int32_t u = g->eu[j], v = g->ev[j];
    int64_t du = g->off[u + 1] - g->off[u], dv = g->off[v + 1] - g->off[v];
    int32_t up = g->col[g->off[u] + a];
    if (up == v) up = g->col[g->off[u] + du - 1]; /* other than v (R7) */
    int32_t vp = g->col[g->off[v] + b];
    if (vp == u) vp = g->col[g->off[v] + dv - 1]; /* other than u */
    if (up == vp) return 0;                       /* a triangle (R9)  */
    /* the path u'-u-v-v' is present; the induced pattern depends on the
     * three remaining pairs */
    int e1 = adj(g->off, g->col, up, v);
    int e2 = adj(g->off, g->col, u, vp);
    int e3 = adj(g->off, g->col, up, vp);
    int s = e1 + e2 + e3;
    if (s == 0) return 1;            /* 3 edges: 3-path            */
    if (s == 1) return e3 ? 3 : 2;   /* 4 edges: 4-cycle or tailed */
    if (s == 2) return 4;            /* 5 edges: chordal 4-cycle   */
    return 5;                        /* 6 edges: 4-clique          */
}

/* Classification of one Alg. 3 output with a in [0, L_{u,v}), b in
 * [0, L_{v,u}).  Bins: 0 = not centred, 1 = 4-cycle, 2 = chordal 4-cycle,
 * 3 = 4-clique.  Definition 4.1: t-u-v-w is centred when v precedes t, u
 * precedes w (true by construction, R8) and (t, w) is an edge. */
int or_classify_centered(const or_graph *g, int64_t j, uint32_t a, uint32_t b) {
    int32_t u = g->eu[j], v = g->ev[j];
    int32_t up = g->col[g->off[u] + g->eiu[j] + 1 + a];
    int32_t vp = g->col[g->off[v] + g->ejv[j] + 1 + b];
    if (up == vp || !adj(g->off, g->col, up, vp)) return 0;
    /* a 4-cycle u'-u-v-v'-u'; the chords (u', v) and (u, v') decide the motif */
    return 1 + adj(g->off, g->col, up, v) + adj(g->off, g->col, u, vp);
}

/* The sampling loop of Alg. 2: k runs of Alg. 1 (sample ids first_id .. first_id+k-1)
 * and the class counts.  hist6 is added to. */
void or_sample_3paths(const or_graph *g, uint64_t k, uint64_t seed, uint64_t first_id,
                      uint64_t hist6[6]) {
    if (g->W == 0) return;
    for (uint64_t s = 0; s < k; s++) {
        uint64_t id = first_id + s;
        uint64_t r = or_draw_r(seed, id, 0, g->W);
        int64_t j = or_upper_bound(g->ptau, g->m, r);
        int32_t u = g->eu[j], v = g->ev[j];
        uint32_t du = (uint32_t)(g->off[u + 1] - g->off[u]);
        uint32_t dv = (uint32_t)(g->off[v + 1] - g->off[v]);
        uint32_t a = or_draw_small(seed, id, 0, 2, du - 1);
        uint32_t b = or_draw_small(seed, id, 0, 3, dv - 1);
        hist6[or_classify_3path(g, j, a, b)]++;
    }
}

/* The sampling loop of Alg. 4: k runs of Alg. 3 and the counts of centred outputs. */
void or_sample_centered(const or_graph *g, uint64_t k, uint64_t seed, uint64_t first_id,
                        uint64_t hist4[4]) {
    if (g->Lambda == 0) return;
    for (uint64_t s = 0; s < k; s++) {
        uint64_t id = first_id + s;
        uint64_t r = or_draw_r(seed, id, 1, g->Lambda);
        int64_t j = or_upper_bound(g->plam, g->m, r);
        int32_t u = g->eu[j], v = g->ev[j];
        uint32_t du = (uint32_t)(g->off[u + 1] - g->off[u]);
        uint32_t dv = (uint32_t)(g->off[v + 1] - g->off[v]);
        uint32_t luv = du - 1 - (uint32_t)g->eiu[j];
        uint32_t lvu = dv - 1 - (uint32_t)g->ejv[j];
        uint32_t a = or_draw_small(seed, id, 1, 2, luv);
        uint32_t b = or_draw_small(seed, id, 1, 3, lvu);
        hist4[or_classify_centered(g, j, a, b)]++;
    }
}

/* The same loops over contiguous id ranges on several host threads; each
 * thread counts privately and the integer counts are summed, so the result
 * equals the single-threaded one exactly. */
int or_sample_mt(const or_graph *g, int centered, uint64_t k, uint64_t seed, uint64_t first_id,
                 uint64_t *hist, int nthreads) {
    int nb = centered ? 4 : 6;
    if (nthreads < 1) nthreads = 1;
    uint64_t *part = (uint64_t *)calloc((size_t)nthreads * 6, sizeof(uint64_t));
    if (!part) return OR_ERR_NOMEM;
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
    for (int t = 0; t < nthreads; t++) {
        uint64_t lo = k / (uint64_t)nthreads * (uint64_t)t;
        uint64_t hi = (t == nthreads - 1) ? k : k / (uint64_t)nthreads * (uint64_t)(t + 1);
        if (centered) or_sample_centered(g, hi - lo, seed, first_id + lo, part + 6 * t);
        else or_sample_3paths(g, hi - lo, seed, first_id + lo, part + 6 * t);
    }
    for (int t = 0; t < nthreads; t++)
        for (int i = 0; i < nb; i++) hist[i] += part[6 * t + i];
    free(part);
    return OR_OK;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Every Alg. 1 outcome (edge j, a, b) has probability exactly 1/W
 * (Claim 3.1), so counting all of them per class gives W times the class
 * probabilities.  Used only for the exact-distribution check. */
void or_enumerate_3path(const or_graph *g, uint64_t cnt6[6]) {
    for (int64_t j = 0; j < g->m; j++) {
        int32_t u = g->eu[j], v = g->ev[j];
        uint32_t du = (uint32_t)(g->off[u + 1] - g->off[u]);
        uint32_t dv = (uint32_t)(g->off[v + 1] - g->off[v]);
        for (uint32_t a = 0; a + 1 < du; a++)
            for (uint32_t b = 0; b + 1 < dv; b++) cnt6[or_classify_3path(g, j, a, b)]++;
    }
}

/* Same for Alg. 3 (each outcome has probability 1/Lambda, Claim 4.3). */
void or_enumerate_centered(const or_graph *g, uint64_t cnt4[4]) {
    for (int64_t j = 0; j < g->m; j++) {
        int32_t u = g->eu[j], v = g->ev[j];
        uint32_t du = (uint32_t)(g->off[u + 1] - g->off[u]);
        uint32_t dv = (uint32_t)(g->off[v + 1] - g->off[v]);
        uint32_t luv = du - 1 - (uint32_t)g->eiu[j];
        uint32_t lvu = dv - 1 - (uint32_t)g->ejv[j];
        for (uint32_t a = 0; a < luv; a++)
            for (uint32_t b = 0; b < lvu; b++) cnt4[or_classify_centered(g, j, a, b)]++;
    }
}

/* ------------------------------------------------------------- estimation */

/* Bernoulli KL divergence D(a, b) of Theorem 5.1 */
static double kl(double a, double b) {
    double t1 = a > 0 ? a * log(a / b) : 0.0;
    double t2 = a < 1 ? (1 - a) * log((1 - a) / (1 - b)) : 0.0;
    return t1 + t2;
}

/* Definition 5.2: the two p with exp(-k D(alpha, p)) = delta (reading R11) */
void or_chernoff_bounds(uint64_t count, uint64_t k, double delta, double *pl, double *pu) {
    double alpha = (double)count / (double)k;
    double target = log(1.0 / delta) / (double)k;
    if (count == 0) {
        *pl = 0.0;
        *pu = 1.0 - pow(delta, 1.0 / (double)k);
        return;
    }
    if (count == k) {
        *pl = pow(delta, 1.0 / (double)k);
        *pu = 1.0;
        return;
    }
    double lo = 0.0, hi = alpha; /* D decreases on (0, alpha) */
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (kl(alpha, mid) > target) lo = mid;
        else hi = mid;
    }
    *pl = 0.5 * (lo + hi);
    lo = alpha;
    hi = 1.0; /* D increases on (alpha, 1) */
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (kl(alpha, mid) > target) hi = mid;
        else lo = mid;
    }
    *pu = 0.5 * (lo + hi);
}

/* The estimators of Alg. 2 and Alg. 4 and the final combination (R10), with
 * the error bars of Section 5 (R11).  est/lo/hi are indexed by motif - 1.
 * W == 0: no 3-path exists, so C2..C6 = 0 and C1 = N1 exactly; Lambda == 0:
 * no 4-cycle exists, so C4..C6 = 0. */
static const double A2[7] = {0, 0, 1, 2, 4, 6, 12}; /* 3-paths per motif, Eq. (1) row 2 */
static const double B[7] = {0, 0, 0, 0, 1, 1, 3};   /* centred 3-paths, Lemma 4.2 */

/* flags bit 0: the 3-star identity C1 = N1 - C3 - 2 C5 - 4 C6 (Alg. 2) takes
 * C5 and C6 from the centred sampler (Alg. 4) instead of the 3-path sampler,
 * with their bars (C3 only the 3-path sampler sees).  flags bit 1: report
 * Alg. 2's own estimates of C4..C6 (from the 3-path sampler) instead of the
 * final combination's centred ones. */
int or_estimate_ex(uint64_t W, uint64_t Lambda, uint64_t n1_lo, uint64_t n1_hi,
                   const uint64_t hist6[6], uint64_t k3, const uint64_t hist4[4], uint64_t kc,
                   double delta, int flags, double est[6], double lo[6], double hi[6]);

int or_estimate(uint64_t W, uint64_t Lambda, uint64_t n1_lo, uint64_t n1_hi,
                const uint64_t hist6[6], uint64_t k3, const uint64_t hist4[4], uint64_t kc,
                double delta, double est[6], double lo[6], double hi[6]) {
    return or_estimate_ex(W, Lambda, n1_lo, n1_hi, hist6, k3, hist4, kc, delta, 0, est, lo, hi);
}

int or_estimate_ex(uint64_t W, uint64_t Lambda, uint64_t n1_lo, uint64_t n1_hi,
                   const uint64_t hist6[6], uint64_t k3, const uint64_t hist4[4], uint64_t kc,
                   double delta, int flags, double est[6], double lo[6], double hi[6]) {
    if (k3 == 0 || kc == 0 || !(delta > 0.0 && delta < 1.0) || (flags & ~3)) return OR_ERR_ARG;
    const int c1_from_centred = flags & 1, three_path_only = flags & 2;
    double n1 = (double)(((u128)n1_hi << 64) | (u128)n1_lo);
    double basic[7] = {0}, blo[7] = {0}, bhi[7] = {0};
    for (int i = 2; i <= 6; i++) {
        if (W == 0) continue;
        double K = (double)W / A2[i];
        basic[i] = (double)hist6[i - 1] * (double)W / (double)k3 / A2[i];
        double pl, pu;
        or_chernoff_bounds(hist6[i - 1], k3, delta, &pl, &pu);
        blo[i] = pl * K;
        bhi[i] = pu * K;
    }
    double cen[7] = {0}, clo[7] = {0}, chi[7] = {0};
    for (int i = 4; i <= 6; i++) {
        if (Lambda == 0) continue;
        double K = (double)Lambda / B[i];
        cen[i] = (double)hist4[i - 3] * (double)Lambda / (double)kc / B[i];
        double pl, pu;
        or_chernoff_bounds(hist4[i - 3], kc, delta, &pl, &pu);
        clo[i] = pl * K;
        chi[i] = pu * K;
    }
    /* C5 and C6 of the 3-star identity: the 3-path sampler's by default */
    const double *e = c1_from_centred ? cen : basic;
    const double *el = c1_from_centred ? clo : blo;
    const double *eh = c1_from_centred ? chi : bhi;
    double c1 = n1 - basic[3] - 2.0 * e[5] - 4.0 * e[6];
    double down = (basic[3] - blo[3]) + 2.0 * (e[5] - el[5]) + 4.0 * (e[6] - el[6]);
    double up = (bhi[3] - basic[3]) + 2.0 * (eh[5] - e[5]) + 4.0 * (eh[6] - e[6]);
    est[0] = c1;
    lo[0] = c1 - up;
    hi[0] = c1 + down;
    for (int i = 2; i <= 3; i++) {
        est[i - 1] = basic[i];
        lo[i - 1] = blo[i];
        hi[i - 1] = bhi[i];
    }
    for (int i = 4; i <= 6; i++) {
        est[i - 1] = three_path_only ? basic[i] : cen[i];
        lo[i - 1] = three_path_only ? blo[i] : clo[i];
        hi[i - 1] = three_path_only ? bhi[i] : chi[i];
    }
    return (W == 0 || Lambda == 0) ? OR_NO_PATHS : OR_OK;
}

/* ----------------------------------------------------------- exact counts */

/* Brute force over all 4-vertex subsets (tiny graphs): the induced motif of
 * each connected subset, told apart by edge count and degree sequence. */
int or_bruteforce_counts(int64_t n, const int64_t *off, const int32_t *col, uint64_t C[6]) {
    if (n > 4096) return OR_ERR_ARG;
    unsigned char *A = (unsigned char *)calloc((size_t)(n * n > 0 ? n * n : 1), 1);
    if (!A) return OR_ERR_NOMEM;
    for (int64_t v = 0; v < n; v++)
        for (int64_t i = off[v]; i < off[v + 1]; i++) A[v * n + col[i]] = 1;
    for (int i = 0; i < 6; i++) C[i] = 0;
    for (int64_t a = 0; a < n; a++)
        for (int64_t b = a + 1; b < n; b++)
            for (int64_t c = b + 1; c < n; c++)
                for (int64_t d = c + 1; d < n; d++) {
                    int64_t q[4] = {a, b, c, d};
                    int deg[4] = {0, 0, 0, 0}, e = 0;
                    for (int x = 0; x < 4; x++)
                        for (int y = x + 1; y < 4; y++)
                            if (A[q[x] * n + q[y]]) { e++; deg[x]++; deg[y]++; }
                    int maxd = 0, mind = 3;
                    for (int x = 0; x < 4; x++) {
                        if (deg[x] > maxd) maxd = deg[x];
                        if (deg[x] < mind) mind = deg[x];
                    }
                    if (e == 3) {
                        if (maxd == 3) C[0]++;          /* 3-star           */
                        else if (mind == 1) C[1]++;     /* 3-path           */
                        /* else a triangle plus an isolated vertex          */
                    } else if (e == 4) {
                        if (maxd == 3) C[2]++;          /* tailed triangle  */
                        else C[3]++;                    /* 4-cycle          */
                    } else if (e == 5) C[4]++;          /* chordal 4-cycle  */
                    else if (e == 6) C[5]++;            /* 4-clique         */
                }
    free(A);
    return OR_OK;
}

static int64_t intersect_count(const int32_t *a, int64_t la, const int32_t *b, int64_t lb) {
    int64_t i = 0, j = 0, c = 0;
    while (i < la && j < lb) {
        if (a[i] < b[j]) i++;
        else if (a[i] > b[j]) j++;
        else { c++; i++; j++; }
    }
    return c;
}

/* Triangles through each edge: t_j = |N(u_j) ∩ N(v_j)| for the edges (u_j,
 * v_j) given (the per-edge counts whose pairs make the chordal 4-cycles of
 * Eq. (1): a chordal 4-cycle is two triangles sharing its chord).  Rows must
 * be sorted ascending. */
int or_triangles_per_edge(int64_t n, const int64_t *off, const int32_t *col, int64_t m,
                          const int32_t *eu, const int32_t *ev, uint32_t *t) {
    for (int64_t j = 0; j < m; j++) {
        const int64_t u = eu[j], v = ev[j];
        if (u < 0 || u >= n || v < 0 || v >= n) return OR_ERR_ARG;
        t[j] = (uint32_t)intersect_count(col + off[u], off[u + 1] - off[u], col + off[v],
                                         off[v + 1] - off[v]);
    }
    return OR_OK;
}

/* Exact induced counts from non-induced ones through Eq. (1).  On a graph
 * with sorted rows:
 *   N1 = sum_v C(d_v, 3)                   3-stars
 *   N2 = W - 3T                            3-paths (Alg. 1 outcomes that are
 *                                          not triangles; 3 per triangle)
 *   N3 = sum_v t_v (d_v - 2)               tailed triangles
 *   N4 = (1/2) sum_{a<c} C(codeg(a, c), 2) 4-cycles (each has 2 diagonals)
 *   N5 = sum_e C(t_e, 2)                   chordal 4-cycles (by their chord)
 *   N6 = number of 4-cliques
 * then back-substitution through the unit upper-triangular matrix of
 * Eq. (1).  out_N and out_C are 6 exact integers each (the counts fit in
 * 64 bits for every graph this is run on; the sums use 128 bits). */
int or_exact_counts(int64_t n, const int64_t *off, const int32_t *col, uint64_t out_N[6],
                    int64_t out_C[6]) {
    u128 N[7] = {0};
    u128 T3 = 0; /* 3 x triangles */
    int64_t *tv = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    unsigned char *mark = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!tv || !cnt || !mark) { free(tv); free(cnt); free(mark); return OR_ERR_NOMEM; }
    u128 W = 0;
    for (int64_t u = 0; u < n; u++) {
        int64_t du = off[u + 1] - off[u];
        N[1] += (u128)du * (u128)(du > 0 ? du - 1 : 0) * (u128)(du > 1 ? du - 2 : 0) / 6;
        for (int64_t i = off[u]; i < off[u + 1]; i++) {
            int32_t v = col[i];
            if (v <= u) continue;
            int64_t dv = off[v + 1] - off[v];
            W += (u128)(du - 1) * (u128)(dv - 1);
            int64_t te = intersect_count(col + off[u], du, col + off[v], dv);
            T3 += (u128)te; /* each triangle is seen from its 3 edges */
            N[5] += (u128)te * (u128)(te > 0 ? te - 1 : 0) / 2;
            tv[u] += te;
            tv[v] += te;
        }
    }
    N[2] = W - T3;
    for (int64_t v = 0; v < n; v++) {
        int64_t dv = off[v + 1] - off[v];
        /* tv counts each triangle at v twice (once per incident edge) */
        N[3] += (u128)(tv[v] / 2) * (u128)(dv >= 2 ? dv - 2 : 0);
    }
    /* 4-cycles: codegrees of pairs (a, c), a < c */
    u128 s4 = 0;
    for (int64_t a = 0; a < n; a++) {
        for (int64_t i = off[a]; i < off[a + 1]; i++) {
            int32_t b = col[i];
            for (int64_t t = off[b]; t < off[b + 1]; t++) {
                int32_t c = col[t];
                if (c > a) cnt[c]++;
            }
        }
        for (int64_t i = off[a]; i < off[a + 1]; i++) {
            int32_t b = col[i];
            for (int64_t t = off[b]; t < off[b + 1]; t++) {
                int32_t c = col[t];
                if (c > a && cnt[c] > 0) {
                    s4 += (u128)cnt[c] * (u128)(cnt[c] - 1) / 2;
                    cnt[c] = 0;
                }
            }
        }
    }
    N[4] = s4 / 2;
    /* 4-cliques a < b < c < d */
    u128 k4 = 0;
    for (int64_t a = 0; a < n; a++) {
        for (int64_t i = off[a]; i < off[a + 1]; i++) mark[col[i]] = 1;
        for (int64_t i = off[a]; i < off[a + 1]; i++) {
            int32_t b = col[i];
            if (b <= a) continue;
            for (int64_t t = off[b]; t < off[b + 1]; t++) {
                int32_t c = col[t];
                if (c <= b || !mark[c]) continue;
                for (int64_t s = off[c]; s < off[c + 1]; s++) {
                    int32_t d = col[s];
                    if (d <= c || !mark[d]) continue;
                    if (find_pos(off, col, b, d) >= 0) k4++;
                }
            }
        }
        for (int64_t i = off[a]; i < off[a + 1]; i++) mark[col[i]] = 0;
    }
    N[6] = k4;
    free(tv);
    free(cnt);
    free(mark);
    /* back-substitution through Eq. (1) */
    __int128 C6 = (__int128)N[6];
    __int128 C5 = (__int128)N[5] - 6 * C6;
    __int128 C4 = (__int128)N[4] - C5 - 3 * C6;
    __int128 C3 = (__int128)N[3] - 4 * C5 - 12 * C6;
    __int128 C2 = (__int128)N[2] - 2 * C3 - 4 * C4 - 6 * C5 - 12 * C6;
    __int128 C1 = (__int128)N[1] - C3 - 2 * C5 - 4 * C6;
    for (int i = 0; i < 6; i++) out_N[i] = (uint64_t)N[i + 1];
    out_C[0] = (int64_t)C1;
    out_C[1] = (int64_t)C2;
    out_C[2] = (int64_t)C3;
    out_C[3] = (int64_t)C4;
    out_C[4] = (int64_t)C5;
    out_C[5] = (int64_t)C6;
    return OR_OK;
}
