/*
 * graphgen.c -- seeded synthetic graph generators.
 *
 * This module only produces inputs: undirected simple graphs in CSR form
 * (int64 row offsets, int32 column indices, every row sorted ascending, no
 * self-loops, no duplicates, symmetric).  It holds none of the arithmetic of
 * the path-sampling method; both the CUDA library and the CPU oracle consume
 * its output.
 *
 * Random numbers come from a counter-based hash (the SplitMix64 finaliser of
 * Steele, Lea & Flood, OOPSLA 2014) keyed by (seed, stream, index), so every
 * graph is a pure function of its parameters and the result does not depend
 * on the number of OpenMP threads.
 *
 * Generators:
 *  - Chung-Lu (Chung & Lu 2002): edge {i,j} present independently with
 *    probability min(1, w_i w_j / sum(w)).  Weights follow a power law
 *    w_i = w_max * (i0 / (i + i0))^(1/(gamma-1)), i0 solved so that the mean
 *    weight is the requested average degree.  Small graphs test every pair;
 *    large graphs use the geometric-skipping method of Miller & Hagberg
 *    (WAW 2011), which draws the same distribution in O(n + m).
 *  - R-MAT (Chakrabarti, Zhan & Faloutsos 2004): edge_factor * 2^scale edge
 *    draws, each descending `scale` quadrant levels with probabilities
 *    (a, b, c, d); self-loops dropped, then symmetrised and deduplicated.
 * Both apply a seeded random relabelling of vertex ids (as real edge lists
 * have ids unrelated to degree).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;
    int64_t nnz;
    int64_t *off; /* n + 1 */
    int32_t *col; /* nnz   */
} gg_csr;

enum { GG_OK = 0, GG_ERR_ARG = -1, GG_ERR_NOMEM = -2 };

/* stream tags keep the hash inputs of different uses apart */
enum { ST_PERM = 1, ST_PAIR = 2, ST_SKIP = 3, ST_RMAT = 4 };

static inline uint64_t sm_fin(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t hrand(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    uint64_t h = sm_fin(seed ^ (stream * 0xD6E8FEB86659FD93ull));
    h = sm_fin(h ^ a);
    return sm_fin(h ^ (b * 0xA0761D6478BD642Full));
}

/* uniform in (0, 1] with 53 random bits */
static inline double unit_open0(uint64_t x) {
    return (double)((x >> 11) + 1) * 0x1.0p-53;
}

static void sort_i32(int32_t *a, int64_t len);

/* ---------------------------------------------------------------- CSR build */

/* Build a symmetric CSR from undirected pairs (pu[i], pv[i]), relabelled by
 * perm (perm == NULL: identity).  Self-loops are dropped; duplicate pairs are
 * merged.  Rows come out sorted ascending. */
static int build_csr(int64_t n, int64_t npairs, const int32_t *pu, const int32_t *pv,
                     const int32_t *perm, gg_csr *out) {
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return GG_ERR_NOMEM;
    for (int64_t i = 0; i < npairs; i++) {
        int32_t a = pu[i], b = pv[i];
        if (a == b) continue;
        if (perm) { a = perm[a]; b = perm[b]; }
        deg[a]++;
        deg[b]++;
    }
    int64_t *off = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!off) { free(deg); return GG_ERR_NOMEM; }
    off[0] = 0;
    for (int64_t v = 0; v < n; v++) off[v + 1] = off[v] + deg[v];
    int64_t total = off[n];
    int32_t *col = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (!col) { free(deg); free(off); return GG_ERR_NOMEM; }
    for (int64_t v = 0; v < n; v++) deg[v] = off[v];
    for (int64_t i = 0; i < npairs; i++) {
        int32_t a = pu[i], b = pv[i];
        if (a == b) continue;
        if (perm) { a = perm[a]; b = perm[b]; }
        col[deg[a]++] = b;
        col[deg[b]++] = a;
    }
    /* sort each row, then drop duplicates */
    int64_t *keep = deg; /* reuse: kept length per row */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; v++) {
        int64_t s = off[v], len = off[v + 1] - off[v];
        sort_i32(col + s, len);
        int64_t w = 0;
        for (int64_t i = 0; i < len; i++)
            if (w == 0 || col[s + i] != col[s + w - 1]) col[s + w++] = col[s + i];
        keep[v] = w;
    }
    int64_t *noff = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!noff) { free(deg); free(off); free(col); return GG_ERR_NOMEM; }
    noff[0] = 0;
    for (int64_t v = 0; v < n; v++) noff[v + 1] = noff[v] + keep[v];
    int32_t *ncol = col;
    if (noff[n] != total) {
        ncol = (int32_t *)malloc((size_t)(noff[n] > 0 ? noff[n] : 1) * sizeof(int32_t));
        if (!ncol) { free(deg); free(off); free(col); free(noff); return GG_ERR_NOMEM; }
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t v = 0; v < n; v++)
            memcpy(ncol + noff[v], col + off[v], (size_t)keep[v] * sizeof(int32_t));
        free(col);
    }
    free(deg);
    free(off);
    out->n = n;
    out->nnz = noff[n];
    out->off = noff;
    out->col = ncol;
    return GG_OK;
}

static void isort_i32(int32_t *a, int64_t len) {
    for (int64_t i = 1; i < len; i++) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; j--; }
        a[j + 1] = x;
    }
}

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

static void sort_i32(int32_t *a, int64_t len) {
    if (len <= 32) isort_i32(a, len);
    else qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
}

/* Fisher-Yates permutation of 0..n-1 */
static int32_t *make_perm(int64_t n, uint64_t seed) {
    int32_t *p = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!p) return NULL;
    for (int64_t i = 0; i < n; i++) p[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; i--) {
        uint64_t j = hrand(seed, ST_PERM, (uint64_t)i, 0) % (uint64_t)(i + 1);
        int32_t t = p[i];
        p[i] = p[j];
        p[j] = t;
    }
    return p;
}

/* ------------------------------------------------------------- Chung-Lu */

static double cl_mean(int64_t n, double w_max, double expo, double i0) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += w_max * pow(i0 / ((double)i + i0), expo);
    return s / (double)n;
}

/* weights w_i = w_max (i0/(i+i0))^(1/(gamma-1)), i0 by bisection in log space */
int gg_chung_lu_weights(int64_t n, double avg_deg, double gamma, double w_max, double *w,
                        double *i0_out) {
    if (n <= 0 || !(gamma > 1.0) || !(avg_deg > 0.0) || !(w_max >= avg_deg)) return GG_ERR_ARG;
    double expo = 1.0 / (gamma - 1.0);
    double lo = -30.0, hi = 40.0; /* log(i0) */
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (cl_mean(n, w_max, expo, exp(mid)) < avg_deg) lo = mid;
        else hi = mid;
    }
    double i0 = exp(0.5 * (lo + hi));
    for (int64_t i = 0; i < n; i++) w[i] = w_max * pow(i0 / ((double)i + i0), expo);
    if (i0_out) *i0_out = i0;
    return GG_OK;
}

/* Pairs of one row u (u < v), exact test of every pair. */
static int64_t cl_row_exact(int64_t n, const double *w, double S, uint64_t seed, int64_t u,
                            int32_t *dst) {
    int64_t c = 0;
    for (int64_t v = u + 1; v < n; v++) {
        double p = w[u] * w[v] / S;
        if (p > 1.0) p = 1.0;
        double r = unit_open0(hrand(seed, ST_PAIR, (uint64_t)u, (uint64_t)v)) ;
        /* r in (0,1]; accept with probability p */
        if (r <= p && p > 0.0) {
            if (dst) dst[c] = (int32_t)v;
            c++;
        }
    }
    return c;
}

/* Pairs of one row u by geometric skipping (weights non-increasing in v). */
static int64_t cl_row_skip(int64_t n, const double *w, double S, uint64_t seed, int64_t u,
                           int32_t *dst) {
    int64_t c = 0;
    int64_t v = u + 1;
    uint64_t t = 0;
    if (v >= n) return 0;
    double p = w[u] * w[v] / S;
    if (p > 1.0) p = 1.0;
    while (v < n && p > 0.0) {
        if (p < 1.0) {
            double r = unit_open0(hrand(seed, ST_SKIP, (uint64_t)u, t++));
            double skip = floor(log(r) / log1p(-p));
            if (skip >= (double)(n - v)) break;
            v += (int64_t)skip;
        }
        if (v >= n) break;
        double q = w[u] * w[v] / S;
        if (q > 1.0) q = 1.0;
        double r = unit_open0(hrand(seed, ST_SKIP, (uint64_t)u, t++));
        if (r <= q / p) {
            if (dst) dst[c] = (int32_t)v;
            c++;
        }
        p = q;
        v++;
    }
    return c;
}

int gg_chung_lu(int64_t n, double avg_deg, double gamma, double w_max, uint64_t seed,
                int exact_pairs, int permute, gg_csr *out) {
    if (n <= 1 || n > INT32_MAX || !out) return GG_ERR_ARG;
    double *w = (double *)malloc((size_t)n * sizeof(double));
    if (!w) return GG_ERR_NOMEM;
    int rc = gg_chung_lu_weights(n, avg_deg, gamma, w_max, w, NULL);
    if (rc) { free(w); return rc; }
    double S = 0.0;
    for (int64_t i = 0; i < n; i++) S += w[i];

    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) { free(w); return GG_ERR_NOMEM; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t u = 0; u < n; u++)
        cnt[u + 1] = exact_pairs ? cl_row_exact(n, w, S, seed, u, NULL)
                                 : cl_row_skip(n, w, S, seed, u, NULL);
    for (int64_t u = 0; u < n; u++) cnt[u + 1] += cnt[u];
    int64_t m = cnt[n];
    int32_t *pu = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t *pv = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!pu || !pv) { free(w); free(cnt); free(pu); free(pv); return GG_ERR_NOMEM; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t u = 0; u < n; u++) {
        int64_t c = exact_pairs ? cl_row_exact(n, w, S, seed, u, pv + cnt[u])
                                : cl_row_skip(n, w, S, seed, u, pv + cnt[u]);
        for (int64_t i = 0; i < c; i++) pu[cnt[u] + i] = (int32_t)u;
    }
    free(w);
    free(cnt);
    int32_t *perm = permute ? make_perm(n, seed) : NULL;
    if (permute && !perm) { free(pu); free(pv); return GG_ERR_NOMEM; }
    rc = build_csr(n, m, pu, pv, perm, out);
    free(pu);
    free(pv);
    free(perm);
    return rc;
}

/* ---------------------------------------------------------------- R-MAT */

int gg_rmat(int scale, double edge_factor, double a, double b, double c, uint64_t seed,
            int permute, gg_csr *out) {
    if (scale < 1 || scale > 30 || !(edge_factor > 0) || !out) return GG_ERR_ARG;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return GG_ERR_ARG;
    int64_t n = (int64_t)1 << scale;
    int64_t draws = (int64_t)llround(edge_factor * (double)n);
    /* integer thresholds on the 32-bit scale */
    uint64_t ta = (uint64_t)(a * 4294967296.0);
    uint64_t tb = (uint64_t)((a + b) * 4294967296.0);
    uint64_t tc = (uint64_t)((a + b + c) * 4294967296.0);
    int32_t *pu = (int32_t *)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    int32_t *pv = (int32_t *)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    if (!pu || !pv) { free(pu); free(pv); return GG_ERR_NOMEM; }
#pragma omp parallel for schedule(static, 4096)
    for (int64_t e = 0; e < draws; e++) {
        uint32_t u = 0, v = 0;
        uint64_t word = 0;
        for (int L = 0; L < scale; L++) {
            if ((L & 1) == 0) word = hrand(seed, ST_RMAT, (uint64_t)e, (uint64_t)(L >> 1));
            uint64_t x = (L & 1) ? (word >> 32) : (word & 0xffffffffull);
            uint32_t bu, bv;
            if (x < ta) { bu = 0; bv = 0; }
            else if (x < tb) { bu = 0; bv = 1; }
            else if (x < tc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        pu[e] = (int32_t)u;
        pv[e] = (int32_t)v;
    }
    int32_t *perm = permute ? make_perm(n, seed ^ 0x5EEDull) : NULL;
    if (permute && !perm) { free(pu); free(pv); return GG_ERR_NOMEM; }
    int rc = build_csr(n, draws, pu, pv, perm, out);
    free(pu);
    free(pv);
    free(perm);
    return rc;
}

/* CSR from caller-provided undirected pairs (self-loops dropped, duplicates merged). */
int gg_from_pairs(int64_t n, int64_t npairs, const int32_t *pu, const int32_t *pv, gg_csr *out) {
    if (n < 0 || npairs < 0 || !out) return GG_ERR_ARG;
    for (int64_t i = 0; i < npairs; i++)
        if (pu[i] < 0 || pu[i] >= n || pv[i] < 0 || pv[i] >= n) return GG_ERR_ARG;
    return build_csr(n, npairs, pu, pv, NULL, out);
}

void gg_free(gg_csr *g) {
    if (!g) return;
    free(g->off);
    free(g->col);
    g->off = NULL;
    g->col = NULL;
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
