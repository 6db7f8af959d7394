// ps_device.cuh -- device-side building blocks of the path-sampling library:
// the graph descriptor, Philox4x32-10, Lemire bounded draws, list searches,
// the adjacency test and a decoupled look-back scan.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ps {

typedef unsigned long long u64;

// ---------------------------------------------------------------- layout

// One edge (u < v) of the relabelled graph, 32 bytes = one DRAM sector:
// everything a sample needs after choosing the edge.  iu / jv are the
// positions of v in N(u) and of u in N(v); ou / ov the row offsets.
struct __align__(16) EdgeRec {
    int32_t u, v, du, dv, iu, jv, ou, ov;
};

// Device view of one loaded graph (passed by value to kernels and stored in
// the batched launch's descriptor table).
struct GraphDev {
    const int64_t *off;      // [n + 1] canonical row offsets
    const int32_t *col;      // [nnz]   canonical adjacency, rows ascending
    const EdgeRec *rec;      // [m]
    const uint64_t *ptau;    // [m] inclusive prefix of tau
    const uint64_t *plam;    // [m] inclusive prefix of lambda
    const int32_t *gtau;     // [Bt + 1] guide: first edge of each r >> tau_shift bucket
    const int32_t *glam;     // [Bl + 1]
    const uint32_t *hub;     // [hubs][hub_words] adjacency bitmaps of the top labels
    const uint64_t *eset;    // hash set of the edges (4-slot buckets), or null
    uint64_t eset_mask;      // buckets - 1
    const int32_t *vtab;     // per-vertex hash tables: slots [2 off(x), 2 off(x+1)), or null
    uint64_t W, Lambda;
    int64_t n, m;
    int32_t hub_start;       // labels >= hub_start have a bitmap row
    int32_t hub_words;
    int32_t tau_shift, lam_shift;
    int32_t adj_mode;        // kAdjHash or kAdjSearch
    int32_t hub_bit_base;    // hub rows hold the bits of labels >= hub_bit_base (a multiple of 32)
};

// Adjacency test variants (chosen by the tuning; results are identical).
enum { kAdjHash = 1, kAdjSearch = 2, kAdjVtab = 3 };

// status block (uint64 words at the start of the workspace)
enum {
    ST_FLAGS = 0,
    ST_DMAX = 1,
    ST_M_UPPER = 2,
    ST_W_LO = 3, ST_W_HI = 4,
    ST_L_LO = 5, ST_L_HI = 6,
    ST_N1_LO = 7, ST_N1_HI = 8,
    ST_HUBS = 9,
    ST_TIER = 10,      // 5 words: row boundaries of the sort tiers
    ST_LONG = 15,      // first row longer than kLongRow (its arcs are walked by a block)
    ST_COUNTER = 16,   // 16 words: tile counters of scans (as uint32 pairs)
    ST_ESET_SPILL = 32, // non-zero: the hash set's key lists overflowed (slow path taken)
    ST_WORDS = 64
};

enum : u64 {
    F_ARG = 1ull,
    F_NOT_SIMPLE = 2ull,
    F_ASYM = 4ull,
    F_OVERFLOW = 8ull,
    F_TIMEOUT = 16ull
};

__device__ __forceinline__ void raise_flag(u64 *status, u64 f) {
    atomicOr(reinterpret_cast<unsigned long long *>(status + ST_FLAGS),
             static_cast<unsigned long long>(f));
}

// Bound on every device spin-wait (iterations with nanosleep back-off).
constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p);

// Waits until *flag is non-zero and returns it, or returns 0 after `limit`
// polls (the caller then reports PS_ERR_TIMEOUT instead of hanging).
__device__ __forceinline__ uint32_t wait_flag(const uint32_t *flag, uint32_t limit) {
    uint32_t f = ld_acquire(flag);
    for (uint32_t it = 0; f == 0u && it < limit; it++) {
        __nanosleep(it < 64 ? 32 : 256);
        f = ld_acquire(flag);
    }
    return f;
}

// ------------------------------------------------------------------ loads

// Read-only gathers of data written by earlier kernels.  PS_LOAD_MODE picks
// the cache path: 0 = the non-coherent path through L1 (__ldg); 1 = L2 only
// (ld.global.cg); 2 = non-coherent without L1 allocation.  In modes 1 and 2
// a 32-byte edge record is one 256-bit load.
#ifndef PS_LOAD_MODE
#define PS_LOAD_MODE 0
#endif
#if PS_LOAD_MODE == 1
#define PS_LD "ld.global.cg"
#elif PS_LOAD_MODE == 2
#define PS_LD "ld.global.nc.L1::no_allocate"
#endif

__device__ __forceinline__ int32_t ldg_i32(const int32_t *p) {
#if PS_LOAD_MODE == 0
    return __ldg(p);
#else
    int32_t v;
    asm(PS_LD ".s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#endif
}
__device__ __forceinline__ int64_t ldg_i64(const int64_t *p) {
#if PS_LOAD_MODE == 0
    return static_cast<int64_t>(__ldg(reinterpret_cast<const long long *>(p)));
#else
    int64_t v;
    asm(PS_LD ".s64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
#endif
}
__device__ __forceinline__ uint64_t ldg_u64(const uint64_t *p) {
#if PS_LOAD_MODE == 0
    return static_cast<uint64_t>(__ldg(reinterpret_cast<const unsigned long long *>(p)));
#else
    uint64_t v;
    asm(PS_LD ".u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
#endif
}
// Gathers of the skewed "hot" structures (guide entries, prefix probes).
// (Evict-last L2 hints on these, on the hub rows' adjacency lists, and
// evict-first on the hash buckets were measured: no gain.)
__device__ __forceinline__ int32_t ldg_i32_hot(const int32_t *p) { return ldg_i32(p); }
__device__ __forceinline__ uint64_t ldg_u64_hot(const uint64_t *p) { return ldg_u64(p); }

__device__ __forceinline__ EdgeRec ldg_rec(const EdgeRec *p) {
    EdgeRec e;
#if PS_LOAD_MODE == 0
    const int4 *q = reinterpret_cast<const int4 *>(p);
    int4 a = __ldg(q), b = __ldg(q + 1);
    e.u = a.x; e.v = a.y; e.du = a.z; e.dv = a.w;
    e.iu = b.x; e.jv = b.y; e.ou = b.z; e.ov = b.w;
#else
    asm(PS_LD ".v8.s32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(e.u), "=r"(e.v), "=r"(e.du), "=r"(e.dv), "=r"(e.iu), "=r"(e.jv), "=r"(e.ou), "=r"(e.ov)
        : "l"(p));
#endif
    return e;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ----------------------------------------------------------------- Philox

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// two-multiplier S-box, key advanced by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; i++) {
        if (i) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Random block t of sample `id` for sampler `stream` (0: 3-path, 1: centred):
// key (seed lo, seed hi), counter (id lo, id hi, t, stream).
__device__ __forceinline__ uint4 sample_block(uint64_t seed, uint64_t id, uint32_t t,
                                              uint32_t stream) {
    return philox4x32_10(make_uint4(static_cast<uint32_t>(id), static_cast<uint32_t>(id >> 32), t,
                                    stream),
                         make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
}

// Lemire's multiply-and-reject (ACM TOMACS 2019): one attempt.  The
// threshold (2^64 mod s) is only computed when the low half is below s.
__device__ __forceinline__ bool lemire64(uint64_t x, uint64_t s, uint64_t &out) {
    const uint64_t lo = x * s;
    if (lo < s) {
        const uint64_t thr = (0ull - s) % s;
        if (lo < thr) return false;
    }
    out = __umul64hi(x, s);
    return true;
}

__device__ __forceinline__ bool lemire32(uint32_t x, uint32_t s, uint32_t &out) {
    const uint64_t p = static_cast<uint64_t>(x) * s;
    const uint32_t lo = static_cast<uint32_t>(p);
    if (lo < s) {
        const uint32_t thr = (0u - s) % s;
        if (lo < thr) return false;
    }
    out = static_cast<uint32_t>(p >> 32);
    return true;
}

// Rejected first attempts walk blocks t = 1, 2, ... on the same word slot.
static __device__ __noinline__ uint64_t draw_r_retry(uint64_t seed, uint64_t id, uint32_t stream,
                                              uint64_t s) {
    uint64_t r = 0;
    for (uint32_t t = 1; t < 4096u; t++) {
        const uint4 w = sample_block(seed, id, t, stream);
        if (lemire64((static_cast<uint64_t>(w.y) << 32) | w.x, s, r)) return r;
    }
    return 0;  // unreachable for any s (probability < 2^-4000)
}

static __device__ __noinline__ uint32_t draw_small_retry(uint64_t seed, uint64_t id, uint32_t stream,
                                                  int slot, uint32_t s) {
    uint32_t r = 0;
    for (uint32_t t = 1; t < 4096u; t++) {
        const uint4 w = sample_block(seed, id, t, stream);
        if (lemire32(slot == 2 ? w.z : w.w, s, r)) return r;
    }
    return 0;
}

// --------------------------------------------------------------- searches

// First j in [lo, hi] with P[j] > r, given P[hi] > r.
__device__ __forceinline__ int64_t upper_bound_in(const uint64_t *P, int64_t lo, int64_t hi,
                                                  uint64_t r) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (ldg_u64_hot(P + mid) > r) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Edge of r: guide bucket r >> shift gives a range [G[b], G[b + 1]] that
// holds the answer; search it exactly.
__device__ __forceinline__ int64_t find_edge(const uint64_t *P, const int32_t *G, int shift,
                                             uint64_t r) {
    const uint64_t b = r >> shift;
    const int64_t lo = ldg_i32_hot(G + b);
    const int64_t hi = ldg_i32_hot(G + b + 1);
    if (lo == hi) return lo;
    return upper_bound_in(P, lo, hi, r);
}

// Is `key` in the sorted list col[o, o + d)?
__device__ __forceinline__ bool in_sorted(const int32_t *col, int64_t o, int64_t d, int32_t key) {
    int64_t lo = o, hi = o + d;  // answer position in [lo, hi)
    while (hi - lo > 8) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (ldg_i32(col + mid) <= key) lo = mid;
        else hi = mid;
    }
    bool hit = false;
#pragma unroll
    for (int i = 0; i < 8; i++)
        if (lo + i < hi) hit |= (ldg_i32(col + lo + i) == key);
    return hit;
}

// Adjacency test of Alg. 2 / Alg. 4 ("determine the induced subgraph").
// The smaller label has the smaller (or equal) degree, so its list is
// searched; pairs of hubs read one bit of the hub bitmap.
__device__ __forceinline__ bool adjacent(const GraphDev &g, int32_t x, int32_t y) {
    if (x == y) return false;
    const int32_t a = min(x, y), b = max(x, y);
    if (a >= g.hub_start) {  // then b > a >= hub_bit_base
        const uint32_t *row = g.hub + static_cast<int64_t>(a - g.hub_start) * g.hub_words;
        return (__ldg(row + ((b - g.hub_bit_base) >> 5)) >> (b & 31)) & 1u;
    }
    const int64_t o = ldg_i64(g.off + a);
    const int64_t e = ldg_i64(g.off + a + 1);
    return in_sorted(g.col, o, e - o, b);
}

// Same when the row of a (the smaller label) is already known.
__device__ __forceinline__ bool adjacent_known(const GraphDev &g, int32_t a, int64_t oa,
                                               int64_t da, int32_t b) {
    if (a >= g.hub_start) {  // then b > a >= hub_bit_base
        const uint32_t *row = g.hub + static_cast<int64_t>(a - g.hub_start) * g.hub_words;
        return (__ldg(row + ((b - g.hub_bit_base) >> 5)) >> (b & 31)) & 1u;
    }
    return in_sorted(g.col, oa, da, b);
}

// ----------------------------------------------------------- edge hash set

// The hash-table adjacency that the O(1) test of Theorem 3.5 assumes: the
// edges {a, b}, a < b, keyed (a << 32) | b, in buckets of four 8-byte slots
// (32 bytes, one DRAM sector) with linear probing from bucket to bucket.
// (8-slot, 64-byte buckets overflow less -- 1.04 instead of 1.18 buckets per
// absent-key lookup at load 1/2 -- but measured slower: 3-path sampling
// 1.75 -> 1.88 ms on R-MAT 20 and 20 -> 29 ms on the 3M-vertex graph.)
// Slots only ever go from empty (all ones) to full, so a lookup that meets a
// bucket with an empty slot before finding its key can stop: had the key
// been inserted, it would sit in that bucket or an earlier one.
constexpr uint64_t kEmptySlot = ~0ull;
constexpr int kBucketSlots = 4;
constexpr int kBucketShift = 2;  // log2(kBucketSlots)

__device__ __forceinline__ uint64_t edge_key(int32_t a, int32_t b) {
    return (static_cast<uint64_t>(static_cast<uint32_t>(a)) << 32) | static_cast<uint32_t>(b);
}

// Mixes the key; its low bits pick the home bucket and its top kBucketShift
// bits the slot an insertion tries first (any slot order is valid for the
// lookups, which read the whole bucket).
__device__ __forceinline__ uint64_t key_hash(uint64_t key) {
    uint64_t h = key * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31;
    h *= 0xD6E8FEB86659FD93ull;
    h ^= h >> 29;
    return h;
}

__device__ __forceinline__ uint64_t key_bucket(uint64_t key, uint64_t mask) { return key_hash(key) & mask; }

struct Bucket {
    ulonglong2 q[kBucketSlots / 2];
};

__device__ __forceinline__ Bucket load_bucket(const uint64_t *set, uint64_t b) {
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(set + (b << kBucketShift));
    Bucket k;
#pragma unroll
    for (int i = 0; i < kBucketSlots / 2; i++) k.q[i] = __ldg(p + i);
    return k;
}

// 1: key present, 0: absent, -1: bucket full without the key (probe on)
__device__ __forceinline__ int bucket_verdict(const Bucket &k, uint64_t key) {
    bool hit = false, empty = false;
#pragma unroll
    for (int i = 0; i < kBucketSlots / 2; i++) {
        hit |= (k.q[i].x == key) | (k.q[i].y == key);
        empty |= (k.q[i].x == kEmptySlot) | (k.q[i].y == kEmptySlot);
    }
    return hit ? 1 : (empty ? 0 : -1);
}

static __device__ __noinline__ bool probe_on(const uint64_t *set, uint64_t mask, uint64_t key,
                                             uint64_t b) {
    for (uint64_t i = 0; i < mask; i++) {
        b = (b + 1) & mask;
        const int v = bucket_verdict(load_bucket(set, b), key);
        if (v >= 0) return v == 1;
    }
    return false;
}

__device__ __forceinline__ bool eset_contains(const uint64_t *set, uint64_t mask, int32_t x, int32_t y) {
    if (x == y) return false;
    const uint64_t key = edge_key(min(x, y), max(x, y));
    const uint64_t b = key_bucket(key, mask);
    const int v = bucket_verdict(load_bucket(set, b), key);
    return v >= 0 ? v == 1 : probe_on(set, mask, key, b);
}

// Two independent lookups (x != y for both) with their first buckets loaded together.
__device__ __forceinline__ void eset_contains2(const uint64_t *set, uint64_t mask, int32_t x0,
                                               int32_t y0, int32_t x1, int32_t y1, bool &r0, bool &r1) {
    const uint64_t k0 = edge_key(min(x0, y0), max(x0, y0));
    const uint64_t k1 = edge_key(min(x1, y1), max(x1, y1));
    const uint64_t b0 = key_bucket(k0, mask), b1 = key_bucket(k1, mask);
    const Bucket q0 = load_bucket(set, b0), q1 = load_bucket(set, b1);
    const int v0 = bucket_verdict(q0, k0), v1 = bucket_verdict(q1, k1);
    r0 = v0 >= 0 ? v0 == 1 : probe_on(set, mask, k0, b0);
    r1 = v1 >= 0 ? v1 == 1 : probe_on(set, mask, k1, b1);
}

// Three independent lookups with their first buckets loaded together.
__device__ __forceinline__ void eset_contains3(const uint64_t *set, uint64_t mask, int32_t x0,
                                               int32_t y0, int32_t x1, int32_t y1, int32_t x2,
                                               int32_t y2, bool &r0, bool &r1, bool &r2) {
    const uint64_t k0 = edge_key(min(x0, y0), max(x0, y0));
    const uint64_t k1 = edge_key(min(x1, y1), max(x1, y1));
    const uint64_t k2 = edge_key(min(x2, y2), max(x2, y2));
    const uint64_t b0 = key_bucket(k0, mask), b1 = key_bucket(k1, mask), b2 = key_bucket(k2, mask);
    const Bucket q0 = load_bucket(set, b0), q1 = load_bucket(set, b1), q2 = load_bucket(set, b2);
    const int v0 = bucket_verdict(q0, k0), v1 = bucket_verdict(q1, k1), v2 = bucket_verdict(q2, k2);
    r0 = (x0 != y0) && (v0 >= 0 ? v0 == 1 : probe_on(set, mask, k0, b0));
    r1 = (x1 != y1) && (v1 >= 0 ? v1 == 1 : probe_on(set, mask, k1, b1));
    r2 = (x2 != y2) && (v2 >= 0 ? v2 == 1 : probe_on(set, mask, k2, b2));
}

// Hash set plus hub rows: a pair whose larger label is one of the top-degree
// labels (>= hub_start, rows of the hub bitmap) is answered from that
// hub's bitmap row, the rest from the hash set.  The sampled edges are
// drawn in proportion to tau, so a lookup (u', v) mostly names a hub v, and
// the hub rows' much-read parts stay in L2.  (The rows' loads once asked L2
// to keep them -- evict-last; with 1024 rows of 375 KB on the 3M-vertex
// graph that hint made 3-path sampling 2-5% slower on both benchmark graphs,
// and it was dropped.)  With no hub rows (hub_start == n) this is the plain
// hash-set test.
__device__ __forceinline__ uint32_t ld_hub_word(const uint32_t *p) { return __ldg(p); }

// Address of the hub-row word holding bit a of hub c's row (a >= hub_bit_base).
__device__ __forceinline__ const uint32_t *hub_word_of(const GraphDev &g, int32_t a, int32_t c) {
    return g.hub + static_cast<int64_t>(c - g.hub_start) * g.hub_words + ((a - g.hub_bit_base) >> 5);
}

// Does the pair a < c have a hub-row bit?  (The rows hold the labels from
// hub_bit_base up: the tests naming a hub mostly name it with another
// high-degree, high-label vertex, and the rest go to the hash set, which
// holds every edge.)
__device__ __forceinline__ bool in_hub_rows(const GraphDev &g, int32_t a, int32_t c) {
    return c >= g.hub_start && a >= g.hub_bit_base;
}

// One pair's first load: its hub-row word (in the first slot of the
// returned bucket) when it has a hub-row bit, else its home bucket.
__device__ __forceinline__ Bucket load_pair(const GraphDev &g, int32_t a, int32_t c, uint64_t b) {
    Bucket q;
    if (in_hub_rows(g, a, c)) {
        q.q[0].x = ld_hub_word(hub_word_of(g, a, c));
    } else {
        q = load_bucket(g.eset, b);
    }
    return q;
}

__device__ __forceinline__ bool resolve_pair(const GraphDev &g, int32_t a, int32_t c, uint64_t key,
                                             uint64_t b, const Bucket &q) {
    if (in_hub_rows(g, a, c)) return ((q.q[0].x >> (a & 31)) & 1u) != 0u;
    const int v = bucket_verdict(q, key);
    return v >= 0 ? v == 1 : probe_on(g.eset, g.eset_mask, key, b);
}

// Three independent tests (x != y for each pair) with all first loads in
// flight together; a pair whose larger label is a hub reads the hub's row.
// ALL = false sends only the first pair to a hub row (it names an endpoint
// of the drawn edge, most often a hub) and keeps the other two on the hash
// set: fewer registers, for kernels that cannot spare them (the batched
// kernel runs at 64).
template <bool ALL>
__device__ __forceinline__ void pair_test3(const GraphDev &g, int32_t x0, int32_t y0, int32_t x1,
                                           int32_t y1, int32_t x2, int32_t y2, bool &r0, bool &r1,
                                           bool &r2) {
    const int32_t a0 = min(x0, y0), c0 = max(x0, y0);
    if (!ALL) {
        if (!in_hub_rows(g, a0, c0)) {
            eset_contains3(g.eset, g.eset_mask, x0, y0, x1, y1, x2, y2, r0, r1, r2);
            return;
        }
        const uint32_t w = ld_hub_word(hub_word_of(g, a0, c0));
        eset_contains2(g.eset, g.eset_mask, x1, y1, x2, y2, r1, r2);
        r0 = ((w >> (a0 & 31)) & 1u) != 0u;
        return;
    }
    const int32_t a1 = min(x1, y1), c1 = max(x1, y1);
    const int32_t a2 = min(x2, y2), c2 = max(x2, y2);
    const uint64_t k0 = edge_key(a0, c0), k1 = edge_key(a1, c1), k2 = edge_key(a2, c2);
    const uint64_t b0 = key_bucket(k0, g.eset_mask), b1 = key_bucket(k1, g.eset_mask),
                   b2 = key_bucket(k2, g.eset_mask);
    const Bucket q0 = load_pair(g, a0, c0, b0), q1 = load_pair(g, a1, c1, b1), q2 = load_pair(g, a2, c2, b2);
    r0 = resolve_pair(g, a0, c0, k0, b0, q0);
    r1 = resolve_pair(g, a1, c1, k1, b1, q1);
    r2 = resolve_pair(g, a2, c2, k2, b2, q2);
}

__device__ __forceinline__ bool pair_test(const GraphDev &g, int32_t x, int32_t y) {
    const int32_t a = min(x, y), c = max(x, y);
    if (in_hub_rows(g, a, c))
        return x != y && ((ld_hub_word(hub_word_of(g, a, c)) >> (a & 31)) & 1u);
    return eset_contains(g.eset, g.eset_mask, x, y);
}

// Two independent tests (x != y for each pair), both loads in flight; ALL as
// for pair_test3.
template <bool ALL>
__device__ __forceinline__ void pair_test2(const GraphDev &g, int32_t x0, int32_t y0, int32_t x1,
                                           int32_t y1, bool &r0, bool &r1) {
    const int32_t a0 = min(x0, y0), c0 = max(x0, y0);
    if (!ALL) {
        if (!in_hub_rows(g, a0, c0)) {
            eset_contains2(g.eset, g.eset_mask, x0, y0, x1, y1, r0, r1);
            return;
        }
        const uint32_t w = ld_hub_word(hub_word_of(g, a0, c0));
        r1 = eset_contains(g.eset, g.eset_mask, x1, y1);
        r0 = ((w >> (a0 & 31)) & 1u) != 0u;
        return;
    }
    const int32_t a1 = min(x1, y1), c1 = max(x1, y1);
    const uint64_t k0 = edge_key(a0, c0), k1 = edge_key(a1, c1);
    const uint64_t b0 = key_bucket(k0, g.eset_mask), b1 = key_bucket(k1, g.eset_mask);
    const Bucket q0 = load_pair(g, a0, c0, b0), q1 = load_pair(g, a1, c1, b1);
    r0 = resolve_pair(g, a0, c0, k0, b0, q0);
    r1 = resolve_pair(g, a1, c1, k1, b1, q1);
}

// ------------------------------------------------ per-vertex hash tables

// Each adjacency list in its own open-addressing table (Theorem 3.5 assumes
// hash-table adjacency lists): the table of vertex x is the 2 d_x int32
// slots starting at 2 off(x), holding the neighbours of x (empty = -1),
// linear probing with wrap-around inside the table.  The slot of y is
// (mix(y) * 2 d_x) >> 32.  Lookups go to the table of the endpoint that is a
// sampled edge's endpoint or else the larger label, so they concentrate on
// the tables of high-degree vertices, which stay in L2.
constexpr int32_t kEmptyLabel = -1;

__device__ __forceinline__ uint32_t label_mix(int32_t y) {
    uint32_t h = static_cast<uint32_t>(y) * 0x9E3779B1u;
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    h ^= h >> 13;
    return h;
}

__device__ __forceinline__ uint64_t vtab_start(int32_t y, uint64_t size) {
    return (static_cast<uint64_t>(label_mix(y)) * size) >> 32;
}

static __device__ __noinline__ bool vtab_probe_on(const int32_t *t, uint64_t size, int32_t y, uint64_t s) {
    for (uint64_t i = 1; i < size; i++) {
        s = (s + 1 == size) ? 0 : s + 1;
        const int32_t x = __ldg(t + s);
        if (x == y) return true;
        if (x == kEmptyLabel) return false;
    }
    return false;
}

// Is y a neighbour of the vertex whose row is [off, off + d)?
struct VtabQuery {
    const int32_t *t;
    uint64_t size, s;
    int32_t y;
    __device__ __forceinline__ void start(const int32_t *vtab, int64_t off, int64_t d, int32_t key) {
        t = vtab + 2 * off;
        size = static_cast<uint64_t>(2 * d);
        y = key;
        s = size ? vtab_start(key, size) : 0;
    }
    __device__ __forceinline__ int32_t first() const { return size ? __ldg(t + s) : kEmptyLabel; }
    __device__ __forceinline__ bool resolve(int32_t x) const {
        if (x == y) return true;
        if (x == kEmptyLabel) return false;
        return vtab_probe_on(t, size, y, s);
    }
};

}  // namespace ps
