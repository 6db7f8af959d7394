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
    uint64_t W, Lambda;
    int64_t n, m;
    int32_t hub_start;       // labels >= hub_start have a bitmap row
    int32_t hub_words;
    int32_t tau_shift, lam_shift;
};

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
    ST_COUNTER = 16,   // 16 words: tile counters of scans (as uint32 pairs)
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

// ------------------------------------------------------------------ loads

__device__ __forceinline__ int32_t ldg_i32(const int32_t *p) { return __ldg(p); }
__device__ __forceinline__ int64_t ldg_i64(const int64_t *p) {
    return static_cast<int64_t>(__ldg(reinterpret_cast<const long long *>(p)));
}
__device__ __forceinline__ uint64_t ldg_u64(const uint64_t *p) {
    return static_cast<uint64_t>(__ldg(reinterpret_cast<const unsigned long long *>(p)));
}
__device__ __forceinline__ EdgeRec ldg_rec(const EdgeRec *p) {
    const int4 *q = reinterpret_cast<const int4 *>(p);
    int4 a = __ldg(q), b = __ldg(q + 1);
    EdgeRec e;
    e.u = a.x; e.v = a.y; e.du = a.z; e.dv = a.w;
    e.iu = b.x; e.jv = b.y; e.ou = b.z; e.ov = b.w;
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
        if (ldg_u64(P + mid) > r) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Edge of r: guide bucket r >> shift gives a range [G[b], G[b + 1]] that
// holds the answer; search it exactly.
__device__ __forceinline__ int64_t find_edge(const uint64_t *P, const int32_t *G, int shift,
                                             uint64_t r) {
    const uint64_t b = r >> shift;
    const int64_t lo = ldg_i32(G + b);
    const int64_t hi = ldg_i32(G + b + 1);
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
    if (a >= g.hub_start) {
        const uint32_t *row = g.hub + static_cast<int64_t>(a - g.hub_start) * g.hub_words;
        return (__ldg(row + (b >> 5)) >> (b & 31)) & 1u;
    }
    const int64_t o = ldg_i64(g.off + a);
    const int64_t e = ldg_i64(g.off + a + 1);
    return in_sorted(g.col, o, e - o, b);
}

// Same when the row of a (the smaller label) is already known.
__device__ __forceinline__ bool adjacent_known(const GraphDev &g, int32_t a, int64_t oa,
                                               int64_t da, int32_t b) {
    if (a >= g.hub_start) {
        const uint32_t *row = g.hub + static_cast<int64_t>(a - g.hub_start) * g.hub_words;
        return (__ldg(row + (b >> 5)) >> (b & 31)) & 1u;
    }
    return in_sorted(g.col, oa, da, b);
}

// ------------------------------------------------------------- warp utils

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T shfl_up_t(T v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}
template <typename T>
__device__ __forceinline__ T shfl_down_t(T v, int d) {
    return __shfl_down_sync(0xffffffffu, v, d);
}
template <typename T>
__device__ __forceinline__ T shfl_idx_t(T v, int l) {
    return __shfl_sync(0xffffffffu, v, l);
}

struct U64x2 {
    uint64_t a, b;
};
template <>
__device__ __forceinline__ U64x2 shfl_up_t<U64x2>(U64x2 v, int d) {
    return U64x2{__shfl_up_sync(0xffffffffu, v.a, d), __shfl_up_sync(0xffffffffu, v.b, d)};
}
template <>
__device__ __forceinline__ U64x2 shfl_down_t<U64x2>(U64x2 v, int d) {
    return U64x2{__shfl_down_sync(0xffffffffu, v.a, d), __shfl_down_sync(0xffffffffu, v.b, d)};
}
template <>
__device__ __forceinline__ U64x2 shfl_idx_t<U64x2>(U64x2 v, int l) {
    return U64x2{__shfl_sync(0xffffffffu, v.a, l), __shfl_sync(0xffffffffu, v.b, l)};
}

struct OpSum {
    template <typename T>
    __device__ __forceinline__ T operator()(T x, T y) const { return x + y; }
    __device__ __forceinline__ U64x2 operator()(U64x2 x, U64x2 y) const {
        return U64x2{x.a + y.a, x.b + y.b};
    }
};
struct OpMax {
    template <typename T>
    __device__ __forceinline__ T operator()(T x, T y) const { return x > y ? x : y; }
};

// ------------------------------------------------ decoupled look-back scan

// Tile status for the single-pass scan of Merrill & Garland (2016): a flag
// per tile (0 = empty, 1 = aggregate ready, 2 = inclusive prefix ready) and
// the two values.  `counter` hands out tile ids in launch order, so a block
// only ever waits on tiles already owned by running blocks.
template <typename T>
struct ScanState {
    uint32_t *flag;
    T *agg;
    T *inc;
    uint32_t *counter;
    u64 *status;
};

template <typename T>
__device__ __forceinline__ T ld_cg(const T *p) {
    return *reinterpret_cast<const volatile T *>(p);
}
template <>
__device__ __forceinline__ U64x2 ld_cg<U64x2>(const U64x2 *p) {
    const volatile uint64_t *q = reinterpret_cast<const volatile uint64_t *>(p);
    return U64x2{q[0], q[1]};
}

// Scans `count` items: item i = load(i); store(i, exclusive_i, inclusive_i).
template <typename T, int BLOCK, int ITEMS, typename Op, typename Load, typename Store>
__global__ void __launch_bounds__(BLOCK)
k_scan(int64_t count, ScanState<T> st, T identity, Op op, Load load, Store store) {
    constexpr int NW = BLOCK / 32;
    __shared__ uint32_t s_tile;
    __shared__ T s_warp[NW];
    __shared__ T s_excl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(st.counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * (int64_t)(BLOCK * ITEMS) + (int64_t)threadIdx.x * ITEMS;

    T v[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; i++) v[i] = (base + i < count) ? load(base + i) : identity;
#pragma unroll
    for (int i = 1; i < ITEMS; i++) v[i] = op(v[i - 1], v[i]);
    const T tsum = v[ITEMS - 1];
    T x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = shfl_up_t(x, o);
        if (lane >= o) x = op(y, x);
    }
    T lane_excl = shfl_up_t(x, 1);
    if (lane == 0) lane_excl = identity;
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? s_warp[lane] : identity;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = shfl_up_t(w, o);
            if (lane >= o) w = op(y, w);
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    const T warp_excl = warp ? s_warp[warp - 1] : identity;
    const T tile_agg = s_warp[NW - 1];

    if (warp == 0) {
        T excl = identity;
        if (tile == 0) {
            if (lane == 0) {
                st.inc[0] = tile_agg;
                __threadfence();
                st_release(st.flag, 2u);
            }
        } else {
            if (lane == 0) {
                st.agg[tile] = tile_agg;
                __threadfence();
                st_release(st.flag + tile, 1u);
            }
            int64_t pred = tile - 1;
            bool timed_out = false;
            while (true) {
                const int64_t p = pred - lane;
                uint32_t f = 2u;
                T val = identity;
                if (p >= 0) {
                    uint32_t it = 0;
                    f = ld_acquire(st.flag + p);
                    while (f == 0u) {
                        if (++it >= kSpinLimit) break;
                        __nanosleep(it < 64 ? 32 : 256);
                        f = ld_acquire(st.flag + p);
                    }
                    if (f == 0u) {
                        timed_out = true;
                        f = 2u;
                    } else {
                        val = (f == 2u) ? ld_cg(st.inc + p) : ld_cg(st.agg + p);
                    }
                }
                const uint32_t incmask = __ballot_sync(0xffffffffu, f == 2u);
                const int stop = incmask ? (__ffs(incmask) - 1) : 31;
                T c = (lane <= stop) ? val : identity;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c = op(c, shfl_down_t(c, o));
                c = shfl_idx_t(c, 0);
                excl = op(c, excl);
                if (incmask) break;
                pred -= 32;
            }
            if (__any_sync(0xffffffffu, timed_out) && lane == 0) raise_flag(st.status, F_TIMEOUT);
            if (lane == 0) {
                st.inc[tile] = op(excl, tile_agg);
                __threadfence();
                st_release(st.flag + tile, 2u);
            }
        }
        if (lane == 0) s_excl = excl;
    }
    __syncthreads();
    // v[i] now holds this thread's inclusive prefix up to item i
    const T run = op(s_excl, op(warp_excl, lane_excl));
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        if (base + i < count) {
            const T exc = (i == 0) ? run : op(run, v[i - 1]);
            store(base + i, exc, op(run, v[i]));
        }
    }
}

}  // namespace ps
