// ps_scan.cuh -- warp utilities, 128-bit accumulation and the single-pass
// decoupled look-back scan used by the load, prefix and exact-count steps
// (not by the sampling kernels).
#pragma once

#include "ps_device.cuh"

namespace ps {

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

// ------------------------------------------------ 128-bit accumulation

__device__ __forceinline__ void add128(uint64_t &lo, uint64_t &hi, uint64_t x) {
    lo += x;
    hi += (lo < x);
}

__device__ __forceinline__ void atomic_add128(u64 *pair, uint64_t lo, uint64_t hi) {
    const unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long *>(pair),
                                             static_cast<unsigned long long>(lo));
    if (old + lo < old) hi += 1;
    if (hi) atomicAdd(reinterpret_cast<unsigned long long *>(pair + 1), static_cast<unsigned long long>(hi));
}

__device__ __forceinline__ void warp_add128(uint64_t &lo, uint64_t &hi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const uint64_t h2 = __shfl_down_sync(0xffffffffu, hi, o);
        add128(lo, hi, l2);
        hi += h2;
    }
}

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

// A tile is BLOCK * ITEMS consecutive items; warp w owns the w-th run of
// 32 * ITEMS of them and walks it in rows of 32 (lane-contiguous, so loads
// and stores coalesce): item wbase + 32 i of the calling lane is its i-th.
// The tile id comes from a ticket (launch order), so a block only ever waits
// on tiles already owned by running blocks.
template <typename T>
__device__ __forceinline__ int64_t scan_ticket(const ScanState<T> &st) {
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(st.counter, 1u);
    __syncthreads();
    return s_tile;
}
template <int BLOCK, int ITEMS>
__device__ __forceinline__ int64_t scan_wbase(int64_t tile) {
    return tile * (int64_t)(BLOCK * ITEMS) + (int64_t)(threadIdx.x >> 5) * (32 * ITEMS) + (threadIdx.x & 31);
}

// The scan of one tile whose items the block holds (v[i] = item
// scan_wbase + 32 i, identity past `count`): each row scanned across the
// warp with the row total carried forward, the warps' runs combined, the
// tile's prefix found by look-back, then store(i, exclusive_i, inclusive_i).
template <typename T, int BLOCK, int ITEMS, typename Op, typename Store>
__device__ __forceinline__ void scan_tile(int64_t tile, int64_t wbase, T (&v)[ITEMS], int64_t count,
                                          const ScanState<T> &st, T identity, Op op, Store store) {
    constexpr int NW = BLOCK / 32;
    __shared__ T s_warp[NW];
    __shared__ T s_excl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T carry = identity;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        T x = v[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = shfl_up_t(x, o);
            if (lane >= o) x = op(y, x);
        }
        x = op(carry, x);
        v[i] = x;  // inclusive prefix within the warp's run
        carry = shfl_idx_t(x, 31);
    }
    if (lane == 31) s_warp[warp] = carry;
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
                    f = wait_flag(st.flag + p, kSpinLimit);
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
    const T run = op(s_excl, warp_excl);
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        T prev = shfl_up_t(v[i], 1);
        const T row_before = (i == 0) ? identity : shfl_idx_t(v[i - 1], 31);
        if (lane == 0) prev = row_before;
        const int64_t idx = wbase + 32 * i;
        if (idx < count) store(idx, op(run, prev), op(run, v[i]));
    }
}

// ------------------------------------------------ edge weights and prefixes

// tau_j = (d_u - 1)(d_v - 1) (Section 3); lambda_j = L_{u,v} L_{v,u} with
// L_{u,v} = d_u - 1 - iu, the neighbours of u after v in the order (Section 4).
__device__ __forceinline__ U64x2 edge_weights(int32_t du, int32_t dv, int32_t iu, int32_t jv) {
    const uint64_t t = static_cast<uint64_t>(du - 1) * static_cast<uint64_t>(dv - 1);
    const uint64_t l = static_cast<uint64_t>(du - 1 - iu) * static_cast<uint64_t>(dv - 1 - jv);
    return U64x2{t, l};
}

// The inclusive prefixes P_tau[j], P_lambda[j].  The weights are
// non-negative, so a running sum that passes 2^64 shows up at the first item
// whose inclusive prefix is below its exclusive one; the last item's
// prefixes are W and Lambda.
struct StorePrefix {
    uint64_t *ptau, *plam;
    u64 *status;
    int64_t m;
    __device__ void operator()(int64_t j, U64x2 exc, U64x2 inc) const {
        ptau[j] = inc.a;
        plam[j] = inc.b;
        if (inc.a < exc.a || inc.b < exc.b) raise_flag(status, F_OVERFLOW);
        if (j == m - 1) {
            status[ST_W_LO] = inc.a;
            status[ST_L_LO] = inc.b;
        }
    }
};

// Scans `count` items: item i = load(i); store(i, exclusive_i, inclusive_i).
template <typename T, int BLOCK, int ITEMS, typename Op, typename Load, typename Store>
__global__ void __launch_bounds__(BLOCK)
k_scan(int64_t count, ScanState<T> st, T identity, Op op, Load load, Store store) {
    const int64_t tile = scan_ticket(st);
    const int64_t wbase = scan_wbase<BLOCK, ITEMS>(tile);
    T v[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const int64_t idx = wbase + 32 * i;
        v[i] = idx < count ? load(idx) : identity;
    }
    scan_tile<T, BLOCK, ITEMS>(tile, wbase, v, count, st, identity, op, store);
}

}  // namespace ps
