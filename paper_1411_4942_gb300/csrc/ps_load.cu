// ps_load.cu -- ps_load_csr: validation of the input graph (Section 2), the
// degree order of Section 4 made the integer order by relabelling, sorted
// adjacency lists, and the edge table (u < v, row-major) with the position of
// each edge in both endpoint lists.
#include <climits>

#include "ps_internal.h"

namespace ps {

// ------------------------------------------------------------ scan plumbing

template <typename T>
ScanState<T> scan_state(ps_graph *g, int counter_slot) {
    ScanState<T> s;
    s.flag = reinterpret_cast<uint32_t *>(g->ws + g->L.scan_flag);
    s.agg = reinterpret_cast<T *>(g->ws + g->L.scan_agg);
    s.inc = reinterpret_cast<T *>(g->ws + g->L.scan_inc);
    s.counter = reinterpret_cast<uint32_t *>(g->status + ST_COUNTER + counter_slot);
    s.status = g->status;
    return s;
}
template ScanState<uint32_t> scan_state<uint32_t>(ps_graph *, int);
template ScanState<int64_t> scan_state<int64_t>(ps_graph *, int);
template ScanState<int32_t> scan_state<int32_t>(ps_graph *, int);
template ScanState<U64x2> scan_state<U64x2>(ps_graph *, int);

int reset_scan(ps_graph *g, int counter_slot, int64_t count, cudaStream_t s) {
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    if (tiles > g->L.scan_tiles) return PS_ERR_WORKSPACE;
    PS_CUDA_TRY(cudaMemsetAsync(g->ws + g->L.scan_flag, 0, sizeof(uint32_t) * (tiles + 1), s));
    PS_CUDA_TRY(cudaMemsetAsync(g->status + ST_COUNTER + counter_slot, 0, sizeof(uint64_t), s));
    return PS_OK;
}

// ------------------------------------------------------------------ degrees

__global__ void k_degrees(int64_t n, int64_t nnz, const int64_t *__restrict__ off,
                          uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, u64 *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) {
        if (ldg_i64(off) != 0 || ldg_i64(off + n) != nnz) raise_flag(status, F_ARG);
    }
    uint32_t dmax = 0;
    bool bad = false, longrow = false;
    for (int64_t v = t0; v < n; v += stride) {
        const int64_t a = ldg_i64(off + v), b = ldg_i64(off + v + 1);
        int64_t d = b - a;
        if (d < 0 || a < 0 || b > nnz) {
            bad = true;
            d = 0;
        }
        if (d > n - 1) longrow = true;  // cannot be a simple row
        keys[v] = static_cast<uint32_t>(d);
        vals[v] = static_cast<uint32_t>(v);
        dmax = max(dmax, static_cast<uint32_t>(d));
    }
    if (bad) raise_flag(status, F_ARG);
    if (longrow) raise_flag(status, F_NOT_SIMPLE);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax)
        atomicMax(reinterpret_cast<unsigned long long *>(status + ST_DMAX), (unsigned long long)dmax);
}

// ------------------------------------------------ rank: stable LSD radix sort

// Per-tile digit histogram, stored digit-major: counts[digit * tiles + tile].
__global__ void __launch_bounds__(kRadixBlock)
k_radix_hist(int64_t n, const uint32_t *__restrict__ keys, int shift, uint32_t *counts, int64_t tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int i = threadIdx.x; i < kRadixTile; i += kRadixBlock) {
        const int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items are ranked round by round in input order; within a
// round, lanes with equal digits are ranked by __match_any_sync and warps by
// their per-digit counts.
__global__ void __launch_bounds__(kRadixBlock)
k_radix_scatter(int64_t n, const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int shift,
                const uint32_t *__restrict__ offsets, int64_t tiles) {
    constexpr int NW = kRadixBlock / 32;
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wcnt[NW][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s_base[threadIdx.x] = offsets[(int64_t)threadIdx.x * tiles + blockIdx.x];
    for (int w = 0; w < NW; w++) s_wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int round = 0; round < kRadixItems; round++) {
        const int64_t idx = base + (int64_t)round * kRadixBlock + threadIdx.x;
        const bool valid = idx < n;
        const uint32_t key = valid ? kin[idx] : 0u;
        const uint32_t digit = valid ? ((key >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t wrank = __popc(peers & lanemask_lt());
        if (valid && lane == __ffs(peers) - 1) s_wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = s_base[digit] + wrank;
            for (int w = 0; w < warp; w++) pos += s_wcnt[w][digit];
            kout[pos] = key;
            vout[pos] = vin[idx];
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < NW; w++) {
            tot += s_wcnt[w][threadIdx.x];
            s_wcnt[w][threadIdx.x] = 0;
        }
        s_base[threadIdx.x] += tot;
        __syncthreads();
    }
}

struct LoadU32 {
    const uint32_t *p;
    __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct StoreExclU32 {
    uint32_t *p;
    __device__ void operator()(int64_t i, uint32_t exc, uint32_t) const { p[i] = exc; }
};

// rank[v] = position of v in (degree, id) order; dnew[r] = degree of row r
__global__ void k_rank(int64_t n, const uint32_t *__restrict__ skeys, const uint32_t *__restrict__ svals,
                       int32_t *rank, int32_t *dnew, uint32_t *inv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const uint32_t v = svals[r];
        rank[v] = static_cast<int32_t>(r);
        dnew[r] = static_cast<int32_t>(skeys[r]);
        if (inv) inv[r] = v;
    }
}

struct LoadDeg {
    const int32_t *d;
    __device__ int64_t operator()(int64_t i) const { return d[i]; }
};
struct StoreOffsets {
    int64_t *off;
    int64_t n;
    __device__ void operator()(int64_t i, int64_t exc, int64_t inc) const {
        off[i] = exc;
        if (i == n - 1) off[n] = inc;
    }
};

// first row whose degree exceeds each tier limit (rows are degree-sorted)
__global__ void k_tiers(int64_t n, const int32_t *__restrict__ dnew, u64 *status) {
    const int lim[5] = {0, kTierA, kTierB, kTierC, kLongRow};
    const int slot[5] = {ST_TIER, ST_TIER + 1, ST_TIER + 2, ST_TIER + 3, ST_LONG};
    const int t = threadIdx.x;
    if (t < 5) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (dnew[mid] > lim[t]) hi = mid;
            else lo = mid + 1;
        }
        status[slot[t]] = static_cast<u64>(lo);
    }
    if (t == 5) status[ST_TIER + 4] = static_cast<u64>(n);
}

// ------------------------------------------------------- row relabel + sort

struct RowIn {
    const int64_t *off;
    const int32_t *col;
    const uint32_t *inv;   // row r of the new graph is input vertex inv[r]
    const int32_t *rank;
    const int64_t *coff;
    int32_t *ccol;
    int32_t *lowcnt;
    int64_t n;
    u64 *status;
};

// Relabelled neighbour, with range and self-loop checks (the bad column is
// replaced by the row itself so no access leaves the arrays).
__device__ __forceinline__ int32_t relabel(const RowIn &R, int64_t i, uint32_t v, int32_t r,
                                          bool &bad_arg, bool &self) {
    const int32_t c = ldg_i32(R.col + i);
    if (c < 0 || c >= R.n) {
        bad_arg = true;
        return r;
    }
    if (c == static_cast<int32_t>(v)) self = true;
    return ldg_i32(R.rank + c);
}

__device__ __forceinline__ void report(const RowIn &R, bool bad_arg, bool not_simple) {
    if (bad_arg) raise_flag(R.status, F_ARG);
    if (not_simple) raise_flag(R.status, F_NOT_SIMPLE);
}

// Tier A: rows of 1..32 entries, one warp, bitonic network in registers.
__global__ void __launch_bounds__(256) k_sort_tier_a(RowIn R) {
    const int lane = threadIdx.x & 31;
    const int64_t r0 = static_cast<int64_t>(R.status[ST_TIER + 0]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_TIER + 1]);
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    bool bad = false, nsimple = false;
    for (int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < r1; r += nw) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int d = static_cast<int>(ldg_i64(R.off + v + 1) - o);
        int32_t x = INT_MAX;
        if (lane < d) x = relabel(R, o + lane, v, (int32_t)r, bad, nsimple);
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
                const bool asc = (lane & k) == 0, lower = (lane & j) == 0;
                x = (lower == asc) ? min(x, y) : max(x, y);
            }
        }
        const int32_t nx = __shfl_down_sync(0xffffffffu, x, 1);
        if (lane + 1 < d && nx == x) nsimple = true;
        const uint32_t low = __popc(__ballot_sync(0xffffffffu, lane < d && x < (int32_t)r));
        if (lane < d) R.ccol[R.coff[r] + lane] = x;
        if (lane == 0) R.lowcnt[r] = (int32_t)low;
    }
    report(R, bad, nsimple);
}

__device__ __forceinline__ int next_pow2(int d) {
    int p = 1;
    while (p < d) p <<= 1;
    return p;
}

// Bitonic sort, ascending, of N = E * THREADS keys held E per thread in
// blocked order (thread t holds keys t*E .. t*E + E - 1).  A compare-exchange
// stage whose partner key sits in the same thread works on registers, one
// whose partner sits in the same warp exchanges by shuffle, and only the
// stages that cross warps go through shared memory (smem: N keys; unused
// when THREADS == 32).  Fully unrolled, so every register index is static.
template <int E, int THREADS>
__device__ __forceinline__ void bitonic_blocked(int32_t (&x)[E], int32_t *smem) {
    constexpr int N = E * THREADS;
    const int lane = threadIdx.x & 31;
    const int base = (THREADS == 32 ? lane : static_cast<int>(threadIdx.x)) * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int i = 0; i < E; i++)
                    if ((i & j) == 0) {
                        const bool asc = ((base | i) & k) == 0;
                        const int32_t a = x[i], b = x[i | j];
                        x[i] = asc ? min(a, b) : max(a, b);
                        x[i | j] = asc ? max(a, b) : min(a, b);
                    }
            } else if (j < 32 * E) {
                const int lm = j / E;
                const bool keep_min = ((lane & lm) == 0) == ((base & k) == 0);
#pragma unroll
                for (int i = 0; i < E; i++) {
                    const int32_t y = __shfl_xor_sync(0xffffffffu, x[i], lm);
                    x[i] = keep_min ? min(x[i], y) : max(x[i], y);
                }
            } else if (THREADS > 32) {
                __syncthreads();  // the previous stage's readers are done
#pragma unroll
                for (int i = 0; i < E; i++) smem[base + i] = x[i];
                __syncthreads();
                const bool keep_min = ((base & j) == 0) == ((base & k) == 0);
#pragma unroll
                for (int i = 0; i < E; i++) {
                    const int32_t y = smem[(base + i) ^ j];
                    x[i] = keep_min ? min(x[i], y) : max(x[i], y);
                }
            }
        }
    }
}

// One row of tier B with P = 32 * E slots: relabel, sort in registers, write
// the row and its lower count.
template <int E>
__device__ __forceinline__ void sort_row_warp(const RowIn &R, int64_t r, uint32_t v, int64_t o, int d,
                                              bool &bad, bool &nsimple) {
    const int lane = threadIdx.x & 31;
    int32_t x[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
        const int idx = lane * E + i;
        x[i] = idx < d ? relabel(R, o + idx, v, static_cast<int32_t>(r), bad, nsimple) : INT_MAX;
    }
    bitonic_blocked<E, 32>(x, nullptr);
    const int32_t after = __shfl_down_sync(0xffffffffu, x[0], 1);  // first key of the next lane
    int32_t *dst = R.ccol + R.coff[r];
    int low = 0;
#pragma unroll
    for (int i = 0; i < E; i++) {
        const int idx = lane * E + i;
        if (idx < d) {
            dst[idx] = x[i];
            low += x[i] < static_cast<int32_t>(r);
            const int32_t nx = (i + 1 < E) ? x[i + 1] : after;
            if (idx + 1 < d && nx == x[i]) nsimple = true;
        }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) low += __shfl_down_sync(0xffffffffu, low, o2);
    if (lane == 0) R.lowcnt[r] = low;
}

// Tier B: rows of 33..1024 entries, one warp, bitonic network in registers,
// in two kernels: rows up to kLongRow entries (two or four keys per lane)
// at 32 registers and full occupancy, the longer ones capped at 64
// registers (four blocks per SM beat the spill-free 105-register build; the
// same holds for tier C at three blocks).
__global__ void __launch_bounds__(256, 8) k_sort_tier_b(RowIn R) {
    const int64_t r0 = static_cast<int64_t>(R.status[ST_TIER + 1]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_LONG]);
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    bool bad = false, nsimple = false;
    for (int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < r1; r += nw) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int d = static_cast<int>(ldg_i64(R.off + v + 1) - o);
        if (d <= 64) sort_row_warp<2>(R, r, v, o, d, bad, nsimple);
        else sort_row_warp<4>(R, r, v, o, d, bad, nsimple);
    }
    report(R, bad, nsimple);
}
static_assert(kLongRow == 128 && kLongRow < kTierB, "tier B's first kernel sorts rows of at most 4 keys per lane");

__global__ void __launch_bounds__(256, 4) k_sort_tier_b2(RowIn R) {
    const int64_t r0 = static_cast<int64_t>(R.status[ST_LONG]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_TIER + 2]);
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    bool bad = false, nsimple = false;
    for (int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < r1; r += nw) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int d = static_cast<int>(ldg_i64(R.off + v + 1) - o);
        if (d <= 256) sort_row_warp<8>(R, r, v, o, d, bad, nsimple);
        else if (d <= 512) sort_row_warp<16>(R, r, v, o, d, bad, nsimple);
        else sort_row_warp<32>(R, r, v, o, d, bad, nsimple);
    }
    report(R, bad, nsimple);
}

// Tier C: rows of 1025..4096 entries, one block of 512, bitonic network in
// registers with the cross-warp stages in shared memory (16 KB, several
// blocks per SM).
template <int E>
__device__ __forceinline__ void sort_row_block(const RowIn &R, int64_t r, uint32_t v, int64_t o, int d,
                                               int32_t *smem, int *s_low, bool &bad, bool &nsimple) {
    constexpr int kThreads = 512;
    const int base = static_cast<int>(threadIdx.x) * E;
    int32_t x[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
        const int idx = base + i;
        x[i] = idx < d ? relabel(R, o + idx, v, static_cast<int32_t>(r), bad, nsimple) : INT_MAX;
    }
    if (threadIdx.x == 0) *s_low = 0;
    bitonic_blocked<E, kThreads>(x, smem);
    __syncthreads();  // the sort's last shared-memory readers are done
#pragma unroll
    for (int i = 0; i < E; i++) smem[base + i] = x[i];
    __syncthreads();
    int32_t *dst = R.ccol + R.coff[r];
    int low = 0;
#pragma unroll
    for (int i = 0; i < E; i++) {
        const int idx = base + i;
        if (idx < d) {
            dst[idx] = x[i];
            low += x[i] < static_cast<int32_t>(r);
            if (idx + 1 < d && smem[idx + 1] == x[i]) nsimple = true;
        }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) low += __shfl_down_sync(0xffffffffu, low, o2);
    if ((threadIdx.x & 31) == 0) atomicAdd(s_low, low);
    __syncthreads();
    if (threadIdx.x == 0) R.lowcnt[r] = *s_low;
    __syncthreads();  // s_low and smem are free for the next row
}

// Bucket of label x for the bucketed row sort: 256 buckets in label order,
// fine near the top labels and coarse far from them -- a float-like code
// (exponent and three mantissa bits) of the distance n - 1 - x from the
// top.  In degree order a long row's neighbours crowd the top labels (their
// density falls roughly as a power of that distance), which this spreads
// evenly: on the 3M-vertex graph a 1025..4096-entry row's largest bucket
// holds at most ~100 entries, against ~900 for the top 8 label bits.
__device__ __forceinline__ int row_bucket(int32_t x, int32_t top) {
    const uint32_t y1 = static_cast<uint32_t>(top - x) + 1u;  // 1 .. n
    const int e = 31 - __clz(y1);
    const uint32_t m = e >= 3 ? (y1 >> (e - 3)) & 7u : (y1 << (3 - e)) & 7u;
    return 255 - (e * 8 + static_cast<int>(m));
}

// One warp sorts the run p[0, s) of shared memory (s <= 32 E).
template <int E>
__device__ __forceinline__ void sort_run_warp(int32_t *p, int s) {
    const int lane = threadIdx.x & 31;
    int32_t x[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
        const int idx = lane * E + i;
        x[i] = idx < s ? p[idx] : INT_MAX;
    }
    bitonic_blocked<E, 32>(x, nullptr);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; i++) {
        const int idx = lane * E + i;
        if (idx < s) p[idx] = x[i];
    }
}

// Tier C by buckets: the row relabelled into shared memory, counted and
// scattered into its 256 buckets (row_bucket), each bucket sorted by one
// warp, the row written out.  A row with a bucket above 256 entries (none on
// the benchmark graphs) takes the block-wide bitonic sort above instead.
constexpr int kBucketRun = 256;

__global__ void __launch_bounds__(512, 3) k_sort_tier_c(RowIn R) {
    __shared__ int32_t s_a[kTierC];
    __shared__ int32_t s_b[kTierC];
    __shared__ uint32_t s_cnt[256], s_start[257];
    __shared__ int s_low, s_big;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t r0 = static_cast<int64_t>(R.status[ST_TIER + 2]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_TIER + 3]);
    const int32_t top = static_cast<int32_t>(R.n - 1);
    bool bad = false, nsimple = false;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int d = static_cast<int>(ldg_i64(R.off + v + 1) - o);
        if (t < 256) s_cnt[t] = 0;
        if (t == 0) {
            s_low = 0;
            s_big = 0;
        }
        __syncthreads();
        for (int i = t; i < d; i += 512) {
            const int32_t x = relabel(R, o + i, v, static_cast<int32_t>(r), bad, nsimple);
            s_a[i] = x;
            atomicAdd(&s_cnt[row_bucket(x, top)], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of the 256 counts, 8 per lane
            uint32_t c[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                c[j] = s_cnt[lane * 8 + j];
                sum += c[j];
                if (c[j] > kBucketRun) s_big = 1;
            }
            uint32_t x = sum;
#pragma unroll
            for (int off2 = 1; off2 < 32; off2 <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, off2);
                if (lane >= off2) x += y;
            }
            uint32_t run = x - sum;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                s_start[lane * 8 + j] = run;
                s_cnt[lane * 8 + j] = run;  // becomes the scatter cursor
                run += c[j];
            }
            if (lane == 31) s_start[256] = run;
        }
        __syncthreads();
        if (s_big) {
            // every thread reads s_big after the barrier, so the branch is uniform
            __syncthreads();
            sort_row_block<8>(R, r, v, o, d, s_b, &s_low, bad, nsimple);
            continue;
        }
        for (int i = t; i < d; i += 512) {
            const int32_t x = s_a[i];
            s_b[atomicAdd(&s_cnt[row_bucket(x, top)], 1u)] = x;
        }
        __syncthreads();
        for (int b = warp; b < 256; b += 16) {
            const int st = static_cast<int>(s_start[b]);
            const int sz = static_cast<int>(s_start[b + 1]) - st;
            if (sz <= 1) continue;
            if (sz <= 32) sort_run_warp<1>(s_b + st, sz);
            else if (sz <= 64) sort_run_warp<2>(s_b + st, sz);
            else if (sz <= 128) sort_run_warp<4>(s_b + st, sz);
            else sort_run_warp<8>(s_b + st, sz);
        }
        __syncthreads();
        int32_t *dst = R.ccol + R.coff[r];
        int low = 0;
        for (int i = t; i < d; i += 512) {
            const int32_t x = s_b[i];
            dst[i] = x;
            low += x < static_cast<int32_t>(r);
            if (i + 1 < d && s_b[i + 1] == x) nsimple = true;
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) low += __shfl_down_sync(0xffffffffu, low, o2);
        if (lane == 0) atomicAdd(&s_low, low);
        __syncthreads();
        if (t == 0) R.lowcnt[r] = s_low;
        __syncthreads();  // the shared arrays are free for the next row
    }
    report(R, bad, nsimple);
}

// Tier D (graphs with more than 2^20 vertices; smaller ones use the bitmap
// sort below): rows above 4096 entries, one block of 1024, stable LSD radix sort
// (8-bit digits) ping-ponging between the output row and a scratch row.  Each
// pass is a warp-level multisplit: every warp owns a contiguous slice of the
// row, counts its digits, gets per-(digit, warp) offsets from one block-wide
// scan, and scatters its slice in order -- stable without block barriers
// inside the scatter.
__global__ void __launch_bounds__(1024) k_sort_tier_d(RowIn R, int32_t *tmp, int bits) {
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_wcnt[32][256];
    __shared__ int s_low;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = static_cast<int64_t>(R.status[ST_TIER + 3]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_TIER + 4]);
    const int64_t tbase = (r0 < r1) ? R.coff[r0] : 0;
    bool bad = false, nsimple = false;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int64_t d = ldg_i64(R.off + v + 1) - o;
        int32_t *out = R.ccol + R.coff[r];
        int32_t *scr = tmp + (R.coff[r] - tbase);
        for (int64_t i = threadIdx.x; i < d; i += blockDim.x)
            scr[i] = relabel(R, o + i, v, (int32_t)r, bad, nsimple);
        __syncthreads();
        int32_t *src = scr, *dst = out;
        const int64_t slice = (d + 31) / 32;
        const int64_t lo = warp * slice;
        const int64_t hi = (lo + slice < d) ? lo + slice : d;
        for (int shift = 0; shift < bits; shift += 8) {
            // (1) per-warp digit counts of the warp's slice
            if (threadIdx.x < 256)
                for (int w = 0; w < 32; w++) s_wcnt[w][threadIdx.x] = 0;
            __syncthreads();
            for (int64_t i = lo + lane; i < hi; i += 32)
                atomicAdd(&s_wcnt[warp][(static_cast<uint32_t>(src[i]) >> shift) & 255u], 1u);
            __syncthreads();
            // (2) offsets in (digit, warp) order: digit totals, their
            // exclusive scan, then the warps in order within each digit
            if (threadIdx.x < 256) {
                uint32_t t = 0;
                for (int w = 0; w < 32; w++) t += s_wcnt[w][threadIdx.x];
                s_tot[threadIdx.x] = t;
            }
            __syncthreads();
            if (warp == 0) {
                uint32_t h[8], run = 0;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    h[q] = s_tot[lane * 8 + q];
                    run += h[q];
                }
                uint32_t x = run;
#pragma unroll
                for (int o2 = 1; o2 < 32; o2 <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o2);
                    if (lane >= o2) x += y;
                }
                uint32_t e = x - run;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    s_tot[lane * 8 + q] = e;
                    e += h[q];
                }
            }
            __syncthreads();
            if (threadIdx.x < 256) {
                uint32_t base = s_tot[threadIdx.x];
                for (int w = 0; w < 32; w++) {
                    const uint32_t c = s_wcnt[w][threadIdx.x];
                    s_wcnt[w][threadIdx.x] = base;
                    base += c;
                }
            }
            __syncthreads();
            // (3) each warp scatters its slice in order
            for (int64_t i0 = lo; i0 < hi; i0 += 32) {
                const int64_t i = i0 + lane;
                const bool valid = i < hi;
                const int32_t x = valid ? src[i] : 0;
                const uint32_t digit = valid ? ((static_cast<uint32_t>(x) >> shift) & 255u) : 256u;
                const uint32_t peers = __match_any_sync(0xffffffffu, digit);
                const uint32_t rank = __popc(peers & lanemask_lt());
                const uint32_t base = valid ? s_wcnt[warp][digit] : 0u;
                __syncwarp();
                if (valid) {
                    dst[base + rank] = x;
                    if (lane == __ffs(peers) - 1) s_wcnt[warp][digit] = base + __popc(peers);
                }
                __syncwarp();
            }
            __syncthreads();
            int32_t *t = src;
            src = dst;
            dst = t;
        }
        if (src != out) {
            for (int64_t i = threadIdx.x; i < d; i += blockDim.x) out[i] = src[i];
            __syncthreads();
        }
        if (threadIdx.x == 0) s_low = 0;
        __syncthreads();
        int low = 0;
        for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
            const int32_t x = out[i];
            low += (x < (int32_t)r);
            if (i + 1 < d && out[i + 1] == x) nsimple = true;
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) low += __shfl_down_sync(0xffffffffu, low, o2);
        if (lane == 0) atomicAdd(&s_low, low);
        __syncthreads();
        if (threadIdx.x == 0) R.lowcnt[r] = s_low;
        __syncthreads();
    }
    report(R, bad, nsimple);
}

// Rows above kTierC entries, one block of 1024 per row, sorted through a
// bitmap of labels in shared memory: a relabelled row is a set of distinct
// labels in [0, n), so setting one bit per entry and reading the bits back
// in order sorts it (a repeated entry finds its bit already set).  Labels
// are taken kBitmapBits at a time (one chunk when n <= 2^20).  Warp w owns
// words [1024 w, 1024 (w + 1)) and reads them lane-interleaved (no bank
// conflicts): one pass counts its bits, a block scan of the warp counts
// gives each warp its output base, and a second pass writes the labels in
// order -- positions from warp scans of the words' bit counts -- and clears
// each word behind it, so the bitmap is empty again for the next chunk.
constexpr int kBitmapThreads = 1024;
constexpr int kBitmapWords = 1 << 15;
constexpr int64_t kBitmapBits = 32ll * kBitmapWords;  // 2^20 labels, 128 KB
constexpr int kWarpWords = kBitmapWords / (kBitmapThreads / 32);  // 1024

__global__ void __launch_bounds__(kBitmapThreads, 1) k_sort_bitmap(RowIn R, int32_t *tmp) {
    extern __shared__ uint32_t s_bits[];
    __shared__ int s_warp[32];
    __shared__ int s_low[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = static_cast<int64_t>(R.status[ST_TIER + 3]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_TIER + 4]);
    const int64_t tbase = (r0 < r1) ? R.coff[r0] : 0;
    bool bad = false, nsimple = false;
    for (int w = tid; w < kBitmapWords; w += kBitmapThreads) s_bits[w] = 0u;
    __syncthreads();
    uint32_t *mine = s_bits + warp * kWarpWords;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int d = static_cast<int>(ldg_i64(R.off + v + 1) - o);
        int32_t *t = tmp + (R.coff[r] - tbase);
        for (int i = tid; i < d; i += kBitmapThreads)
            t[i] = relabel(R, o + i, v, static_cast<int32_t>(r), bad, nsimple);
        __syncthreads();
        int32_t *dst = R.ccol + R.coff[r];
        int written = 0, low = 0;
        for (int64_t c0 = 0; c0 < R.n; c0 += kBitmapBits) {
            for (int i = tid; i < d; i += kBitmapThreads) {
                const int64_t x = static_cast<int64_t>(t[i]) - c0;
                if (x >= 0 && x < kBitmapBits) {
                    const uint32_t m = 1u << (x & 31);
                    if (atomicOr(s_bits + (x >> 5), m) & m) nsimple = true;
                }
            }
            __syncthreads();
            int cnt = 0;
            for (int k = lane; k < kWarpWords; k += 32) cnt += __popc(mine[k]);
#pragma unroll
            for (int q = 16; q > 0; q >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, q);
            if (lane == 0) s_warp[warp] = cnt;
            __syncthreads();
            if (warp == 0) {
                const int c = s_warp[lane];
                int incl = c;
#pragma unroll
                for (int q = 1; q < 32; q <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, q);
                    if (lane >= q) incl += y;
                }
                s_warp[lane] = incl - c;  // exclusive warp bases
                if (lane == 31) s_low[0] = incl;  // chunk total
            }
            __syncthreads();
            int run = written + s_warp[warp];
            const int total = s_low[0];
            const int64_t wbase = c0 + 32ll * warp * kWarpWords;
            for (int k = lane; k < kWarpWords; k += 32) {
                uint32_t bits = mine[k];
                mine[k] = 0u;
                const int c = __popc(bits);
                int incl = c;
#pragma unroll
                for (int q = 1; q < 32; q <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, q);
                    if (lane >= q) incl += y;
                }
                int pos = run + incl - c;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int32_t label = static_cast<int32_t>(wbase + 32ll * k + b);
                    dst[pos++] = label;
                    low += label < static_cast<int32_t>(r);
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            written += total;
            __syncthreads();  // s_warp / s_low reused by the next chunk
        }
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) low += __shfl_xor_sync(0xffffffffu, low, q);
        if (lane == 0) s_low[warp] = low;
        __syncthreads();
        if (warp == 0) {
            int c = s_low[lane];
#pragma unroll
            for (int q = 16; q > 0; q >>= 1) c += __shfl_xor_sync(0xffffffffu, c, q);
            if (lane == 0) R.lowcnt[r] = c;
        }
        __syncthreads();
    }
    report(R, bad, nsimple);
}

// ------------------------------------------------------------- edge table

struct LoadUp {
    const int32_t *dnew;
    const int32_t *low;
    __device__ int64_t operator()(int64_t i) const { return (int64_t)dnew[i] - low[i]; }
};
struct StoreUbase {
    int64_t *ubase;
    int64_t n;
    u64 *status;
    __device__ void operator()(int64_t i, int64_t exc, int64_t inc) const {
        ubase[i] = exc;
        if (i == n - 1) {
            ubase[n] = inc;
            status[ST_M_UPPER] = static_cast<u64>(inc);
        }
    }
};

// Slots of a bucket are tried from the key's own first slot on, which spreads
// the first attempts over the four slots (fewer failed compare-and-swaps than
// always starting at slot 0).
__device__ __forceinline__ bool eset_insert(uint64_t *set, uint64_t mask, uint64_t key) {
    const uint64_t h = key_hash(key);
    const int first = static_cast<int>(h >> (64 - kBucketShift));
    uint64_t b = h & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        unsigned long long *slot = reinterpret_cast<unsigned long long *>(set + (b << kBucketShift));
        for (int q = 0; q < kBucketSlots; q++) {
            const unsigned long long old =
                atomicCAS(slot + ((first + q) & (kBucketSlots - 1)), kEmptySlot, key);
            if (old == kEmptySlot || old == key) return true;
        }
        b = (b + 1) & mask;
    }
    return false;
}

// Inserts every edge {r, x}, r < x, into the hash set with compare-and-swap:
// the upper arcs of the sorted rows (row r's entries after its lowcnt[r]
// lower ones) are exactly the edges, so the set needs neither the edge table
// nor its order and is built as soon as the rows are sorted, on a side
// stream beside the edge table.  The set's contents are deterministic, its
// slot layout is not.  kInsertBatch keys per lane: their first
// compare-and-swaps are issued together (most succeed at once), and only
// the keys whose first slot was taken go on to the full insertion.
constexpr int kInsertBatch = 4;
// resident blocks per SM of the direct hash set build (4, 8 and 16 measured
// the same)
constexpr int kEsetBlocksPerSm = 8;

__device__ __forceinline__ bool eset_insert_batch(uint64_t *set, uint64_t mask, const uint64_t (&key)[kInsertBatch],
                                                  const bool (&ok)[kInsertBatch]) {
    unsigned long long old[kInsertBatch];
#pragma unroll
    for (int u = 0; u < kInsertBatch; u++) {
        old[u] = kEmptySlot;
        if (ok[u]) {
            const uint64_t h = key_hash(key[u]);
            const int first = static_cast<int>(h >> (64 - kBucketShift));
            unsigned long long *slot = reinterpret_cast<unsigned long long *>(set + ((h & mask) << kBucketShift));
            old[u] = atomicCAS(slot + first, kEmptySlot, key[u]);
        }
    }
    bool good = true;
#pragma unroll
    for (int u = 0; u < kInsertBatch; u++)
        if (ok[u] && old[u] != kEmptySlot && old[u] != key[u]) good &= eset_insert(set, mask, key[u]);
    return good;
}

// The upper arcs in row-major order are the edges in edge order: edge
// t = ubase[r] + q is the q-th upper arc of row r, at position
// lowcnt[r] + q of N(r).  Each warp takes kEsetChunk consecutive edges (rows
// are in degree order, so 32 consecutive rows can hold 32 sqrt(2m) edges:
// the work is split by edges, not rows): it finds the row of its first edge
// by a binary search of ubase, then walks windows of 32 rows, each lane
// finding its edges' rows within the window by a shuffle search of their
// ubase values, and hands kInsertBatch keys per lane at a time to `f`.
constexpr int64_t kEsetChunk = 1024;

template <typename F>
__device__ __forceinline__ void for_each_edge_key(int64_t n, int64_t m, const int64_t *__restrict__ coff,
                                                  const int32_t *__restrict__ ccol, const int32_t *__restrict__ lowcnt,
                                                  const int64_t *__restrict__ ubase, F &f) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; c * kEsetChunk < m; c += nwarps) {
        const int64_t t_lo = c * kEsetChunk, t_hi = (t_lo + kEsetChunk < m) ? t_lo + kEsetChunk : m;
        // the row holding edge t_lo: the last r with ubase[r] <= t_lo
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (ldg_i64(ubase + mid) <= t_lo) lo = mid;
            else hi = mid - 1;
        }
        // every window advances r0, so the walk ends by the last row even when
        // an asymmetric input has fewer edges than the chunks cover
        for (int64_t r0 = lo, t = t_lo; t < t_hi && r0 < n; r0 += 32) {
            const int64_t r = r0 + lane;
            int64_t ub = m, first = 0;  // lanes past the last row never match
            if (r < n) {
                ub = ldg_i64(ubase + r);
                first = ldg_i64(coff + r) + ldg_i32(lowcnt + r);  // the row's first upper arc
            }
            const int64_t w_end = ldg_i64(ubase + (r0 + 32 < n ? r0 + 32 : n));
            const int64_t seg_end = w_end < t_hi ? w_end : t_hi;
            for (int64_t t0 = t; t0 < seg_end; t0 += 32 * kInsertBatch) {
                uint64_t key[kInsertBatch];
                bool ok[kInsertBatch];
#pragma unroll
                for (int u = 0; u < kInsertBatch; u++) {
                    const int64_t tt = t0 + 32 * u + lane;
                    int at = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int64_t x = __shfl_sync(0xffffffffu, ub, at + step);
                        if (x <= tt) at += step;
                    }
                    const int64_t i = __shfl_sync(0xffffffffu, first, at) + (tt - __shfl_sync(0xffffffffu, ub, at));
                    ok[u] = tt < seg_end;
                    key[u] = ok[u] ? edge_key(static_cast<int32_t>(r0 + at), ldg_i32(ccol + i)) : 0ull;
                }
                f(key, ok);
            }
            t = seg_end;
        }
    }
}

// Direct build (tables smaller than one region, or no scratch): every key
// inserted with compare-and-swap into the table in global memory.
struct InsertDirect {
    uint64_t *set;
    uint64_t mask;
    bool failed;
    __device__ void operator()(const uint64_t (&key)[kInsertBatch], const bool (&ok)[kInsertBatch]) {
        failed |= !eset_insert_batch(set, mask, key, ok);
    }
};

__global__ void __launch_bounds__(256)
k_eset_upper(int64_t n, int64_t m, const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
             const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase, uint64_t *set, uint64_t mask,
             u64 *status) {
    InsertDirect f{set, mask, false};
    for_each_edge_key(n, m, coff, ccol, lowcnt, ubase, f);
    if (f.failed) raise_flag(status, F_OVERFLOW);
}

// Region build.  The table is cut into regions of kRegionBuckets buckets
// (64 KB), each small enough for one block's shared memory.  The edge-table
// kernel appends every key to the list of its home bucket's region
// (EsetLists); then one block per region inserts that region's keys with
// shared-memory compare-and-swap, probing linearly within the region, and
// writes the whole region out (empty slots included, so the table needs no
// clearing).  A key whose probe runs past its region's end goes to the
// overflow list, and that list is inserted at the end by ordinary global
// compare-and-swap, probing on into the following regions -- already
// written, so every bucket between a key's home and its place is full, as a
// lookup assumes.  The random read-modify-writes of the direct build become
// sequential writes of the table plus the key lists' traffic.
constexpr int kRegionThreads = 512;

// One block per region (grid-stride): the region's keys into shared memory,
// then the region written out.
__global__ void __launch_bounds__(kRegionThreads)
k_eset_regions(int64_t regions, int64_t region_buckets, EsetLists lists, uint64_t *set, u64 *status) {
    extern __shared__ unsigned long long s_tab[];
    const int64_t slots = region_buckets << kBucketShift;
    for (int64_t reg = blockIdx.x; reg < regions; reg += gridDim.x) {
        for (int64_t q = threadIdx.x; q < slots; q += kRegionThreads) s_tab[q] = kEmptySlot;
        __syncthreads();
        const int64_t b0 = reg * region_buckets;
        const int64_t len = lists.cur[reg] < lists.cap ? lists.cur[reg] : lists.cap;
        uint64_t *list = lists.keys + reg * lists.cap;
        for (int64_t e = threadIdx.x; e < len; e += kRegionThreads) {
            const unsigned long long key = list[e];
            const uint64_t h = key_hash(key);
            const int first = static_cast<int>(h >> (64 - kBucketShift));
            bool placed = false;
            for (int64_t b = static_cast<int64_t>(h & lists.mask) - b0; b < region_buckets && !placed; b++) {
                for (int q = 0; q < kBucketSlots; q++) {
                    const unsigned long long old =
                        atomicCAS(s_tab + (b << kBucketShift) + ((first + q) & (kBucketSlots - 1)), kEmptySlot, key);
                    if (old == kEmptySlot || old == key) {
                        placed = true;
                        break;
                    }
                }
            }
            if (!placed) {  // rare: every bucket from its home to the region's end is full
                const uint32_t o = atomicAdd(lists.ov_count, 1u);
                if (o < lists.ov_cap) lists.ov_keys[o] = key;
                else status[ST_ESET_SPILL] = 1;
            }
        }
        __syncthreads();
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(set) + (b0 << kBucketShift);
        for (int64_t q = threadIdx.x; q < slots; q += kRegionThreads) dst[q] = s_tab[q];
        __syncthreads();
    }
}

// The overflow list (keys beyond their region list's capacity, and keys
// whose probe ran past their region): global compare-and-swap.
__global__ void __launch_bounds__(256)
k_eset_leftovers(EsetLists lists, uint64_t *set, u64 *status) {
    const int64_t ov = *lists.ov_count < lists.ov_cap ? *lists.ov_count : lists.ov_cap;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool failed = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ov; e += stride)
        failed |= !eset_insert(set, lists.mask, lists.ov_keys[e]);
    if (failed) raise_flag(status, F_OVERFLOW);
}

// The slow path, only when the overflow list itself overflowed (the keys it
// could not hold are in no list): every edge inserted again by direct
// compare-and-swap (a key already present stops at once).
__global__ void __launch_bounds__(256)
k_eset_spill_fallback(int64_t n, int64_t m, const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
                      const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase, uint64_t *set,
                      uint64_t mask, u64 *status) {
    if (ld_acquire(reinterpret_cast<const uint32_t *>(status + ST_ESET_SPILL)) == 0u) return;
    InsertDirect f{set, mask, false};
    for_each_edge_key(n, m, coff, ccol, lowcnt, ubase, f);
    if (f.failed) raise_flag(status, F_OVERFLOW);
}

// ------------------------------------------------------------------- driver

// Runs independent kernels of one call on the device's side streams: fork()
// makes them wait for the caller's stream, join() makes the caller's stream
// wait for them.  The destructor joins on every return path, so no side work
// outlives a call that failed halfway.  Without side streams every kernel
// runs on the caller's stream.
class SideFork {
  public:
    SideFork(ps_graph *g, cudaStream_t s) : g_(g), s_(s) { side_[0] = side_[1] = s; }
    ~SideFork() { join(); }
    SideFork(const SideFork &) = delete;
    SideFork &operator=(const SideFork &) = delete;

    int fork(int count) {
        cudaStream_t side[2];
        if (get_side_streams(g_->device, side) != PS_OK) return PS_OK;
        PS_CUDA_TRY(cudaEventRecord(g_->ev[0], s_));
        for (int i = 0; i < count; i++) {
            PS_CUDA_TRY(cudaStreamWaitEvent(side[i], g_->ev[0], 0));
            side_[i] = side[i];
            used_ = i + 1;
        }
        return PS_OK;
    }
    cudaStream_t side(int i) const { return side_[i]; }
    int join() {
        int rc = PS_OK;
        for (int i = 0; i < used_; i++)
            if (cudaEventRecord(g_->ev[1 + i], side_[i]) != cudaSuccess ||
                cudaStreamWaitEvent(s_, g_->ev[1 + i], 0) != cudaSuccess)
                rc = PS_ERR_CUDA;
        used_ = 0;
        return rc;
    }

  private:
    ps_graph *g_;
    cudaStream_t s_;
    cudaStream_t side_[2];
    int used_ = 0;
};

int load_graph(ps_graph *g, const int64_t *d_off, const int32_t *d_col, cudaStream_t s) {
    const Layout &L = g->L;
    const int64_t n = L.n, nnz = L.nnz;
    char *ws = g->ws;
    const int sms = g->sm_count;
    PS_CUDA_TRY(cudaMemsetAsync(g->status, 0, ST_WORDS * sizeof(uint64_t), s));
    PS_CUDA_TRY(cudaMemsetAsync(g->lowcnt, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
    uint32_t *k0 = reinterpret_cast<uint32_t *>(ws + L.keys0);
    uint32_t *k1 = reinterpret_cast<uint32_t *>(ws + L.keys1);
    uint32_t *v0 = reinterpret_cast<uint32_t *>(ws + L.vals0);
    uint32_t *v1 = reinterpret_cast<uint32_t *>(ws + L.vals1);

    // (1) degrees and offset validation; nothing else may index with bad offsets
    k_degrees<<<sms * 8, 256, 0, s>>>(n, nnz, d_off, k0, v0, g->status);
    PS_LAUNCH_CHECK();
    uint64_t st[ST_WORDS];
    PS_CUDA_TRY(cudaMemcpyAsync(st, g->status, sizeof(st), cudaMemcpyDeviceToHost, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    if (st[ST_FLAGS] & F_ARG) return PS_ERR_ARG;
    g->d_max = static_cast<int64_t>(st[ST_DMAX]);

    // (2) stable LSD radix sort of (degree, id): ties keep increasing id
    int bits = 0;
    while (bits < 32 && (static_cast<uint64_t>(g->d_max) >> bits) != 0) bits++;
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws + L.rcounts);
    const int64_t tiles = L.radix_tiles;
    for (int shift = 0; shift < bits && n > 0; shift += 8) {
        k_radix_hist<<<(unsigned)tiles, kRadixBlock, 0, s>>>(n, k0, shift, counts, tiles);
        PS_LAUNCH_CHECK();
        int rc = run_scan<uint32_t>(g, 0, 256 * tiles, 0u, OpSum(), LoadU32{counts},
                                    StoreExclU32{counts}, s);
        if (rc) return rc;
        k_radix_scatter<<<(unsigned)tiles, kRadixBlock, 0, s>>>(n, k0, v0, k1, v1, shift, counts,
                                                                tiles);
        PS_LAUNCH_CHECK();
        uint32_t *t = k0;
        k0 = k1;
        k1 = t;
        t = v0;
        v0 = v1;
        v1 = t;
    }
    // k0/v0 hold the sorted (degree, vertex) pairs; v1 receives inv[r]
    if (n > 0) {
        k_rank<<<sms * 8, 256, 0, s>>>(n, k0, v0, g->rank, g->dnew, v1);
        PS_LAUNCH_CHECK();
    }
    const uint32_t *inv = v1;
    PS_CUDA_TRY(cudaMemsetAsync(g->off, 0, sizeof(int64_t), s));
    int rc = run_scan<int64_t>(g, 1, n, (int64_t)0, OpSum(), LoadDeg{g->dnew}, StoreOffsets{g->off, n}, s);
    if (rc) return rc;
    k_tiers<<<1, 32, 0, s>>>(n, g->dnew, g->status);
    PS_LAUNCH_CHECK();

    // (3) relabel + sort every row, by tier; the tiers touch disjoint rows, so
    // the long-row tiers run on side streams next to the short-row ones
    RowIn R{d_off, d_col, inv, g->rank, g->off, g->col, g->lowcnt, n, g->status};
    if (n > 0) {
        SideFork fork(g, s);
        if (g->d_max > kTierB) {
            rc = fork.fork(2);
            if (rc) return rc;
        }
        // rows above kTierC: the bitmap sort when all labels fit one chunk
        // (R-MAT 20: 0.11 ms against 0.25 ms for the radix sort), the block
        // radix sort otherwise (3 chunks on the 3M-vertex graph: +0.4 ms)
        const bool bitmap = n <= kBitmapBits;
        if (bitmap && g->d_max > kTierC) {
            const int smem = kBitmapWords * static_cast<int>(sizeof(uint32_t));
            PS_CUDA_TRY(cudaFuncSetAttribute(k_sort_bitmap, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_sort_bitmap<<<sms, kBitmapThreads, smem, fork.side(1)>>>(R, reinterpret_cast<int32_t *>(g->rec));
            PS_LAUNCH_CHECK();
        }
        if (!bitmap && g->d_max > kTierC) {
            int vb = 0;
            while (vb < 31 && (static_cast<uint64_t>(n - 1) >> vb) != 0) vb++;
            k_sort_tier_d<<<sms * 2, 1024, 0, fork.side(1)>>>(R, reinterpret_cast<int32_t *>(g->rec), vb);
            PS_LAUNCH_CHECK();
        }
        if (g->d_max > kTierB) {
            k_sort_tier_c<<<sms * 3, 512, 0, fork.side(0)>>>(R);
            PS_LAUNCH_CHECK();
        }
        k_sort_tier_b<<<sms * 8, 256, 0, s>>>(R);
        PS_LAUNCH_CHECK();
        if (g->d_max > kLongRow) {
            k_sort_tier_b2<<<sms * 4, 256, 0, s>>>(R);
            PS_LAUNCH_CHECK();
        }
        k_sort_tier_a<<<sms * 16, 256, 0, s>>>(R);
        PS_LAUNCH_CHECK();
        rc = fork.join();
        if (rc) return rc;
    }

    // (4) the edge numbering: ubase[r] = the edges (upper arcs) of the rows before r
    PS_CUDA_TRY(cudaMemsetAsync(g->ubase, 0, sizeof(int64_t), s));
    rc = run_scan<int64_t>(g, 2, n, (int64_t)0, OpSum(), LoadUp{g->dnew, g->lowcnt},
                           StoreUbase{g->ubase, n, g->status}, s);
    if (rc) return rc;

    // (5) the edge table; with the region build of the hash set (tables of
    // at least one region), its kernel also lists every edge's key by region
    const bool region_build = nnz > 0 && g->eset && L.eset_regions > 0;
    EsetLists lists{};
    if (region_build) {
        int shift = 0;
        while ((int64_t{1} << shift) < kRegionBuckets) shift++;
        lists.cur = reinterpret_cast<uint32_t *>(ws + L.eregion);
        lists.ov_count = lists.cur + L.eset_regions;
        lists.keys = reinterpret_cast<uint64_t *>(ws + L.ekeys);
        lists.ov_keys = lists.keys + L.eset_regions * L.eset_cap;
        lists.cap = L.eset_cap;
        lists.ov_cap = L.eset_ov_cap;
        lists.mask = static_cast<uint64_t>(L.eset_buckets - 1);
        lists.shift = shift;
        PS_CUDA_TRY(cudaMemsetAsync(lists.cur, 0, sizeof(uint32_t) * (L.eset_regions + 1), s));
    }
    rc = build_edge_table(g, s, region_build ? &lists : nullptr);
    if (rc) return rc;

    // (6) the edge hash set.  Only sampling reads it, so it is built on a side
    // stream beside the prefix step; ps_tau_prefix waits for it before its end
    // (wait_eset).
    if (nnz > 0 && g->eset) {
        cudaStream_t es = s;
        cudaStream_t side[2];
        if (get_side_streams(g->device, side) == PS_OK) {
            PS_CUDA_TRY(cudaEventRecord(g->ev[0], s));
            PS_CUDA_TRY(cudaStreamWaitEvent(side[0], g->ev[0], 0));
            es = side[0];
        }
        g->eset_pending = true;
        const uint64_t eset_mask = static_cast<uint64_t>(L.eset_buckets - 1);
        const int64_t m_cap = L.m_cap;
        int64_t eb = ((m_cap + kEsetChunk - 1) / kEsetChunk + 7) / 8;  // a warp per chunk of edges
        if (eb > (int64_t)sms * kEsetBlocksPerSm) eb = (int64_t)sms * kEsetBlocksPerSm;
        if (eb < 1) eb = 1;
        if (region_build) {
            const int64_t regions = L.eset_regions;
            const int smem = static_cast<int>(kRegionBuckets * kBucketSlots * sizeof(uint64_t));
            PS_CUDA_TRY(cudaFuncSetAttribute(k_eset_regions, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            const int64_t rb = regions < (int64_t)sms * 3 ? regions : (int64_t)sms * 3;
            k_eset_regions<<<(unsigned)rb, kRegionThreads, smem, es>>>(regions, kRegionBuckets, lists, g->eset,
                                                                       g->status);
            PS_LAUNCH_CHECK();
            int64_t lb = (L.eset_ov_cap + 255) / 256;
            if (lb > (int64_t)sms * 4) lb = (int64_t)sms * 4;
            k_eset_leftovers<<<(unsigned)lb, 256, 0, es>>>(lists, g->eset, g->status);
            PS_LAUNCH_CHECK();
            k_eset_spill_fallback<<<(unsigned)eb, 256, 0, es>>>(n, m_cap, g->off, g->col, g->lowcnt, g->ubase,
                                                               g->eset, eset_mask, g->status);
            PS_LAUNCH_CHECK();
        } else {
            PS_CUDA_TRY(cudaMemsetAsync(g->eset, 0xFF, sizeof(uint64_t) * kBucketSlots * L.eset_buckets, es));
            k_eset_upper<<<(unsigned)eb, 256, 0, es>>>(n, m_cap, g->off, g->col, g->lowcnt, g->ubase, g->eset,
                                                      eset_mask, g->status);
            PS_LAUNCH_CHECK();
        }
        PS_CUDA_TRY(cudaEventRecord(g->ev[3], es));
    }

    // N_1 and the hub count (for ps_tau_prefix), read back with the flags
    rc = launch_vertex_totals(g, s);
    if (rc) return rc;
    PS_CUDA_TRY(cudaMemcpyAsync(st, g->status, sizeof(st), cudaMemcpyDeviceToHost, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    g->load_totals[0] = st[ST_W_LO];
    g->load_totals[1] = st[ST_L_LO];
    g->load_totals[2] = st[ST_N1_LO];
    g->load_totals[3] = st[ST_N1_HI];
    g->load_totals[4] = st[ST_HUBS];
    g->load_flags = st[ST_FLAGS];
    const uint64_t m_upper = st[ST_M_UPPER];
    uint64_t flags = st[ST_FLAGS];
    if (2 * m_upper != static_cast<uint64_t>(nnz)) flags |= F_ASYM;
    // a prefix sum past 2^64 is reported by ps_tau_prefix, as documented
    const int status = flags_to_status(flags & ~static_cast<uint64_t>(F_OVERFLOW));
    if (status != PS_OK) return status;
    g->m = static_cast<int64_t>(m_upper);
    return PS_OK;
}

}  // namespace ps
