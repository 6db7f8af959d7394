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

template <typename T, typename Op, typename Load, typename Store>
static int run_scan(ps_graph *g, int slot, int64_t count, T identity, Op op, Load load, Store store,
                    cudaStream_t s) {
    if (count <= 0) return PS_OK;
    int rc = reset_scan(g, slot, count, s);
    if (rc) return rc;
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    k_scan<T, kScanBlock, kScanItems><<<(unsigned)tiles, kScanBlock, 0, s>>>(
        count, scan_state<T>(g, slot), identity, op, load, store);
    PS_LAUNCH_CHECK();
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

// arcrow[q] = the row holding arc q << kArcRowShift (every such arc lies in
// exactly one non-empty row); arcrow[Q] = n - 1 closes the last interval.
// Kernels that give each thread a run of arcs find its row between two
// entries instead of searching all n offsets.
__global__ void k_arc_rows(int64_t n, int64_t nnz, const int64_t *__restrict__ coff, int32_t *arcrow) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t q_end = (nnz + (1ll << kArcRowShift) - 1) >> kArcRowShift;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int64_t a = coff[r], b = coff[r + 1];
        for (int64_t q = (a + (1ll << kArcRowShift) - 1) >> kArcRowShift; (q << kArcRowShift) < b; q++)
            arcrow[q] = static_cast<int32_t>(r);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) arcrow[q_end] = static_cast<int32_t>(n > 0 ? n - 1 : 0);
}

// Row of arc i (the last row r with coff[r] <= i), searched between the
// arc-to-row entries around i.
__device__ __forceinline__ int64_t row_of_arc(const int64_t *coff, const int32_t *arcrow, int64_t i) {
    const int64_t q = i >> kArcRowShift;
    int64_t lo = ldg_i32(arcrow + q), hi = ldg_i32(arcrow + q + 1);
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (ldg_i64(coff + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// first row whose degree exceeds each tier limit (rows are degree-sorted)
__global__ void k_tiers(int64_t n, const int32_t *__restrict__ dnew, u64 *status) {
    const int lim[4] = {0, kTierA, kTierB, kTierC};
    const int t = threadIdx.x;
    if (t < 4) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (dnew[mid] > lim[t]) hi = mid;
            else lo = mid + 1;
        }
        status[ST_TIER + t] = static_cast<u64>(lo);
    }
    if (t == 4) status[ST_TIER + 4] = static_cast<u64>(n);
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

// Tier B: rows of 33..1024 entries, one warp, bitonic network in registers.
// (Capped at 64 registers: four blocks per SM beat the spill-free 105-register
// build; the same holds for tier C at three blocks.)
__global__ void __launch_bounds__(256, 4) k_sort_tier_b(RowIn R) {
    const int64_t r0 = static_cast<int64_t>(R.status[ST_TIER + 1]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_TIER + 2]);
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    bool bad = false, nsimple = false;
    for (int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < r1; r += nw) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int d = static_cast<int>(ldg_i64(R.off + v + 1) - o);
        if (d <= 64) sort_row_warp<2>(R, r, v, o, d, bad, nsimple);
        else if (d <= 128) sort_row_warp<4>(R, r, v, o, d, bad, nsimple);
        else if (d <= 256) sort_row_warp<8>(R, r, v, o, d, bad, nsimple);
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

__global__ void __launch_bounds__(512, 3) k_sort_tier_c(RowIn R) {
    extern __shared__ int32_t s_dyn[];
    __shared__ int s_low;
    const int64_t r0 = static_cast<int64_t>(R.status[ST_TIER + 2]);
    const int64_t r1 = static_cast<int64_t>(R.status[ST_TIER + 3]);
    bool bad = false, nsimple = false;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const uint32_t v = R.inv[r];
        const int64_t o = ldg_i64(R.off + v);
        const int d = static_cast<int>(ldg_i64(R.off + v + 1) - o);
        if (d <= 2048) sort_row_block<4>(R, r, v, o, d, s_dyn, &s_low, bad, nsimple);
        else sort_row_block<8>(R, r, v, o, d, s_dyn, &s_low, bad, nsimple);
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

// Edge j = (u, v), u < v, in row-major order: j = ubase[u] + (iu - lowcnt[u]).
// Each lower arc (v -> u, at position jv of N(v)) finds v in the upper part
// of N(u) and writes the whole 32-byte record of its edge: a full sector, so
// the scattered writes cost no partial-sector traffic.  The upper part of
// N(u) holds only neighbours of degree >= d_u, so it has at most sqrt(2m)
// entries (the searches from the other side, in lower parts, are about 2^3.7
// times longer on skewed graphs); the search halves it down to a window of
// kEdgeWindow entries and then reads the whole window with independent loads
// (one memory round trip instead of four dependent ones).  A lower arc
// without its upper partner means an asymmetric input.
constexpr int kEdgeItems = 8;
constexpr int kEdgeWindow = 16;
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

// (Advancing four arcs' searches in step, and full occupancy at 32
// registers, both measured slower.)
__global__ void __launch_bounds__(256)
k_edges(int64_t n, int64_t nnz, const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
        const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase,
        const int32_t *__restrict__ arcrow, EdgeRec *rec, int64_t m_cap, u64 *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool asym = false;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c * kEdgeItems < nnz; c += stride) {
        const int64_t i0 = c * kEdgeItems;
        int64_t r = row_of_arc(coff, arcrow, i0);
        int64_t ro = ldg_i64(coff + r);
        int64_t rend = ldg_i64(coff + r + 1);
        for (int t = 0; t < kEdgeItems; t++) {
            const int64_t i = i0 + t;
            if (i >= nnz) break;
            while (rend <= i) {
                r++;
                ro = rend;
                rend = ldg_i64(coff + r + 1);
            }
            const int32_t x = ldg_i32(ccol + i);
            if (x >= r) continue;  // upper arcs are written from the other side
            const int64_t ox = ldg_i64(coff + x);
            const int32_t lx = ldg_i32(lowcnt + x);
            const int64_t dx = ldg_i64(coff + x + 1) - ox;
            // r sits in the upper part [a, b) of N(x) when the input is symmetric
            int64_t a = ox + lx, b = ox + dx;
            while (b - a > kEdgeWindow) {
                const int64_t mid = a + ((b - a) >> 1);
                if (ldg_i32(ccol + mid) <= r) a = mid;
                else b = mid;
            }
            int below = 0;
            bool hit = false;
#pragma unroll
            for (int w = 0; w < kEdgeWindow; w++)
                if (a + w < b) {
                    const int32_t c = ldg_i32(ccol + a + w);
                    below += c < r;
                    hit |= c == r;
                }
            if (!hit) {
                asym = true;
                continue;
            }
            const int32_t iu = static_cast<int32_t>(a + below - ox);
            const int64_t j = ldg_i64(ubase + x) + (iu - lx);
            if (j < 0 || j >= m_cap) {
                asym = true;
                continue;
            }
            const int32_t dr = static_cast<int32_t>(rend - ro);
            const int32_t p = static_cast<int32_t>(i - ro);
            int4 *e = reinterpret_cast<int4 *>(rec + j);
            e[0] = make_int4(x, static_cast<int32_t>(r), static_cast<int32_t>(dx), dr);
            e[1] = make_int4(iu, p, static_cast<int32_t>(ox), static_cast<int32_t>(ro));
        }
    }
    if (asym) raise_flag(status, F_ASYM);
}

// Inserts every edge (u < v) of the edge table into the hash set with
// compare-and-swap; the set's contents are deterministic, its slot layout is
// not.  (A separate pass: inside the edge-table kernel the dependent CAS
// chains stall threads that are already waiting on their searches, and
// reading the keys from the sorted rows instead of the table's coalesced
// (u, v) pairs measured 2.7x slower.)
__global__ void __launch_bounds__(256)
k_eset_build(int64_t m, const EdgeRec *__restrict__ rec, uint64_t *set, uint64_t mask, u64 *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool failed = false;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const int2 uv = __ldg(reinterpret_cast<const int2 *>(rec + j));
        failed |= !eset_insert(set, mask, edge_key(uv.x, uv.y));
    }
    if (failed) raise_flag(status, F_OVERFLOW);
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
    if (n > 0) {
        k_arc_rows<<<sms * 4, 256, 0, s>>>(n, nnz, g->off, g->arcrow);
        PS_LAUNCH_CHECK();
    }
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
            const int smem = kTierC * (int)sizeof(int32_t);
            k_sort_tier_c<<<sms * 4, 512, smem, fork.side(0)>>>(R);
            PS_LAUNCH_CHECK();
        }
        k_sort_tier_b<<<sms * 4, 256, 0, s>>>(R);
        PS_LAUNCH_CHECK();
        k_sort_tier_a<<<sms * 16, 256, 0, s>>>(R);
        PS_LAUNCH_CHECK();
        rc = fork.join();
        if (rc) return rc;
    }

    // (4) the edge numbering and the edge table
    PS_CUDA_TRY(cudaMemsetAsync(g->ubase, 0, sizeof(int64_t), s));
    rc = run_scan<int64_t>(g, 2, n, (int64_t)0, OpSum(), LoadUp{g->dnew, g->lowcnt},
                           StoreUbase{g->ubase, n, g->status}, s);
    if (rc) return rc;
    if (nnz > 0) {
        int64_t blocks = ((nnz + kEdgeItems - 1) / kEdgeItems + 255) / 256;
        if (blocks > (int64_t)sms * 64) blocks = (int64_t)sms * 64;
        k_edges<<<(unsigned)blocks, 256, 0, s>>>(n, nnz, g->off, g->col, g->lowcnt, g->ubase, g->arcrow,
                                                 g->rec, L.m_cap, g->status);
        PS_LAUNCH_CHECK();
    }

    // (5) the edge hash set.  Only sampling reads it, so it is built on a side
    // stream and left running: the caller's stream goes on to the prefixes,
    // which wait for it only before their final status read (wait_eset).
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
        PS_CUDA_TRY(cudaMemsetAsync(g->eset, 0xFF, sizeof(uint64_t) * kBucketSlots * L.eset_buckets, es));
        // four blocks per SM: room for the prefix step's kernels beside it
        // (the full-width grid measured 0.08 ms slower on R-MAT 20, 0.9 ms on
        // the 3M-vertex graph)
        int64_t eb = (L.m_cap + 255) / 256;
        if (eb > (int64_t)sms * 4) eb = (int64_t)sms * 4;
        if (eb < 1) eb = 1;
        k_eset_build<<<(unsigned)eb, 256, 0, es>>>(L.m_cap, g->rec, g->eset, eset_mask, g->status);
        PS_LAUNCH_CHECK();
        PS_CUDA_TRY(cudaEventRecord(g->ev[3], es));
    }
    PS_CUDA_TRY(cudaMemcpyAsync(st, g->status, sizeof(st), cudaMemcpyDeviceToHost, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    const uint64_t m_upper = st[ST_M_UPPER];
    uint64_t flags = st[ST_FLAGS];
    if (2 * m_upper != static_cast<uint64_t>(nnz)) flags |= F_ASYM;
    const int status = flags_to_status(flags);
    if (status != PS_OK) return status;
    g->m = static_cast<int64_t>(m_upper);
    return PS_OK;
}

}  // namespace ps
