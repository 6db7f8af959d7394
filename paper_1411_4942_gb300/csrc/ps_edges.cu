// ps_edges.cu -- the edge table of Sections 3-4 by transposition.
//
// Edge j = (u, v), u < v, is the j-th upper arc in row-major order of the
// canonical CSR: j = ubase[u] + (iu - lowcnt[u]), iu the position of v in
// N(u).  Its record also needs jv, the position of u in N(v).  Listing the
// lower arcs (v -> u, u < v) in row-major order gives the same edges ordered
// by (v, u); a STABLE sort of that list by u orders them by (u, v), which is
// exactly the edge order.  So after the sort, entry j names edge j: u is its
// key, the arc's index i gives jv = i - off(v), and v is the (j - ubase[u])-th
// upper neighbour of u.  No per-edge search is needed, and every record is
// written in order (coalesced 32-byte stores).  The same kernel computes the
// weights tau_j and lambda_j and their exact prefixes (a look-back scan in
// edge order), so the prefix step never reads the records back.
//
// The sort is an LSD radix sort with 8-bit digits over the bits of n - 1 (3
// passes for up to 2^24 vertices).  Each pass: per-tile digit counts, one
// scan of the counts (digit-major, so it yields every (digit, tile) run's
// global offset), then a scatter in which every tile ranks its items stably
// in shared memory -- each warp ranks its own contiguous slice with
// __match_any_sync, warps in order -- and writes each digit's run
// contiguously.
//
// Scratch (the load step's own; nothing here is live afterwards): the
// ping-pong (key, value) buffers use the prefix regions of the workspace
// (P_tau and P_lambda, 8 bytes per edge each) and, for the sorted list, the
// G_tau region (written only later, by the guide-table build); the digit
// counts have their own region.
#include "ps_internal.h"

namespace ps {

constexpr int kSortBlock = 256;
constexpr int kSortItems = 16;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int64_t kSortTile = static_cast<int64_t>(kSortBlock) * kSortItems;

int64_t edge_sort_tiles(int64_t m) { return m > 0 ? (m + kSortTile - 1) / kSortTile : 1; }

// (1) The lower arcs of every row, compacted in row-major order: entry
// t = lbase(r) + p for the p-th entry of row r (p < lowcnt[r]), where
// lbase(r) = off(r) - ubase[r] counts the lower arcs of the rows before r.
// key = the smaller endpoint, value = the arc's index.  Rows up to kLongRow
// entries (labels below ST_LONG; rows are in degree order): warp w takes
// rows [32 w, 32 w + 32), whose lower arcs are one contiguous range of the
// output, written 32 * kListBatch entries at a time, each lane finding its
// entries' rows among the warp's 32 by a shuffle search of their lbase values
// (the batch's column reads are independent, so they are in flight
// together).  Longer rows: a warp per row up to kTierC entries, a block per
// row above.  An asymmetric input can have
// more lower arcs than the buffers hold; those beyond m_cap are dropped (the
// status check after the load rejects the graph).
constexpr int kListBatch = 4;

__global__ void __launch_bounds__(256)
k_lower_arcs(int64_t n, const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
             const int64_t *__restrict__ ubase, uint32_t *__restrict__ key, uint32_t *__restrict__ val,
             int64_t m_cap, const u64 *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    const int64_t r_long = static_cast<int64_t>(status[ST_LONG]);
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w * 32 < r_long; w += nwarps) {
        const int64_t r = w * 32 + lane;
        const int64_t r_end = (w * 32 + 32 < r_long) ? w * 32 + 32 : r_long;
        const int64_t lb_end = ldg_i64(coff + r_end) - ldg_i64(ubase + r_end);
        int64_t o = 0, lb = lb_end;  // lanes past the last row never match
        if (r < r_end) {
            o = ldg_i64(coff + r);
            lb = o - ldg_i64(ubase + r);
        }
        const int64_t lb0 = __shfl_sync(0xffffffffu, lb, 0);
        for (int64_t t0 = lb0; t0 < lb_end; t0 += 32 * kListBatch) {
            int64_t t[kListBatch], i[kListBatch];
            int32_t c[kListBatch];
#pragma unroll
            for (int u = 0; u < kListBatch; u++) {
                t[u] = t0 + 32 * u + lane;
                // the last lane whose row starts at or before t holds t
                int at = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int64_t x = __shfl_sync(0xffffffffu, lb, at + step);
                    if (x <= t[u]) at += step;
                }
                i[u] = __shfl_sync(0xffffffffu, o, at) + (t[u] - __shfl_sync(0xffffffffu, lb, at));
            }
#pragma unroll
            for (int u = 0; u < kListBatch; u++) c[u] = (t[u] < lb_end && t[u] < m_cap) ? ldg_i32(ccol + i[u]) : 0;
#pragma unroll
            for (int u = 0; u < kListBatch; u++)
                if (t[u] < lb_end && t[u] < m_cap) {
                    key[t[u]] = static_cast<uint32_t>(c[u]);
                    val[t[u]] = static_cast<uint32_t>(i[u]);
                }
        }
    }
}

// Rows of kLongRow + 1 .. kTierC entries: a warp per row, the next row's
// offsets fetched while the current one is copied.
__global__ void __launch_bounds__(256)
k_lower_arcs_mid(const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
                 const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase,
                 uint32_t *__restrict__ key, uint32_t *__restrict__ val, int64_t m_cap,
                 const u64 *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    const int64_t r_end = static_cast<int64_t>(status[ST_TIER + 3]);
    int64_t r = static_cast<int64_t>(status[ST_LONG]) + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int64_t o_ = 0, ub_ = 0;
    int32_t low_ = 0;
    if (r < r_end) {
        o_ = ldg_i64(coff + r);
        ub_ = ldg_i64(ubase + r);
        low_ = ldg_i32(lowcnt + r);
    }
    for (; r < r_end; r += nw) {
        const int64_t o = o_, lb = o_ - ub_;
        const int32_t low = low_;
        if (r + nw < r_end) {
            o_ = ldg_i64(coff + r + nw);
            ub_ = ldg_i64(ubase + r + nw);
            low_ = ldg_i32(lowcnt + r + nw);
        }
        for (int64_t p0 = 0; p0 < low; p0 += 32 * kListBatch) {
            int32_t c[kListBatch];
#pragma unroll
            for (int u = 0; u < kListBatch; u++) {
                const int64_t p = p0 + 32 * u + lane;
                c[u] = (p < low && lb + p < m_cap) ? ldg_i32(ccol + o + p) : 0;
            }
#pragma unroll
            for (int u = 0; u < kListBatch; u++) {
                const int64_t p = p0 + 32 * u + lane;
                if (p < low && lb + p < m_cap) {
                    key[lb + p] = static_cast<uint32_t>(c[u]);
                    val[lb + p] = static_cast<uint32_t>(o + p);
                }
            }
        }
    }
}

// Rows above kTierC entries: a block per row.
__global__ void __launch_bounds__(256)
k_lower_arcs_long(int64_t n, const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
                  const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase,
                  uint32_t *__restrict__ key, uint32_t *__restrict__ val, int64_t m_cap,
                  const u64 *__restrict__ status) {
    const int64_t r0 = static_cast<int64_t>(status[ST_TIER + 3]);
    for (int64_t r = r0 + blockIdx.x; r < n; r += gridDim.x) {
        const int64_t o = ldg_i64(coff + r), low = ldg_i32(lowcnt + r);
        const int64_t lb = o - ldg_i64(ubase + r);
        for (int64_t p0 = 0; p0 < low; p0 += 256 * kListBatch) {
            int32_t c[kListBatch];
#pragma unroll
            for (int u = 0; u < kListBatch; u++) {
                const int64_t p = p0 + 256 * u + threadIdx.x;
                c[u] = (p < low && lb + p < m_cap) ? ldg_i32(ccol + o + p) : 0;
            }
#pragma unroll
            for (int u = 0; u < kListBatch; u++) {
                const int64_t p = p0 + 256 * u + threadIdx.x;
                if (p < low && lb + p < m_cap) {
                    key[lb + p] = static_cast<uint32_t>(c[u]);
                    val[lb + p] = static_cast<uint32_t>(o + p);
                }
            }
        }
    }
}

// (2a) Digit counts of every tile: counts[digit * tiles + tile].
__global__ void __launch_bounds__(kSortBlock)
k_esort_hist(int64_t count, const uint32_t *__restrict__ key, int shift, uint32_t *counts, int64_t tiles) {
    __shared__ uint32_t s_h[kSortWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortBlock) (&s_h[0][0])[d] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (32 * kSortItems) + lane;
    // all of a thread's keys in flight at once, then the counts
    uint32_t k[kSortItems];
#pragma unroll
    for (int q = 0; q < kSortItems; q++) {
        const int64_t idx = base + 32 * q;
        k[q] = idx < count ? __ldg(key + idx) : 0u;
    }
#pragma unroll
    for (int q = 0; q < kSortItems; q++)
        if (base + 32 * q < count) atomicAdd(&s_h[warp][(k[q] >> shift) & 255u], 1u);
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) c += s_h[w][threadIdx.x];
    counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = c;
}

struct LoadCounts {
    const uint32_t *p;
    __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct StoreCountsExcl {
    uint32_t *p;
    __device__ void operator()(int64_t i, uint32_t exc, uint32_t) const { p[i] = exc; }
};

// (2b) Stable scatter of one tile by the digit at `shift`; offsets[digit *
// tiles + tile] is where the tile's run of that digit starts.  Item order
// within a tile: warp w owns the w-th slice of 32 * kSortItems items and
// walks it in rows of 32 lanes, so (warp, row, lane) is index order.  Only
// the keys and their ranks stay in registers (values are read when placed),
// which keeps four blocks resident per SM.
__global__ void __launch_bounds__(kSortBlock, 4)
k_esort_scatter(int64_t count, const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int shift,
                const uint32_t *__restrict__ offsets, int64_t tiles) {
    __shared__ uint32_t s_key[kSortTile];
    __shared__ uint32_t s_val[kSortTile];
    __shared__ uint32_t s_cnt[kSortWarps][256];  // per-warp counts, then per-warp bases
    __shared__ uint32_t s_start[256];            // first tile-local slot of each digit
    __shared__ uint32_t s_glob[256];             // global start of the tile's run of each digit
    __shared__ uint32_t s_wsum[kSortWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)warp * (32 * kSortItems) + lane;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortBlock) (&s_cnt[0][0])[d] = 0u;
    s_glob[threadIdx.x] = offsets[(int64_t)threadIdx.x * tiles + blockIdx.x];
    uint32_t k[kSortItems];
#pragma unroll
    for (int q = 0; q < kSortItems; q++) {
        const int64_t idx = base + 32 * q;
        k[q] = idx < count ? kin[idx] : 0u;
    }
    __syncthreads();
    // stable rank of every item among its warp's items of the same digit
    // (below 32 * kSortItems, two to a register)
    static_assert(32 * kSortItems <= 65536 && kSortItems % 2 == 0, "ranks packed in 16 bits");
    uint32_t rank2[kSortItems / 2];
#pragma unroll
    for (int q = 0; q < kSortItems; q++) {
        const bool ok = base + 32 * q < count;
        const uint32_t d = ok ? ((k[q] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = ok ? s_cnt[warp][d] : 0u;
        const uint32_t r = before + __popc(peers & lanemask_lt());
        if (q & 1) rank2[q / 2] |= r << 16;
        else rank2[q / 2] = r;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) s_cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t = digit t: per-warp bases within the digit, then the digits'
    // tile-local starts (a block scan of the digit totals)
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) {
            const uint32_t c = s_cnt[w][d];
            s_cnt[w][d] = run;
            run += c;
        }
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) before += (w < warp) ? s_wsum[w] : 0u;
        s_start[d] = before + x - run;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSortItems; q++) {
        const int64_t idx = base + 32 * q;
        if (idx < count) {
            const uint32_t d = (k[q] >> shift) & 255u;
            const uint32_t p = s_start[d] + s_cnt[warp][d] + ((rank2[q / 2] >> (16 * (q & 1))) & 0xFFFFu);
            s_key[p] = k[q];
            s_val[p] = vin[idx];
        }
    }
    __syncthreads();
    const int64_t n_tile = count - tile0 < kSortTile ? count - tile0 : kSortTile;
    for (int p = threadIdx.x; p < n_tile; p += kSortBlock) {
        const uint32_t kk = s_key[p];
        const uint32_t d = (kk >> shift) & 255u;
        const int64_t g = static_cast<int64_t>(s_glob[d]) + (p - static_cast<int64_t>(s_start[d]));
        kout[g] = kk;
        vout[g] = s_val[p];
    }
}

// (3) Edge j from the sorted entry j: u its key, i its arc (in row v, at
// position jv), v the (j - ubase[u])-th upper neighbour of u.  The checks
// that u's upper range holds j and that arc i lies in v's row (where, holding
// u < v, it is a lower arc) hold exactly when the input is symmetric (every
// lower arc has its upper partner and vice versa); otherwise F_ASYM.  A
// thread builds Q edges at j0, j0 + step, ..., their loads issued together
// stage by stage (the chain sorted entry -> row of u -> v -> row of v is
// otherwise a string of dependent round trips per edge), and returns their
// weights (zero past m or for a bad edge).  With the region build of the
// hash set (lists.keys set), every edge's key also goes to the end of its
// home region's list (one atomic per edge).
template <int Q>
__device__ __forceinline__ void edge_group(int64_t j0, int step, int64_t m, int64_t n,
                                           const uint32_t *__restrict__ skey, const uint32_t *__restrict__ sval,
                                           const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
                                           const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase,
                                           EdgeRec *rec, u64 *status, const EsetLists &lists, U64x2 (&w)[Q],
                                           bool &asym) {
    // every offset, label and degree is below 2^31 (nnz < 2^31), so the
    // stages work in 32 bits
    int32_t u[Q], i[Q], ou[Q], du[Q], iu[Q], v[Q], ov[Q], dv[Q];
    bool ok[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int64_t j = j0 + step * q;
        const uint32_t uk = j < m ? __ldg(skey + j) : 0u;
        i[q] = j < m ? static_cast<int32_t>(__ldg(sval + j)) : 0;
        ok[q] = j < m && uk < static_cast<uint64_t>(n);
        u[q] = ok[q] ? static_cast<int32_t>(uk) : 0;
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int64_t o = ldg_i64(coff + u[q]);
        ou[q] = static_cast<int32_t>(o);
        du[q] = static_cast<int32_t>(ldg_i64(coff + u[q] + 1) - o);
        const int64_t rank_in_upper = j0 + step * q - ldg_i64(ubase + u[q]);
        const int64_t pos = ldg_i32(lowcnt + u[q]) + rank_in_upper;
        ok[q] = ok[q] && rank_in_upper >= 0 && pos < du[q];
        iu[q] = ok[q] ? static_cast<int32_t>(pos) : 0;
    }
#pragma unroll
    for (int q = 0; q < Q; q++) v[q] = ok[q] ? ldg_i32(ccol + ou[q] + iu[q]) : 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int64_t o = ldg_i64(coff + v[q]);
        ov[q] = static_cast<int32_t>(o);
        dv[q] = static_cast<int32_t>(ldg_i64(coff + v[q] + 1) - o);
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int64_t j = j0 + step * q;
        w[q] = U64x2{0, 0};
        if (j >= m) continue;
        const int32_t jv = i[q] - ov[q];
        if (!ok[q] || jv < 0 || jv >= dv[q]) {
            asym = true;
            continue;
        }
        int4 *e = reinterpret_cast<int4 *>(rec + j);
        e[0] = make_int4(u[q], v[q], du[q], dv[q]);
        e[1] = make_int4(iu[q], jv, ou[q], ov[q]);
        w[q] = edge_weights(du[q], dv[q], iu[q], jv);
        if (lists.keys) {
            const uint64_t key = edge_key(u[q], v[q]);
            const uint64_t reg = (key_hash(key) & lists.mask) >> lists.shift;
            const uint32_t pos = atomicAdd(lists.cur + reg, 1u);
            if (pos < lists.cap) {
                lists.keys[reg * lists.cap + pos] = key;
            } else {
                const uint32_t o = atomicAdd(lists.ov_count, 1u);
                if (o < lists.ov_cap) lists.ov_keys[o] = key;
                else status[ST_ESET_SPILL] = 1;
            }
        }
    }
}

// The edge table and the exact prefixes of its weights in one pass: each
// block takes a tile of the look-back scan (kRecScanItems edges per thread,
// lane-contiguous rows of 32), builds its edges kRecItems rows at a time,
// parks their weights in shared memory and scans them (so the records are
// never read back for the prefix sums).
constexpr int kRecItems = 4;
constexpr int kRecScanItems = 8;
static_assert(kRecScanItems % kRecItems == 0, "whole groups per tile");
static_assert(kScanBlock * kRecScanItems >= kScanTile, "scan flags are reset per kScanTile items");

// (Capped at 64 registers, four blocks per SM: while one block waits at the
// tile's barriers or on its look-back, the others build records; the
// uncapped 80-register build, three blocks per SM, took 1 ms more per load
// on the 3M-vertex graph.)
__global__ void __launch_bounds__(kScanBlock, 4)
k_edge_records_scan(int64_t m, int64_t n, const uint32_t *__restrict__ skey, const uint32_t *__restrict__ sval,
                    const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
                    const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase, EdgeRec *rec,
                    u64 *status, EsetLists lists, ScanState<U64x2> st, uint64_t *ptau, uint64_t *plam) {
    __shared__ U64x2 s_w[kRecScanItems * kScanBlock];
    const int64_t tile = scan_ticket(st);
    const int64_t wbase = scan_wbase<kScanBlock, kRecScanItems>(tile);
    bool asym = false;
#pragma unroll
    for (int g0 = 0; g0 < kRecScanItems; g0 += kRecItems) {
        U64x2 w[kRecItems];
        edge_group<kRecItems>(wbase + 32 * g0, 32, m, n, skey, sval, coff, ccol, lowcnt, ubase, rec, status, lists,
                              w, asym);
#pragma unroll
        for (int q = 0; q < kRecItems; q++) s_w[(g0 + q) * kScanBlock + threadIdx.x] = w[q];
    }
    if (asym) raise_flag(status, F_ASYM);
    U64x2 v[kRecScanItems];
#pragma unroll
    for (int i = 0; i < kRecScanItems; i++) v[i] = s_w[i * kScanBlock + threadIdx.x];
    scan_tile<U64x2, kScanBlock, kRecScanItems>(tile, wbase, v, m, st, U64x2{0, 0}, OpSum(),
                                                StorePrefix{ptau, plam, status, m});
}

int build_edge_table(ps_graph *g, cudaStream_t s, const EsetLists *lists) {
    const Layout &L = g->L;
    const int64_t n = L.n, nnz = L.nnz, m = L.m_cap;
    if (nnz <= 0 || m <= 0) return PS_OK;
    const int sms = g->sm_count;
    char *ws = g->ws;
    // (key, value) buffers of m entries each: the lower arcs are listed into
    // the P_tau region, the passes ping-pong between it and the P_lambda
    // region, and the last pass writes to the G_tau region (at least 8 bytes
    // per edge), which nothing reads before the guide tables are built -- so
    // the prefixes can be written while the sorted list is still being read
    uint32_t *ka = reinterpret_cast<uint32_t *>(ws + L.ptau), *va = ka + m;
    uint32_t *kb = reinterpret_cast<uint32_t *>(ws + L.plam), *vb = kb + m;
    uint32_t *kg = reinterpret_cast<uint32_t *>(ws + L.gtau), *vg = kg + m;
    int bits = 0;
    while (bits < 31 && (static_cast<uint64_t>(n > 0 ? n - 1 : 0) >> bits) != 0) bits++;
    const int passes = bits > 0 ? (bits + 7) / 8 : 1;
    if (n > 0) {
        int64_t blocks = (n + 255) / 256;  // a warp per 32 rows
        if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
        k_lower_arcs<<<(unsigned)blocks, 256, 0, s>>>(n, g->off, g->col, g->ubase, ka, va, m, g->status);
        PS_LAUNCH_CHECK();
        if (g->d_max > kLongRow) {
            k_lower_arcs_mid<<<(unsigned)(sms * 6), 256, 0, s>>>(g->off, g->col, g->lowcnt, g->ubase, ka, va, m,
                                                                  g->status);
            PS_LAUNCH_CHECK();
        }
        if (g->d_max > kTierC) {
            k_lower_arcs_long<<<(unsigned)(sms * 4), 256, 0, s>>>(n, g->off, g->col, g->lowcnt, g->ubase, ka, va, m,
                                                                   g->status);
            PS_LAUNCH_CHECK();
        }
    }
    const int64_t tiles = edge_sort_tiles(m);
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws + L.ecounts);
    for (int pass = 0; pass < passes; pass++) {
        const int shift = 8 * pass;
        const bool last = pass == passes - 1;
        uint32_t *ko = last ? kg : kb, *vo = last ? vg : vb;
        k_esort_hist<<<(unsigned)tiles, kSortBlock, 0, s>>>(m, ka, shift, counts, tiles);
        PS_LAUNCH_CHECK();
        int rc = run_scan<uint32_t>(g, 0, 256 * tiles, 0u, OpSum(), LoadCounts{counts}, StoreCountsExcl{counts}, s);
        if (rc) return rc;
        k_esort_scatter<<<(unsigned)tiles, kSortBlock, 0, s>>>(m, ka, va, ko, vo, shift, counts, tiles);
        PS_LAUNCH_CHECK();
        uint32_t *t = ka;
        ka = ko;
        kb = t;
        t = va;
        va = vo;
        vb = t;
    }
    // ka/va: the sorted list, in the G_tau region
    int rc = reset_scan(g, 3, m, s);
    if (rc) return rc;
    const int64_t stiles = (m + kScanBlock * kRecScanItems - 1) / (kScanBlock * kRecScanItems);
    EsetLists none{};
    k_edge_records_scan<<<(unsigned)stiles, kScanBlock, 0, s>>>(
        m, n, ka, va, g->off, g->col, g->lowcnt, g->ubase, g->rec, g->status, lists ? *lists : none,
        scan_state<U64x2>(g, 3), g->ptau, g->plam);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

}  // namespace ps
