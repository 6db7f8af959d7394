// ps_order.cu -- ps_sample_3paths_ordered / ps_sample_centered_ordered: the
// samplers of Alg. 1 and Alg. 3 with the samples taken in the order of their
// edge draws.
//
// Every sample is independent (Claim 3.1: each draw is a fresh r), and the
// histograms are sums, so the order in which ids are classified changes no
// count.  In id order, consecutive samples draw unrelated edges: the guide
// entry, the prefix probe, the edge record and the row N(u) of every sample
// are separate random reads of HBM.  Here the ids of a chunk are first
// counting-sorted by r >> shift into kOrderBuckets equal-width ranges of
// [0, W) (or [0, Lambda)); the sampling grid then walks the sorted ids, so the
// samples in flight at any time draw from a narrow band of consecutive edges
// and those reads mostly hit L1 and L2.  Only the second endpoint's row and
// the adjacency tests stay random.
#include "ps_internal.h"
#include "ps_sample.cuh"

namespace ps {

// kOrderBuckets equal-width ranges of r; a chunk of ids is split into at
// most kOrderMaxRuns contiguous runs, one per block of the counting sort.
// On R-MAT 20 with 2^24 samples, finer orders made the 3-path sampling
// kernel faster (1.08 ms at 256 buckets, 0.96 ms at 65536 through a second
// pass, 0.94 ms with global atomics) but cost more to sort than they saved.
constexpr int kOrderBuckets = 256;
constexpr int kOrderMaxRuns = 1024;
constexpr int kOrderThreads = 512;
constexpr int kOrderWarps = kOrderThreads / 32;
constexpr int kOrderItems = 8;                            // ids per scatter thread and tile
constexpr int kOrderTile = kOrderItems * kOrderThreads;   // ids a scatter block sorts in shared memory at once
// hist[b * kOrderMaxRuns + run]: run counts, then offsets; then the bucket totals
constexpr size_t kOrderHist = static_cast<size_t>(kOrderMaxRuns) * kOrderBuckets * sizeof(uint32_t);
constexpr size_t kOrderHeader = kOrderHist + kOrderBuckets * sizeof(uint32_t);
// after the header, per sample of a chunk: the sorted order (uint32 id
// offsets from the chunk's first id), then each id's bucket (uint8)
// By default (tuning draw_order 0) chunks below kOrderMinChunk samples, and
// graphs below kOrderMinEdges edges (whose records and rows mostly stay in
// L2 anyway), take the plain sampler: there the sort costs more than it
// saves.  The counts are the same either way.
constexpr uint64_t kOrderMinChunk = 1ull << 18;
constexpr int64_t kOrderMinEdges = 1ll << 20;
// From this many edges the default sorts by 16 bits of r in two passes: a
// 256th of r then spans too many edges for their records and rows to be
// read again before L2 drops them.  Measured (one box, both samplers):
// 3M-vertex graph, 116.6M edges, 14.75 / 5.47 -> 14.22 / 5.16 ms with the
// sorts; R-MAT 20, 15.7M edges, 1.22 / 0.87 -> 1.23 / 0.96 ms.
constexpr int64_t kOrderTwoPassEdges = 1ll << 25;

// The edge draw r of sample id, exactly as the samplers take it.
template <int SAMPLER>
__device__ __forceinline__ uint64_t draw_r_of(uint64_t total, uint64_t seed, uint64_t id) {
    const uint4 w = sample_block(seed, id, 0, SAMPLER);
    uint64_t r;
    if (!lemire64((static_cast<uint64_t>(w.y) << 32) | w.x, total, r)) r = draw_r_retry(seed, id, SAMPLER, total);
    return r;
}

// Bucket of every id of block b's run [b * per, (b + 1) * per) into bkt, and
// the run's bucket counts into hist[bucket * kOrderMaxRuns + b] (per-warp
// counters first).  Two draws per iteration, so two Philox chains overlap.
// With `high` set (the two-pass order), r >> shift is a 16-bit range: its low
// byte is the bucket of this pass and its high byte is stored in high[] for
// the second pass.
template <int SAMPLER>
__global__ void __launch_bounds__(kOrderThreads)
k_order_count(uint64_t total, uint64_t kk, uint64_t seed, uint64_t first_id, int shift, uint64_t per,
              uint32_t *hist, uint8_t *bkt, uint8_t *high) {
    __shared__ uint32_t s_h[kOrderWarps][kOrderBuckets];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kOrderWarps * kOrderBuckets; i += kOrderThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = lo + per < kk ? lo + per : kk;
    for (uint64_t s = lo + threadIdx.x; s < hi; s += 2 * kOrderThreads) {
        const uint64_t s2 = s + kOrderThreads;
        uint32_t c = static_cast<uint32_t>(draw_r_of<SAMPLER>(total, seed, first_id + s) >> shift);
        uint32_t c2 = static_cast<uint32_t>(draw_r_of<SAMPLER>(total, seed, first_id + s2) >> shift);
        if (high) {
            high[s] = static_cast<uint8_t>(c >> 8);
            if (s2 < hi) high[s2] = static_cast<uint8_t>(c2 >> 8);
            c &= 255u;
            c2 &= 255u;
        }
        bkt[s] = static_cast<uint8_t>(c);
        atomicAdd(&s_h[warp][c], 1u);
        if (s2 < hi) {
            bkt[s2] = static_cast<uint8_t>(c2);
            atomicAdd(&s_h[warp][c2], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += kOrderThreads) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kOrderWarps; w++) c += s_h[w][b];
        hist[(size_t)b * kOrderMaxRuns + blockIdx.x] = c;
    }
}

// The second pass's counts: the bucket of every position is the stored high
// byte; per-run counts as in k_order_count.
__global__ void __launch_bounds__(kOrderThreads)
k_order_count_bytes(uint64_t kk, uint64_t per, const uint8_t *__restrict__ bkt, uint32_t *hist) {
    __shared__ uint32_t s_h[kOrderWarps][kOrderBuckets];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kOrderWarps * kOrderBuckets; i += kOrderThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = lo + per < kk ? lo + per : kk;
    for (uint64_t s = lo + threadIdx.x; s < hi; s += kOrderThreads) atomicAdd(&s_h[warp][bkt[s]], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += kOrderThreads) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kOrderWarps; w++) c += s_h[w][b];
        hist[(size_t)b * kOrderMaxRuns + blockIdx.x] = c;
    }
}

// Exclusive prefix of v[0..kOrderBuckets) across the first kOrderBuckets
// threads of the block (every thread must call it); returns thread t's
// exclusive prefix and leaves the total in *total.
__device__ __forceinline__ uint32_t bucket_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t x = t < kOrderBuckets ? v : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31 && warp < kOrderBuckets / 32) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kOrderBuckets / 32; w++) {
        const uint32_t sw = s_warp[w];
        before += w < warp ? sw : 0u;
        all += sw;
    }
    __syncthreads();
    *total = all;
    return before + x - (t < kOrderBuckets ? v : 0u);
}

// Block b (kOrderBuckets threads, 4 runs each): bucket b's run counts become
// exclusive offsets within the bucket, and totals[b] its size.
__global__ void __launch_bounds__(kOrderBuckets)
k_order_offsets(int runs, uint32_t *hist, uint32_t *totals) {
    static_assert(4 * kOrderBuckets == kOrderMaxRuns, "4 runs per thread");
    __shared__ uint32_t s_warp[kOrderBuckets / 32];
    uint32_t *p = hist + (size_t)blockIdx.x * kOrderMaxRuns + 4 * threadIdx.x;
    uint32_t c[4], sum = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        c[i] = 4 * threadIdx.x + i < runs ? p[i] : 0u;
        sum += c[i];
    }
    uint32_t all;
    uint32_t run = bucket_scan(sum, s_warp, &all);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (4 * threadIdx.x + i < runs) p[i] = run;
        run += c[i];
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = all;
}

// Block b places its run of ids, kOrderTile at a time: each tile is first
// counting-sorted by bucket in shared memory, then each bucket's ids are
// written as one contiguous piece at the run's cursor for that bucket
// (base[bucket] + the run's offset within it, advanced after every tile), so
// the stores coalesce.  The buckets of the next tile are loaded while the
// current one is placed.  The value placed for input position q is q, or
// vals[q] when vals is given (the second pass of the two-pass order, whose
// input is the first pass's output); a byte carry[q] travels with it into
// carry_out when carry is given.
__global__ void __launch_bounds__(kOrderThreads)
k_order_scatter(uint64_t kk, uint64_t per, const uint32_t *__restrict__ hist, const uint32_t *__restrict__ totals,
                const uint8_t *__restrict__ bkt, const uint32_t *__restrict__ vals, const uint8_t *__restrict__ carry,
                uint32_t *__restrict__ ids, uint8_t *__restrict__ carry_out) {
    __shared__ uint32_t s_cur[kOrderBuckets], s_cnt[kOrderBuckets], s_off[kOrderBuckets];
    __shared__ uint32_t s_warp[kOrderBuckets / 32];
    __shared__ uint32_t s_id[kOrderTile];
    __shared__ uint8_t s_b[kOrderTile];
    __shared__ uint8_t s_c[kOrderTile];
    const int t = threadIdx.x;
    {
        // the buckets' first positions: exclusive prefix of their totals
        uint32_t all;
        const uint32_t base = bucket_scan(t < kOrderBuckets ? totals[t] : 0u, s_warp, &all);
        if (t < kOrderBuckets) s_cur[t] = base + hist[(size_t)t * kOrderMaxRuns + blockIdx.x];
    }
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = lo + per < kk ? lo + per : kk;
    uint32_t nxt[kOrderItems];
#pragma unroll
    for (int i = 0; i < kOrderItems; i++) {
        const uint64_t q = lo + (uint64_t)i * kOrderThreads + t;
        nxt[i] = q < hi ? static_cast<uint32_t>(bkt[q]) : static_cast<uint32_t>(kOrderBuckets);
    }
    for (uint64_t t0 = lo; t0 < hi; t0 += kOrderTile) {
        if (t < kOrderBuckets) s_cnt[t] = 0;
        uint32_t myb[kOrderItems], rank[kOrderItems];
#pragma unroll
        for (int i = 0; i < kOrderItems; i++) {
            myb[i] = nxt[i];
            const uint64_t q = t0 + kOrderTile + (uint64_t)i * kOrderThreads + t;
            nxt[i] = q < hi ? static_cast<uint32_t>(bkt[q]) : static_cast<uint32_t>(kOrderBuckets);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kOrderItems; i++)
            if (myb[i] < kOrderBuckets) rank[i] = atomicAdd(s_cnt + myb[i], 1u);
        __syncthreads();
        uint32_t all;
        const uint32_t off = bucket_scan(t < kOrderBuckets ? s_cnt[t] : 0u, s_warp, &all);
        if (t < kOrderBuckets) s_off[t] = off;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kOrderItems; i++) {
            if (myb[i] < kOrderBuckets) {
                const uint32_t p = s_off[myb[i]] + rank[i];
                const uint64_t q = t0 + (uint64_t)i * kOrderThreads + t;
                s_id[p] = vals ? vals[q] : static_cast<uint32_t>(q);
                s_b[p] = static_cast<uint8_t>(myb[i]);
                if (carry) s_c[p] = carry[q];
            }
        }
        __syncthreads();
        for (uint32_t p = t; p < all; p += kOrderThreads) {
            const uint32_t b = s_b[p];
            const uint32_t dst = s_cur[b] + (p - s_off[b]);
            ids[dst] = s_id[p];
            if (carry) carry_out[dst] = s_c[p];
        }
        __syncthreads();
        if (t < kOrderBuckets) s_cur[t] += s_cnt[t];
    }
}

template <int SAMPLER, int BLOCK, int ADJ>
__global__ void __launch_bounds__(BLOCK, sample_min_blocks<BLOCK>())
k_sample_ordered(GraphDev g, uint64_t kk, uint64_t seed, uint64_t first_id, const uint32_t *__restrict__ ids,
                 uint64_t *hist) {
    Counts6 cnt;
    cnt.zero();
    const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
    for (uint64_t p = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; p < kk; p += stride) {
        const uint64_t id = first_id + __ldg(ids + p);
        cnt.add(SAMPLER == 0 ? sample_3path<ADJ>(g, seed, id) : sample_centred<ADJ>(g, seed, id));
    }
    flush_counts<BLOCK>(cnt, SAMPLER == 0 ? 6 : 4, hist);
}

template <int SAMPLER, int BLOCK, int ADJ>
static int ordered_t(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *hist,
                     char *scratch, uint64_t chunk, cudaStream_t s) {
    const uint64_t total = SAMPLER == 0 ? g->stats.W : g->stats.Lambda;
    // the two-pass order sorts by 16 bits of r (65536 ranges), the one-pass by 8
    const bool two_pass = g->tune.draw_order == 2 || (g->tune.draw_order == 0 && g->m >= kOrderTwoPassEdges);
    const uint64_t ranges = two_pass ? 65536u : static_cast<uint64_t>(kOrderBuckets);
    int shift = 0;
    while (shift < 63 && ((total - 1) >> shift) >= ranges) shift++;
    uint32_t *hist_runs = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *totals = reinterpret_cast<uint32_t *>(scratch + kOrderHist);
    // per sample of a chunk: the sorted ids, the first pass's ids, the
    // bucket byte, the high byte and the high byte in first-pass order
    uint32_t *ids = reinterpret_cast<uint32_t *>(scratch + kOrderHeader);
    uint32_t *ids1 = ids + chunk;
    uint8_t *bkt = reinterpret_cast<uint8_t *>(ids1 + chunk);
    uint8_t *high = bkt + chunk;
    uint8_t *high1 = high + chunk;
    int per_sm = g->tune.blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_ordered<SAMPLER, BLOCK, ADJ>,
                                                                  BLOCK, 0));
        per_sm = occ > 0 ? occ : 1;
    }
    const uint64_t full = (uint64_t)g->sm_count * per_sm;
    while (k > 0) {
        const uint64_t kk = k < chunk ? k : chunk;
        if (kk < kOrderMinChunk && g->tune.draw_order == 0) {
            const int rc = launch_sampler(g, SAMPLER, kk, seed, first_id, hist, s);
            if (rc) return rc;
        } else {
            uint64_t runs = (uint64_t)g->sm_count * 2;  // one wave of the count kernel
            if (runs > (uint64_t)kOrderMaxRuns) runs = kOrderMaxRuns;
            const uint64_t per = (kk + runs - 1) / runs;
            runs = (kk + per - 1) / per;
            uint64_t blocks = (kk + BLOCK - 1) / BLOCK;
            if (blocks > full) blocks = full;
            k_order_count<SAMPLER><<<(unsigned)runs, kOrderThreads, 0, s>>>(total, kk, seed, first_id, shift, per,
                                                                         hist_runs, bkt, two_pass ? high : nullptr);
            PS_LAUNCH_CHECK();
            k_order_offsets<<<kOrderBuckets, kOrderBuckets, 0, s>>>(static_cast<int>(runs), hist_runs, totals);
            PS_LAUNCH_CHECK();
            if (!two_pass) {
                k_order_scatter<<<(unsigned)runs, kOrderThreads, 0, s>>>(kk, per, hist_runs, totals, bkt, nullptr,
                                                                         nullptr, ids, nullptr);
                PS_LAUNCH_CHECK();
            } else {
                // least significant byte first, then the high byte: every id
                // ends in its 16-bit range of r (in range order; within a range
                // the order of a tile's ids is free)
                k_order_scatter<<<(unsigned)runs, kOrderThreads, 0, s>>>(kk, per, hist_runs, totals, bkt, nullptr,
                                                                         high, ids1, high1);
                PS_LAUNCH_CHECK();
                k_order_count_bytes<<<(unsigned)runs, kOrderThreads, 0, s>>>(kk, per, high1, hist_runs);
                PS_LAUNCH_CHECK();
                k_order_offsets<<<kOrderBuckets, kOrderBuckets, 0, s>>>(static_cast<int>(runs), hist_runs, totals);
                PS_LAUNCH_CHECK();
                k_order_scatter<<<(unsigned)runs, kOrderThreads, 0, s>>>(kk, per, hist_runs, totals, high1, ids1,
                                                                         nullptr, ids, nullptr);
                PS_LAUNCH_CHECK();
            }
            k_sample_ordered<SAMPLER, BLOCK, ADJ><<<(unsigned)blocks, BLOCK, 0, s>>>(g->dev, kk, seed, first_id, ids,
                                                                                    hist);
            PS_LAUNCH_CHECK();
        }
        k -= kk;
        first_id += kk;
    }
    return PS_OK;
}

template <int SAMPLER, int BLOCK>
static int ordered_b(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *hist,
                     char *scratch, uint64_t chunk, cudaStream_t s) {
    switch (g->tune.adj_mode) {
        case kAdjVtab: return ordered_t<SAMPLER, BLOCK, kAdjVtab>(g, k, seed, first_id, hist, scratch, chunk, s);
        case kAdjHash: return ordered_t<SAMPLER, BLOCK, kAdjHash>(g, k, seed, first_id, hist, scratch, chunk, s);
        default: return ordered_t<SAMPLER, BLOCK, kAdjSearch>(g, k, seed, first_id, hist, scratch, chunk, s);
    }
}

template <int SAMPLER>
static int ordered_s(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *hist,
                     char *scratch, uint64_t chunk, cudaStream_t s) {
    switch (g->tune.block_size) {
        case 128: return ordered_b<SAMPLER, 128>(g, k, seed, first_id, hist, scratch, chunk, s);
        case 256: return ordered_b<SAMPLER, 256>(g, k, seed, first_id, hist, scratch, chunk, s);
        case 512: return ordered_b<SAMPLER, 512>(g, k, seed, first_id, hist, scratch, chunk, s);
        case 1024: return ordered_b<SAMPLER, 1024>(g, k, seed, first_id, hist, scratch, chunk, s);
        default: return PS_ERR_ARG;
    }
}

// Bytes per sample of a chunk: its sorted id, its id after the first of two
// passes, its bucket byte and its high byte in both orders.
constexpr size_t kOrderPerSample = 2 * sizeof(uint32_t) + 3 * sizeof(uint8_t);

size_t ordered_scratch_bytes(uint64_t k_chunk) {
    if (k_chunk == 0 || k_chunk > kOrderMaxChunk) return 0;
    return kOrderHeader + static_cast<size_t>(k_chunk) * kOrderPerSample;
}

int launch_ordered(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *d_hist,
                   void *d_scratch, size_t scratch_bytes, cudaStream_t s) {
    if (scratch_bytes < ordered_scratch_bytes(1)) return PS_ERR_WORKSPACE;
    uint64_t chunk = (scratch_bytes - kOrderHeader) / kOrderPerSample;
    if (chunk > kOrderMaxChunk) chunk = kOrderMaxChunk;
    if (g->tune.draw_order < 0 || (g->tune.draw_order == 0 && g->m < kOrderMinEdges))
        return launch_sampler(g, sampler, k, seed, first_id, d_hist, s);
    char *scratch = static_cast<char *>(d_scratch);
    return sampler == 0 ? ordered_s<0>(g, k, seed, first_id, d_hist, scratch, chunk, s)
                        : ordered_s<1>(g, k, seed, first_id, d_hist, scratch, chunk, s);
}

}  // namespace ps
