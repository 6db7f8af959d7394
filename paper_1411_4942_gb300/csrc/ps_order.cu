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

// kOrderBuckets equal-width ranges of r; a chunk of ids is split into at most
// kOrderMaxBlocks contiguous runs, one per block of the counting sort, which
// keeps its bucket counters in shared memory.
constexpr int kOrderBuckets = 1 << 14;
constexpr int kOrderMaxBlocks = 512;
constexpr int kOrderThreads = 512;
constexpr int kOrderSmem = kOrderBuckets * static_cast<int>(sizeof(uint32_t));
constexpr size_t kOrderHist = static_cast<size_t>(kOrderMaxBlocks) * kOrderBuckets * sizeof(uint32_t);
constexpr size_t kOrderHeader = kOrderHist + kOrderBuckets * sizeof(uint32_t);  // run counts, bases
// after the header: the chunk's ids (uint32), then their buckets (uint16)
constexpr int kOrderScanThreads = 1024;
constexpr int kOrderPerThread = kOrderBuckets / kOrderScanThreads;
// By default (tuning draw_order 0) chunks below kOrderMinChunk samples, and
// graphs below kOrderMinEdges edges (whose records and rows mostly stay in
// L2 anyway), take the plain sampler: there the sort costs more than it
// saves.  The counts are the same either way.
constexpr uint64_t kOrderMinChunk = 1ull << 18;
constexpr int64_t kOrderMinEdges = 1ll << 20;

// The edge draw r of sample id, exactly as the samplers take it.
template <int SAMPLER>
__device__ __forceinline__ uint64_t draw_r_of(uint64_t total, uint64_t seed, uint64_t id) {
    const uint4 w = sample_block(seed, id, 0, SAMPLER);
    uint64_t r;
    if (!lemire64((static_cast<uint64_t>(w.y) << 32) | w.x, total, r)) r = draw_r_retry(seed, id, SAMPLER, total);
    return r;
}

// Bucket of every id of block b's run [b * per, (b + 1) * per) into bkt, and
// the run's bucket counts into row b of hist.
template <int SAMPLER>
__global__ void __launch_bounds__(kOrderThreads)
k_order_count(uint64_t total, uint64_t kk, uint64_t seed, uint64_t first_id, int shift, uint64_t per,
              uint32_t *hist, uint16_t *bkt) {
    extern __shared__ uint32_t s_h[];
    for (int b = threadIdx.x; b < kOrderBuckets; b += kOrderThreads) s_h[b] = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = lo + per < kk ? lo + per : kk;
    for (uint64_t s = lo + threadIdx.x; s < hi; s += kOrderThreads) {
        const uint32_t c = static_cast<uint32_t>(draw_r_of<SAMPLER>(total, seed, first_id + s) >> shift);
        bkt[s] = static_cast<uint16_t>(c);
        atomicAdd(s_h + c, 1u);
    }
    __syncthreads();
    uint32_t *row = hist + (size_t)blockIdx.x * kOrderBuckets;
    for (int b = threadIdx.x; b < kOrderBuckets; b += kOrderThreads) row[b] = s_h[b];
}

// For every bucket (one thread each): the runs' counts become exclusive
// offsets within the bucket, and base[bucket] its total.  Eight rows are
// loaded before any is rewritten, so their loads overlap.
__global__ void __launch_bounds__(256)
k_order_runs(int runs, uint32_t *hist, uint32_t *base) {
    const int b = blockIdx.x * 256 + threadIdx.x;
    if (b >= kOrderBuckets) return;
    uint32_t run = 0;
    uint32_t *p = hist + b;
    int r = 0;
    for (; r + 8 <= runs; r += 8) {
        uint32_t c[8];
#pragma unroll
        for (int i = 0; i < 8; i++) c[i] = p[(size_t)(r + i) * kOrderBuckets];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            p[(size_t)(r + i) * kOrderBuckets] = run;
            run += c[i];
        }
    }
    for (; r < runs; r++) {
        const uint32_t c = p[(size_t)r * kOrderBuckets];
        p[(size_t)r * kOrderBuckets] = run;
        run += c;
    }
    base[b] = run;
}

// Exclusive prefix of the bucket totals, in place (one block).
__global__ void __launch_bounds__(kOrderScanThreads)
k_order_bases(uint32_t *base) {
    extern __shared__ uint32_t s_v[];  // kOrderBuckets
    __shared__ uint32_t s_warp[kOrderScanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int i = t; i < kOrderBuckets; i += kOrderScanThreads) s_v[i] = base[i];
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kOrderPerThread; i++) sum += s_v[t * kOrderPerThread + i];
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - sum + (warp ? s_warp[warp - 1] : 0u);
#pragma unroll
    for (int i = 0; i < kOrderPerThread; i++) {
        const uint32_t c = s_v[t * kOrderPerThread + i];
        s_v[t * kOrderPerThread + i] = run;
        run += c;
    }
    __syncthreads();
    for (int i = t; i < kOrderBuckets; i += kOrderScanThreads) base[i] = s_v[i];
}

// Block b places its run of ids: cursors start at base[bucket] + the run's
// offset within the bucket and advance with shared-memory atomics.
__global__ void __launch_bounds__(kOrderThreads)
k_order_scatter(uint64_t kk, uint64_t per, const uint32_t *__restrict__ hist, const uint32_t *__restrict__ base,
                const uint16_t *__restrict__ bkt, uint32_t *ids) {
    extern __shared__ uint32_t s_c[];
    const uint32_t *row = hist + (size_t)blockIdx.x * kOrderBuckets;
    for (int b = threadIdx.x; b < kOrderBuckets; b += kOrderThreads) s_c[b] = base[b] + row[b];
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = lo + per < kk ? lo + per : kk;
    for (uint64_t s = lo + threadIdx.x; s < hi; s += kOrderThreads) {
        const uint32_t pos = atomicAdd(s_c + bkt[s], 1u);
        ids[pos] = static_cast<uint32_t>(s);
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
    int shift = 0;
    while (shift < 63 && ((total - 1) >> shift) >= static_cast<uint64_t>(kOrderBuckets)) shift++;
    uint32_t *hist_runs = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *base = reinterpret_cast<uint32_t *>(scratch + kOrderHist);
    uint32_t *ids = reinterpret_cast<uint32_t *>(scratch + kOrderHeader);
    uint16_t *bkt = reinterpret_cast<uint16_t *>(scratch + kOrderHeader + chunk * sizeof(uint32_t));
    int per_sm = g->tune.blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_ordered<SAMPLER, BLOCK, ADJ>,
                                                                  BLOCK, 0));
        per_sm = occ > 0 ? occ : 1;
    }
    const uint64_t full = (uint64_t)g->sm_count * per_sm;
    PS_CUDA_TRY(cudaFuncSetAttribute(k_order_count<SAMPLER>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOrderSmem));
    PS_CUDA_TRY(cudaFuncSetAttribute(k_order_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kOrderSmem));
    PS_CUDA_TRY(cudaFuncSetAttribute(k_order_bases, cudaFuncAttributeMaxDynamicSharedMemorySize, kOrderSmem));
    while (k > 0) {
        const uint64_t kk = k < chunk ? k : chunk;
        if (kk < kOrderMinChunk && g->tune.draw_order == 0) {
            const int rc = launch_sampler(g, SAMPLER, kk, seed, first_id, hist, s);
            if (rc) return rc;
        } else {
            uint64_t runs = (uint64_t)g->sm_count * 2;
            if (runs > (uint64_t)kOrderMaxBlocks) runs = kOrderMaxBlocks;
            const uint64_t per = (kk + runs - 1) / runs;
            runs = (kk + per - 1) / per;
            uint64_t blocks = (kk + BLOCK - 1) / BLOCK;
            if (blocks > full) blocks = full;
            k_order_count<SAMPLER><<<(unsigned)runs, kOrderThreads, kOrderSmem, s>>>(total, kk, seed, first_id, shift,
                                                                                  per, hist_runs, bkt);
            PS_LAUNCH_CHECK();
            k_order_runs<<<kOrderBuckets / 256, 256, 0, s>>>(static_cast<int>(runs), hist_runs, base);
            PS_LAUNCH_CHECK();
            k_order_bases<<<1, kOrderScanThreads, kOrderSmem, s>>>(base);
            PS_LAUNCH_CHECK();
            k_order_scatter<<<(unsigned)runs, kOrderThreads, kOrderSmem, s>>>(kk, per, hist_runs, base, bkt, ids);
            PS_LAUNCH_CHECK();
            k_sample_ordered<SAMPLER, BLOCK, ADJ><<<(unsigned)blocks, BLOCK, 0, s>>>(g->dev, kk, seed, first_id,
                                                                                    ids, hist);
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

// Bytes per sample of a chunk: its id and its bucket.
constexpr size_t kOrderPerSample = sizeof(uint32_t) + sizeof(uint16_t);

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
