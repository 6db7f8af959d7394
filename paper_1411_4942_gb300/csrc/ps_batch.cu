// ps_batch.cu -- ps_batch_sample: one persistent launch over a queue of work
// items drawn from many loaded graphs.  Each block takes an item (a range of
// sample ids of one graph and one sampler), runs it with the same per-sample
// code as the plain launches and adds its class counts to the item's slot.
//
// When every graph of a descriptor table uses the same adjacency variant
// (recorded on the host by ps_batch_prepare), the launch uses a kernel
// compiled for that variant alone, which needs fewer registers and so keeps
// more warps resident; mixed tables use the kernel that handles all of them.
#include <mutex>
#include <unordered_map>

#include "ps_internal.h"
#include "ps_sample.cuh"

namespace ps {

namespace {
std::mutex g_table_mutex;
std::unordered_map<const void *, int> g_table_adj;  // d_table -> common variant (0: mixed)
}  // namespace

void note_table_adjacency(const void *d_table, int adj) {
    std::lock_guard<std::mutex> lock(g_table_mutex);
    g_table_adj[d_table] = adj;
}

static int table_adjacency(const void *d_table) {
    std::lock_guard<std::mutex> lock(g_table_mutex);
    auto it = g_table_adj.find(d_table);
    return it == g_table_adj.end() ? 0 : it->second;
}

template <int ADJ>
__device__ __forceinline__ int batch_sample(const GraphDev &g, int sampler, uint64_t seed, uint64_t id) {
    return sampler == 0 ? sample_3path<ADJ, false>(g, seed, id) : sample_centred<ADJ, false>(g, seed, id);
}

// Two samples of one thread with the hash-set adjacency, their steps
// interleaved: both draws (edge, record, neighbours) as straight-line code,
// then both samples' tests, so the two dependent chains overlap.  The same
// counts as two calls of batch_sample.
__device__ __forceinline__ void batch_sample2_hash(const GraphDev &g, int sampler, uint64_t seed, uint64_t id0,
                                                   uint64_t id1, int &c0, int &c1) {
    EdgeRec e0, e1;
    int32_t a0, b0, a1, b1;
    if (sampler == 0) {
        path3_draw(g, seed, id0, e0, a0, b0);
        path3_draw(g, seed, id1, e1, a1, b1);
        bool x0, y0, z0, x1, y1, z1;
        pair_test3<false>(g, a0, e0.v, e0.u, b0, a0, b0, x0, y0, z0);
        pair_test3<false>(g, a1, e1.v, e1.u, b1, a1, b1, x1, y1, z1);
        c0 = a0 == b0 ? 0 : class3(x0, y0, z0);
        c1 = a1 == b1 ? 0 : class3(x1, y1, z1);
    } else {
        centred_draw(g, seed, id0, e0, a0, b0);
        centred_draw(g, seed, id1, e1, a1, b1);
        bool k0, k1;
        eset_contains2(g.eset, g.eset_mask, a0, b0, a1, b1, k0, k1);
        // the chords only for centred paths (the pair test also answers u' == v')
        k0 = k0 && a0 != b0;
        k1 = k1 && a1 != b1;
        bool p0 = false, q0 = false, p1 = false, q1 = false;
        if (k0) pair_test2<false>(g, e0.v, a0, e0.u, b0, p0, q0);
        if (k1) pair_test2<false>(g, e1.v, a1, e1.u, b1, p1, q1);
        c0 = k0 ? 1 + (int)p0 + (int)q0 : 0;
        c1 = k1 ? 1 + (int)p1 + (int)q1 : 0;
    }
}

// ADJ = 0: any variant, chosen per item; otherwise the table's only variant.
// counter[0] hands out items; counter[1] counts items skipped because their
// graph does not use the variant this kernel was compiled for.  Registers
// are capped for 1024 resident threads per SM with one sample per thread in
// flight (SPT = 1), 512 with two (SPT = 2, hash-set graphs; other variants
// take their two samples one after the other).
template <int BLOCK, int ADJ, int SPT>
__global__ void __launch_bounds__(BLOCK, (SPT == 1 ? 1024 : 512) / BLOCK)
k_batch(const GraphDev *__restrict__ table, int32_t n_graphs, const ps_work *__restrict__ items,
        int64_t n_items, uint64_t *hist, uint32_t *counter) {
    __shared__ int64_t s_item;
    __shared__ GraphDev s_g;
    __shared__ ps_work s_w;
    while (true) {
        if (threadIdx.x == 0) {
            const int64_t it = static_cast<int64_t>(atomicAdd(counter, 1u));
            s_item = it;
            if (it < n_items) {
                s_w = items[it];
                if (s_w.graph < static_cast<uint32_t>(n_graphs)) {
                    s_g = table[s_w.graph];
                    if (ADJ != 0 && s_g.adj_mode != ADJ) {
                        s_w.count = 0;
                        atomicAdd(counter + 1, 1u);
                    }
                } else {
                    s_w.count = 0;  // item names no graph: skipped
                }
            }
        }
        __syncthreads();
        if (s_item >= n_items) break;
        const ps_work w = s_w;
        Counts6 cnt;
        cnt.zero();
        const int sampler = static_cast<int>(w.sampler);
        const bool any = sampler == 0 ? s_g.W > 0 : s_g.Lambda > 0;
        if (any && SPT == 2 && (ADJ == kAdjHash || (ADJ == 0 && s_g.adj_mode == kAdjHash))) {
            for (uint32_t s = threadIdx.x; s < w.count; s += 2 * BLOCK) {
                // a lone last sample repeats its own id as the second, whose class is dropped
                const uint32_t s1 = s + BLOCK < w.count ? s + BLOCK : s;
                int c0, c1;
                batch_sample2_hash(s_g, sampler, w.seed, w.first_id + s, w.first_id + s1, c0, c1);
                cnt.add(c0);
                if (s1 != s) cnt.add(c1);
            }
        } else if (any) {
            for (uint32_t s = threadIdx.x; s < w.count; s += BLOCK) {
                if (ADJ != 0) {
                    cnt.add(batch_sample<ADJ>(s_g, sampler, w.seed, w.first_id + s));
                } else {
                    const int adj = s_g.adj_mode;
                    cnt.add(adj == kAdjVtab   ? batch_sample<kAdjVtab>(s_g, sampler, w.seed, w.first_id + s)
                            : adj == kAdjHash ? batch_sample<kAdjHash>(s_g, sampler, w.seed, w.first_id + s)
                                              : batch_sample<kAdjSearch>(s_g, sampler, w.seed, w.first_id + s));
                }
            }
        }
        flush_counts<BLOCK>(cnt, sampler == 0 ? 6 : 4, hist + 6ull * w.slot);
    }
}

template <int BLOCK, int ADJ, int SPT>
static int launch_batch_t(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                          uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<BLOCK, ADJ, SPT>, BLOCK, 0));
        per_sm = occ > 0 ? occ : 1;
    }
    int64_t blocks = (int64_t)sm_count_of_current_device() * per_sm;
    if (blocks > n_items) blocks = n_items;
    PS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, 2 * sizeof(uint32_t), s));
    k_batch<BLOCK, ADJ, SPT><<<(unsigned)blocks, BLOCK, 0, s>>>(static_cast<const GraphDev *>(d_table), n_graphs,
                                                                d_items, n_items, d_hist, d_counter);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

template <int BLOCK, int ADJ>
static int launch_batch_s(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                          uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    return t.samples_per_thread >= 2
               ? launch_batch_t<BLOCK, ADJ, 2>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s)
               : launch_batch_t<BLOCK, ADJ, 1>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
}

template <int BLOCK>
static int launch_batch_b(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                          uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    switch (table_adjacency(d_table)) {
        case kAdjHash:
            return launch_batch_s<BLOCK, kAdjHash>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case kAdjSearch:
            return launch_batch_s<BLOCK, kAdjSearch>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case kAdjVtab:
            return launch_batch_s<BLOCK, kAdjVtab>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        default:
            return launch_batch_s<BLOCK, 0>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
    }
}

int launch_batch(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                 uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    if (n_items <= 0) return PS_OK;
    switch (t.block_size) {
        case 128: return launch_batch_b<128>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case 256: return launch_batch_b<256>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case 512: return launch_batch_b<512>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case 1024: return launch_batch_b<1024>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        default: return PS_ERR_ARG;
    }
}

}  // namespace ps
