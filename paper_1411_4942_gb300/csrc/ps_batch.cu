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

// ADJ = 0: any variant, chosen per item; otherwise the table's only variant.
// counter[0] hands out items; counter[1] counts items skipped because their
// graph does not use the variant this kernel was compiled for.  Registers
// are capped for 1024 resident threads per SM, the plain samplers' occupancy.
template <int BLOCK, int ADJ>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK)
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
        if (any) {
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

template <int BLOCK, int ADJ>
static int launch_batch_t(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                          uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<BLOCK, ADJ>, BLOCK, 0));
        per_sm = occ > 0 ? occ : 1;
    }
    int64_t blocks = (int64_t)sm_count_of_current_device() * per_sm;
    if (blocks > n_items) blocks = n_items;
    PS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, 2 * sizeof(uint32_t), s));
    k_batch<BLOCK, ADJ><<<(unsigned)blocks, BLOCK, 0, s>>>(static_cast<const GraphDev *>(d_table), n_graphs,
                                                           d_items, n_items, d_hist, d_counter);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

template <int BLOCK>
static int launch_batch_b(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                          uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    switch (table_adjacency(d_table)) {
        case kAdjHash:
            return launch_batch_t<BLOCK, kAdjHash>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case kAdjSearch:
            return launch_batch_t<BLOCK, kAdjSearch>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case kAdjVtab:
            return launch_batch_t<BLOCK, kAdjVtab>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        default:
            return launch_batch_t<BLOCK, 0>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
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
