// ps_batch.cu -- ps_batch_sample: one persistent launch over a queue of work
// items drawn from many loaded graphs.  Each block takes an item (a range of
// sample ids of one graph and one sampler), runs it with the same per-sample
// code as the plain launches and adds its class counts to the item's slot.
#include "ps_internal.h"
#include "ps_sample.cuh"

namespace ps {

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
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
                if (s_w.graph < static_cast<uint32_t>(n_graphs)) s_g = table[s_w.graph];
                else s_w.count = 0;  // item names no graph: skipped
            }
        }
        __syncthreads();
        if (s_item >= n_items) break;
        const ps_work w = s_w;
        Counts6 cnt;
        cnt.zero();
        const int adj = s_g.adj_mode;
        if (w.sampler == 0) {
            if (s_g.W > 0)
                for (uint32_t s = threadIdx.x; s < w.count; s += BLOCK)
                    cnt.add(adj == kAdjVtab   ? sample_3path<kAdjVtab>(s_g, w.seed, w.first_id + s)
                            : adj == kAdjHash ? sample_3path<kAdjHash>(s_g, w.seed, w.first_id + s)
                                              : sample_3path<kAdjSearch>(s_g, w.seed, w.first_id + s));
        } else {
            if (s_g.Lambda > 0)
                for (uint32_t s = threadIdx.x; s < w.count; s += BLOCK)
                    cnt.add(adj == kAdjVtab   ? sample_centred<kAdjVtab>(s_g, w.seed, w.first_id + s)
                            : adj == kAdjHash ? sample_centred<kAdjHash>(s_g, w.seed, w.first_id + s)
                                              : sample_centred<kAdjSearch>(s_g, w.seed, w.first_id + s));
        }
        flush_counts<BLOCK>(cnt, w.sampler == 0 ? 6 : 4, hist + 6ull * w.slot);
    }
}

template <int BLOCK>
static int launch_batch_t(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                          uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<BLOCK>, BLOCK, 0));
        per_sm = occ > 0 ? occ : 1;
    }
    int64_t blocks = (int64_t)sm_count_of_current_device() * per_sm;
    if (blocks > n_items) blocks = n_items;
    PS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s));
    k_batch<BLOCK><<<(unsigned)blocks, BLOCK, 0, s>>>(static_cast<const GraphDev *>(d_table), n_graphs,
                                                      d_items, n_items, d_hist, d_counter);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

int launch_batch(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                 uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s) {
    if (n_items <= 0) return PS_OK;
    switch (t.block_size) {
        case 128: return launch_batch_t<128>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case 256: return launch_batch_t<256>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case 512: return launch_batch_t<512>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        case 1024: return launch_batch_t<1024>(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, s);
        default: return PS_ERR_ARG;
    }
}

}  // namespace ps
