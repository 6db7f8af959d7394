// ps_sample.cu -- ps_sample_3paths / ps_sample_centered: persistent
// grid-stride kernels over sample ids, each thread drawing and classifying
// samples independently and counting classes in registers.
#include "ps_internal.h"
#include "ps_sample.cuh"

namespace ps {

template <int SAMPLER, int BLOCK, int ADJ>
__global__ void __launch_bounds__(BLOCK, sample_min_blocks<BLOCK>())
k_sample(GraphDev g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *hist) {
    Counts6 cnt;
    cnt.zero();
    const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
    for (uint64_t s = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; s < k; s += stride) {
        const uint64_t id = first_id + s;
        cnt.add(SAMPLER == 0 ? sample_3path<ADJ>(g, seed, id) : sample_centred<ADJ>(g, seed, id));
    }
    flush_counts<BLOCK>(cnt, SAMPLER == 0 ? 6 : 4, hist);
}

template <int SAMPLER, int BLOCK, int ADJ>
static int launch_t(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *hist,
                    cudaStream_t s) {
    int per_sm = g->tune.blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample<SAMPLER, BLOCK, ADJ>, BLOCK, 0));
        per_sm = occ > 0 ? occ : 1;
    }
    const uint64_t full = (uint64_t)g->sm_count * per_sm;
    // per-thread counters are 32-bit: keep every thread under 2^30 samples per launch
    const uint64_t max_chunk = full * BLOCK * (1ull << 30);
    while (k > 0) {
        const uint64_t kk = k < max_chunk ? k : max_chunk;
        uint64_t blocks = (kk + BLOCK - 1) / BLOCK;
        if (blocks > full) blocks = full;
        k_sample<SAMPLER, BLOCK, ADJ><<<(unsigned)blocks, BLOCK, 0, s>>>(g->dev, kk, seed, first_id, hist);
        PS_LAUNCH_CHECK();
        k -= kk;
        first_id += kk;
    }
    return PS_OK;
}

template <int BLOCK>
static int launch_b(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id,
                    uint64_t *hist, cudaStream_t s) {
    if (g->tune.adj_mode == kAdjVtab)
        return sampler == 0 ? launch_t<0, BLOCK, kAdjVtab>(g, k, seed, first_id, hist, s)
                            : launch_t<1, BLOCK, kAdjVtab>(g, k, seed, first_id, hist, s);
    if (g->tune.adj_mode == kAdjHash)
        return sampler == 0 ? launch_t<0, BLOCK, kAdjHash>(g, k, seed, first_id, hist, s)
                            : launch_t<1, BLOCK, kAdjHash>(g, k, seed, first_id, hist, s);
    return sampler == 0 ? launch_t<0, BLOCK, kAdjSearch>(g, k, seed, first_id, hist, s)
                        : launch_t<1, BLOCK, kAdjSearch>(g, k, seed, first_id, hist, s);
}

int launch_sampler(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id,
                   uint64_t *d_hist, cudaStream_t s) {
    switch (g->tune.block_size) {
        case 128: return launch_b<128>(g, sampler, k, seed, first_id, d_hist, s);
        case 256: return launch_b<256>(g, sampler, k, seed, first_id, d_hist, s);
        case 512: return launch_b<512>(g, sampler, k, seed, first_id, d_hist, s);
        case 1024: return launch_b<1024>(g, sampler, k, seed, first_id, d_hist, s);
        default: return PS_ERR_ARG;
    }
}

}  // namespace ps
