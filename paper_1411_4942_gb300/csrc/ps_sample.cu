// ps_sample.cu -- ps_sample_3paths / ps_sample_centered: persistent
// grid-stride kernels over sample ids, each thread drawing and classifying
// samples independently and counting classes in registers.
#include "ps_internal.h"
#include "ps_sample.cuh"

namespace ps {

template <int SAMPLER, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_sample(GraphDev g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *hist) {
    Counts6 cnt;
    cnt.zero();
    const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
    for (uint64_t s = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; s < k; s += stride) {
        const uint64_t id = first_id + s;
        cnt.add(SAMPLER == 0 ? sample_3path(g, seed, id) : sample_centred(g, seed, id));
    }
    flush_counts<BLOCK>(cnt, SAMPLER == 0 ? 6 : 4, hist);
}

template <int SAMPLER, int BLOCK>
static int launch_t(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *hist,
                    cudaStream_t s) {
    int per_sm = g->tune.blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample<SAMPLER, BLOCK>, BLOCK, 0));
        per_sm = occ > 0 ? occ : 1;
    }
    const uint64_t full = (uint64_t)g->sm_count * per_sm;
    // per-thread counters are 32-bit: keep every thread under 2^31 samples per launch
    const uint64_t max_chunk = full * BLOCK * (1ull << 30);
    while (k > 0) {
        const uint64_t kk = k < max_chunk ? k : max_chunk;
        uint64_t blocks = (kk + BLOCK - 1) / BLOCK;
        if (blocks > full) blocks = full;
        k_sample<SAMPLER, BLOCK><<<(unsigned)blocks, BLOCK, 0, s>>>(g->dev, kk, seed, first_id, hist);
        PS_LAUNCH_CHECK();
        k -= kk;
        first_id += kk;
    }
    return PS_OK;
}

int launch_sampler(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id,
                   uint64_t *d_hist, cudaStream_t s) {
    const int bs = g->tune.block_size;
#define PS_SAMPLER_CASE(B)                                                       \
    if (bs == B)                                                                 \
        return sampler == 0 ? launch_t<0, B>(g, k, seed, first_id, d_hist, s)    \
                            : launch_t<1, B>(g, k, seed, first_id, d_hist, s);
    PS_SAMPLER_CASE(128)
    PS_SAMPLER_CASE(256)
    PS_SAMPLER_CASE(512)
    PS_SAMPLER_CASE(1024)
#undef PS_SAMPLER_CASE
    return PS_ERR_ARG;
}

}  // namespace ps
