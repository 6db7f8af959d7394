// ps_probe.cu -- ps_l2_read_probe: a measurement utility, not part of the
// method.  It reads a caller's buffer over and over with loads that are
// cached in L2 only (ld.global.cg), so for a buffer that fits in L2 the
// caller's event timing gives the L2 read bandwidth against which a graph
// small enough to stay in L2 is reported.
#include "ps_internal.h"

namespace ps {
namespace {

// Block b reads its own slice of the buffer `passes` times (the slices
// split the buffer evenly, so every byte is read `passes` times in all).
__global__ void __launch_bounds__(512)
k_l2_read(const int4 *__restrict__ buf, int64_t n16, int passes, unsigned long long *sink) {
    const int64_t per = (n16 + gridDim.x - 1) / gridDim.x;
    const int64_t lo = per * blockIdx.x;
    const int64_t hi = lo + per < n16 ? lo + per : n16;
    unsigned int x = 0;
    for (int p = 0; p < passes; p++) {
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const int4 v = __ldcg(buf + i);
            x ^= static_cast<unsigned int>(v.x ^ v.y ^ v.z ^ v.w);
        }
    }
    if (x) atomicXor(sink, static_cast<unsigned long long>(x));
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" int ps_l2_read_probe(const void *d_buf, uint64_t bytes, int32_t passes, uint64_t *d_sink,
                                ps_stream_t stream) {
    if (!d_buf || !d_sink || bytes == 0 || (bytes & 15u) != 0 || passes <= 0 ||
        (reinterpret_cast<uintptr_t>(d_buf) & 15u) != 0)
        return PS_ERR_ARG;
    int dev = 0, sms = 0;
    PS_CUDA_TRY(cudaGetDevice(&dev));
    PS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t n16 = static_cast<int64_t>(bytes / 16);
    int64_t blocks = static_cast<int64_t>(sms) * 4;
    if (blocks > n16) blocks = n16;
    k_l2_read<<<(unsigned)blocks, 512, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const int4 *>(d_buf), n16, passes, reinterpret_cast<unsigned long long *>(d_sink));
    PS_LAUNCH_CHECK();
    return PS_OK;
}
